"""Parity at the benchmark's full size: the star workload (modified-biharmonic kernel, p = 16,
~10.5M nodes, depth 10), in the launch configuration bench.py times, on sampled targets that the
oracle computes one by one (every leaf level is represented)."""
import numpy as np
import pytest

import paper_1908_07392_gb300 as V
from paper_1908_07392_gb300 import inputs as I
from gpu_util import TOL_FP64, TOL_SPLIT, gpu_eval, oracle_eval, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    V.load_library()


def _sample(w, seed, per_level=3):
    rng = np.random.default_rng(seed)
    nn = w.p * w.p
    idx = []
    for l in np.unique(w.tree.level):
        leaves = np.flatnonzero(w.tree.level == l)
        for leaf in rng.choice(leaves, min(per_level, leaves.size), replace=False):
            idx.append(leaf * nn + rng.integers(nn))
    return np.array(sorted(idx))


def _split_engines(w):
    """Split-precision results with the engines as bench.py chooses them (vp_autotune, then vp_eval
    with the near field overlapping the far field), and with every launch on tcgen05."""
    import torch
    vp = V.VolumePotential(w.kernel, w.alpha, w.p, w.tree, precision=V.VP_PREC_SPLIT)
    try:
        f = torch.from_numpy(np.ascontiguousarray(w.f)).cuda()
        u = torch.empty_like(f); g = torch.empty(2, f.numel(), dtype=torch.float64, device="cuda")
        V.vp_autotune(vp.tree, f, u, g)
        out = {}
        u1, g1 = vp(f)
        torch.cuda.synchronize()
        out["autotuned"] = (u1.cpu().numpy(), g1[0].cpu().numpy(), g1[1].cpu().numpy())
        V.vp_tree_set_engine(vp.tree, V.ENGINE_TCGEN05)
        u2, g2 = vp(f)
        torch.cuda.synchronize()
        V.vp_device_status()
        out["tcgen05"] = (u2.cpu().numpy(), g2[0].cpu().numpy(), g2[1].cpu().numpy())
        return out
    finally:
        vp.close()


@pytest.mark.parametrize("alpha", [300.0, 30.0])
def test_star_workload_sampled(alpha):
    w = I.star_adaptive_workload(seed=2, alpha=alpha, p=16, tol=1e-11, max_depth=10)
    idx = _sample(w, int(alpha))
    ou, oux, ouy = oracle_eval(w, idx)
    results = {"fp64": (gpu_eval(w, precision=V.VP_PREC_FP64), TOL_FP64),
               "split mma.sync": (gpu_eval(w, precision=V.VP_PREC_SPLIT), TOL_SPLIT)}
    for name, r in _split_engines(w).items():
        results["split " + name] = (r, TOL_SPLIT)
    for name, ((u, ux, uy), tol) in results.items():
        errs = (rel_err(u[idx], ou), rel_err(ux[idx], oux), rel_err(uy[idx], ouy))
        assert max(errs) < tol, (name, errs)
