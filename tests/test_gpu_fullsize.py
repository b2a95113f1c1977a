"""Parity at the benchmark's full size: the star workload (modified-biharmonic kernel, p = 16,
~10.5M nodes, depth 10), in the launch configuration bench.py times.

Against the oracle on 200 targets chosen where mistakes would show: nodes on the outer ring of
leaves that touch a leaf of another level (coarse/fine near tables, W and X lists), the outermost
nodes of the deepest leaves (the blend band), leaf corners, and nodes of every level. The split
form is also compared with the FP64 form at every node (the FP64 form being pinned to the oracle)."""
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


def _split_engines(w):
    """Split-precision results with the engines as bench.py chooses them (vp_autotune, then vp_eval
    with the near field overlapping the far field), and with every launch on either tcgen05 engine."""
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
        V.vp_tree_set_engine(vp.tree, V.ENGINE_TCGEN05_N64)
        u3, g3 = vp(f)
        torch.cuda.synchronize()
        V.vp_device_status()
        out["tcgen05_n64"] = (u3.cpu().numpy(), g3[0].cpu().numpy(), g3[1].cpu().numpy())
        V.vp_tree_set_engine(vp.tree, V.ENGINE_TCGEN05_T)
        u4, g4 = vp(f)
        torch.cuda.synchronize()
        V.vp_device_status()
        out["tcgen05_t"] = (u4.cpu().numpy(), g4[0].cpu().numpy(), g4[1].cpu().numpy())
        return out
    finally:
        vp.close()


def _transition_leaves(w):
    """Leaves with an adjacent leaf (edge or corner) of another level."""
    t = w.tree
    L = int(t.level.max())
    dim = 1 << L
    lvmap = np.empty((dim + 2, dim + 2), np.int8)
    lvmap[:] = -1
    for lv, x, y in zip(t.level, t.ix, t.iy):
        sh = L - lv
        lvmap[1 + (y << sh):1 + ((y + 1) << sh), 1 + (x << sh):1 + ((x + 1) << sh)] = lv
    out = []
    for k, (lv, x, y) in enumerate(zip(t.level, t.ix, t.iy)):
        sh = L - lv
        x0, x1, y0, y1 = x << sh, (x + 1) << sh, y << sh, (y + 1) << sh
        ring = np.concatenate([lvmap[y0, x0:x1 + 2], lvmap[y1 + 1, x0:x1 + 2],
                               lvmap[y0:y1 + 2, x0], lvmap[y0:y1 + 2, x1 + 1]])
        ring = ring[ring >= 0]
        if np.any(ring != lv):
            out.append(k)
    return np.array(out)


def _targeted_sample(w, seed, n=200):
    """n node indices: outer-ring nodes of transition leaves (80), outer-ring nodes of the deepest
    leaves (60), leaf corners (30), and nodes of every level (the rest)."""
    rng = np.random.default_rng(seed)
    p, nn = w.p, w.p * w.p
    ring = np.array([j * p + i for j in range(p) for i in range(p) if i in (0, p - 1) or j in (0, p - 1)])
    corners = np.array([0, p - 1, (p - 1) * p, nn - 1])
    trans = _transition_leaves(w)
    deep = np.flatnonzero(w.tree.level == w.tree.level.max())
    picks = [rng.choice(trans, 80, replace=trans.size < 80) * nn + rng.choice(ring, 80),
             rng.choice(deep, 60, replace=deep.size < 60) * nn + rng.choice(ring, 60),
             rng.choice(w.tree.n_leaves, 30) * nn + rng.choice(corners, 30)]
    levels = np.unique(w.tree.level)
    rest = n - sum(x.size for x in picks)
    for k in range(rest):
        leaves = np.flatnonzero(w.tree.level == levels[k % levels.size])
        picks.append(np.array([rng.choice(leaves) * nn + rng.integers(nn)]))
    idx = np.unique(np.concatenate(picks))
    while idx.size < n:  # duplicates removed: top up with random nodes
        idx = np.unique(np.concatenate([idx, rng.choice(w.n_nodes, n - idx.size)]))
    return idx, trans.size


@pytest.mark.parametrize("alpha", [300.0, 30.0])
def test_star_workload_sampled(alpha):
    w = I.star_adaptive_workload(seed=2, alpha=alpha, p=16, tol=1e-11, max_depth=10)
    idx, n_trans = _targeted_sample(w, int(alpha))
    assert idx.size >= 200 and n_trans > 100
    ou, oux, ouy = oracle_eval(w, idx)
    results = {"fp64": (gpu_eval(w, precision=V.VP_PREC_FP64), TOL_FP64),
               "split mma.sync": (gpu_eval(w, precision=V.VP_PREC_SPLIT), TOL_SPLIT)}
    for name, r in _split_engines(w).items():
        results["split " + name] = (r, TOL_SPLIT)
    for name, ((u, ux, uy), tol) in results.items():
        errs = (rel_err(u[idx], ou), rel_err(ux[idx], oux), rel_err(uy[idx], ouy))
        assert max(errs) < tol, (name, errs)
    # every node: each split result against the FP64 result (pinned to the oracle above)
    f64 = results["fp64"][0]
    for name, ((u, ux, uy), _) in results.items():
        if name == "fp64":
            continue
        errs = (rel_err(u, f64[0]), rel_err(ux, f64[1]), rel_err(uy, f64[2]))
        assert max(errs) < TOL_SPLIT, (name, "every node vs fp64", errs)
