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


@pytest.mark.parametrize("alpha", [300.0, 30.0])
def test_star_workload_sampled(alpha):
    w = I.star_adaptive_workload(seed=2, alpha=alpha, p=16, tol=1e-11, max_depth=10)
    idx = _sample(w, int(alpha))
    ou, oux, ouy = oracle_eval(w, idx)
    for prec, tol in ((V.VP_PREC_FP64, TOL_FP64), (V.VP_PREC_SPLIT, TOL_SPLIT)):
        u, ux, uy = gpu_eval(w, precision=prec)
        errs = (rel_err(u[idx], ou), rel_err(ux[idx], oux), rel_err(uy[idx], ouy))
        assert max(errs) < tol, (prec, errs)
