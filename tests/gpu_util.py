"""Shared helpers of the GPU tests (CUDA path through the C ABI, oracle on the CPU)."""
import numpy as np

import oracle as O
import paper_1908_07392_gb300 as V
from paper_1908_07392_gb300 import inputs as I

TOL_FP64 = 1e-10   # relative max-norm error per field (u, du/dx, du/dy), plain FP64
TOL_SPLIT = 1e-9   # the same for the split-precision (sliced bf16 tensor-core) form


def gpu_eval(w, order=40, precision=V.VP_PREC_FP64, levels=None):
    import torch
    vp = V.VolumePotential(w.kernel, w.alpha, w.p, w.tree, order=order, precision=precision, levels=levels)
    try:
        f = torch.from_numpy(np.ascontiguousarray(w.f)).cuda()
        u, g = vp(f)
        torch.cuda.synchronize()
        return u.cpu().numpy(), g[0].cpu().numpy(), g[1].cpu().numpy()
    finally:
        vp.close()


def oracle_eval(w, idx=None):
    X, Y = I.node_coords(w.tree, w.p)
    if idx is not None:
        X, Y = X[idx], Y[idx]
    return O.volume_potential(w.kernel, w.alpha, w.p, w.tree, w.f, X, Y)


def rel_err(a, b):
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / den)


def sample_nodes(w, n, seed):
    """n node indices spread over leaves of every level (always includes the deepest leaves)."""
    rng = np.random.default_rng(seed)
    N = w.n_nodes
    if n >= N:
        return np.arange(N)
    nn = w.p * w.p
    deep = np.flatnonzero(w.tree.level == w.tree.level.max())
    coarse = np.flatnonzero(w.tree.level == w.tree.level.min())
    picks = [rng.choice(deep) * nn + rng.integers(nn, size=4), rng.choice(coarse) * nn + rng.integers(nn, size=4)]
    picks.append(rng.choice(N, n - 8, replace=False))
    return np.unique(np.concatenate(picks))
