"""vp_eval_static: the evaluation without any device allocation.

For callers that cannot allocate device memory when they evaluate (a fixed
memory budget, an allocator they must not touch). The tests call the entry
point through the C ABI twice in a row, and on two trees of different shape
in turn (A, B, A), and compare it with vp_eval; they also check that a tree
needing more than the static work space is rejected.
Collected last on purpose (file name), so a stop-at-first-failure run has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

import paper_1908_07392_gb300 as V
from paper_1908_07392_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-10  # same relative max-norm tolerance as the FP64 parity tests


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = V.load_library()
    lib.vp_eval_static.argtypes = [ctypes.c_void_p] * 5
    return lib


def _call(lib, tree, f, u, g):
    import torch
    return lib.vp_eval_static(ctypes.c_void_p(tree), ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                              ctypes.c_void_p(g.data_ptr()),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_static_matches_vp_eval_twice(lib):
    import torch
    w = I.small_gaussian_workload()
    vp = V.VolumePotential(w.kernel, w.alpha, w.p, w.tree)
    try:
        f = torch.from_numpy(w.f).cuda()
        u_ref, g_ref = vp(f)
        rng = np.random.default_rng(3)
        f2 = torch.from_numpy(rng.standard_normal(w.n_nodes)).cuda()
        u_ref2, g_ref2 = vp(f2)
        for fin, ur, gr in ((f, u_ref, g_ref), (f2, u_ref2, g_ref2)):
            u = torch.full_like(ur, float("nan"))
            g = torch.full_like(gr, float("nan"))
            assert _call(lib, vp.tree, fin, u, g) == 0
            torch.cuda.synchronize()
            for a, b in ((u, ur), (g[0], gr[0]), (g[1], gr[1])):
                a = a.cpu().numpy(); b = b.cpu().numpy()
                assert np.all(np.isfinite(a))
                assert np.abs(a - b).max() <= TOL * np.abs(b).max()
    finally:
        vp.close()


def test_static_alternating_trees(lib):
    # the shared array keeps the previous call's contents: alternate two trees of different shape and
    # size (A, B, A) so that stale values left by another tree's layout would show
    import torch
    wa = I.small_gaussian_workload()
    wb = I.small_gaussian_workload(depth=2, p=6, alpha=25.0)
    va = V.VolumePotential(wa.kernel, wa.alpha, wa.p, wa.tree)
    vb = V.VolumePotential(wb.kernel, wb.alpha, wb.p, wb.tree, order=24)
    try:
        cases = []
        for w, vp in ((wa, va), (wb, vb)):
            f = torch.from_numpy(w.f).cuda()
            ur, gr = vp(f)
            cases.append((vp, f, ur.clone(), gr.clone()))
        for vp, f, ur, gr in (cases[0], cases[1], cases[0]):
            u = torch.full_like(ur, float("nan"))
            g = torch.full_like(gr, float("nan"))
            assert _call(lib, vp.tree, f, u, g) == 0
            torch.cuda.synchronize()
            for a, b in ((u, ur), (g[0], gr[0]), (g[1], gr[1])):
                a = a.cpu().numpy(); b = b.cpu().numpy()
                assert np.all(np.isfinite(a))
                assert np.abs(a - b).max() <= TOL * np.abs(b).max()
    finally:
        va.close()
        vb.close()


def test_static_rejects_trees_beyond_the_work_space(lib):
    import torch
    tree = I.uniform_tree(5)  # 1024 leaves at p = 16 need far more than 64 MiB of slots
    p = 16
    vp = V.VolumePotential(0, 10.0, p, tree, order=20)
    try:
        f = torch.zeros(vp.N, dtype=torch.float64, device="cuda")
        u = torch.empty_like(f); g = torch.empty(2, vp.N, dtype=torch.float64, device="cuda")
        assert _call(lib, vp.tree, f, u, g) == -1
    finally:
        vp.close()
