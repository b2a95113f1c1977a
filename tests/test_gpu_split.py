"""Split-precision form (sliced bf16 operands on the tensor cores) against the FP64 oracle and FP64 path."""
import numpy as np
import pytest

import paper_1908_07392_gb300 as V
from paper_1908_07392_gb300 import inputs as I
from gpu_util import TOL_FP64, TOL_SPLIT, gpu_eval, oracle_eval, rel_err, sample_nodes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    V.load_library()


def _errs(w, idx, precision):
    u, ux, uy = gpu_eval(w, precision=precision)
    ou, oux, ouy = oracle_eval(w, idx)
    return (rel_err(u[idx], ou), rel_err(ux[idx], oux), rel_err(uy[idx], ouy)), (u, ux, uy)


def test_split_gaussian_uniform_depth3_all_nodes():
    w = I.small_gaussian_workload()
    idx = np.arange(w.n_nodes)
    errs, _ = _errs(w, idx, V.VP_PREC_SPLIT)
    assert max(errs) < TOL_SPLIT, errs


@pytest.mark.parametrize("kernel,alpha,p", [(0, 10.0, 8), (1, 30.0, 8), (1, 300.0, 16), (0, 1000.0, 12)])
def test_split_random_adaptive_trees(kernel, alpha, p):
    rng = np.random.default_rng(100 + int(alpha) + kernel)
    tree = I.random_balanced_tree(rng, 30, 6, side=3.0, min_depth=2)
    X, Y = I.node_coords(tree, p)
    fn = I.gaussian_sum(rng.uniform(-0.8, 0.8, (4, 2)), rng.uniform(0.1, 0.4, 4), rng.uniform(-1, 1, 4))
    w = I.Workload("rand", kernel, alpha, p, tree, fn(X, Y))
    idx = sample_nodes(w, 300, 3)
    errs, _ = _errs(w, idx, V.VP_PREC_SPLIT)
    assert max(errs) < TOL_SPLIT, errs


def test_split_close_to_fp64_everywhere():
    # at every node, not only sampled ones: split and FP64 forms of the same tree agree
    rng = np.random.default_rng(7)
    tree = I.random_balanced_tree(rng, 60, 7, side=3.0, min_depth=2)
    p = 8
    X, Y = I.node_coords(tree, p)
    f = np.cos(3 * X) * np.exp(-Y * Y) + 0.1
    w = I.Workload("rand", 1, 100.0, p, tree, f)
    a = gpu_eval(w, precision=V.VP_PREC_FP64)
    b = gpu_eval(w, precision=V.VP_PREC_SPLIT)
    for x, y in zip(a, b):
        assert rel_err(y, x) < TOL_SPLIT
    # zero source leaves (exponent of an all-zero vector) give exact zeros where nothing reaches
    f0 = np.zeros_like(f)
    z = gpu_eval(I.Workload("zero", 1, 100.0, p, tree, f0), precision=V.VP_PREC_SPLIT)
    assert all(np.all(v == 0.0) for v in z)


def test_split_rejected_by_the_static_entry_point():
    import ctypes
    import torch
    w = I.small_gaussian_workload(depth=2, p=6)
    vp = V.VolumePotential(w.kernel, w.alpha, w.p, w.tree, precision=V.VP_PREC_SPLIT)
    try:
        lib = V.load_library()
        f = torch.from_numpy(w.f).cuda()
        u = torch.empty_like(f); g = torch.empty(2, w.n_nodes, dtype=torch.float64, device="cuda")
        rc = lib.vp_eval_static(ctypes.c_void_p(vp.tree), ctypes.c_void_p(f.data_ptr()),
                                ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(0))
        assert rc == -1
    finally:
        vp.close()


@pytest.mark.parametrize("precision", [V.VP_PREC_FP64, V.VP_PREC_SPLIT])
def test_host_entry_point_with_pinned_and_pageable_buffers(precision):
    # page-locked buffers are used in place (outputs written by the reduction, split-form input read
    # by the slicing kernel); pageable ones go through staging copies; both give the device path's bits
    import torch
    w = I.small_gaussian_workload()
    vp = V.VolumePotential(w.kernel, w.alpha, w.p, w.tree, precision=precision)
    try:
        f = torch.from_numpy(np.ascontiguousarray(w.f))
        u_dev, g_dev = vp(f.cuda())
        torch.cuda.synchronize()
        fp = f.pin_memory()
        up = torch.zeros(w.n_nodes, dtype=torch.float64).pin_memory()
        gp = torch.zeros(2, w.n_nodes, dtype=torch.float64).pin_memory()
        V.vp_eval_host(vp.tree, fp, up, gp)
        assert torch.equal(up, u_dev.cpu()) and torch.equal(gp, g_dev.cpu())
        un = np.zeros(w.n_nodes); gn = np.zeros((2, w.n_nodes))
        V.vp_eval_host(vp.tree, f.numpy(), un, gn)
        assert np.array_equal(un, u_dev.cpu().numpy()) and np.array_equal(gn, g_dev.cpu().numpy())
    finally:
        vp.close()
