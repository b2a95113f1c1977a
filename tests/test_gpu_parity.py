"""Parity of the CUDA path (through the C ABI) with the FP64 oracle."""
import numpy as np
import pytest

import paper_1908_07392_gb300 as V
from paper_1908_07392_gb300 import inputs as I
from gpu_util import TOL_FP64, gpu_eval, oracle_eval, rel_err, sample_nodes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    V.load_library()


def _check(w, idx=None, tol=TOL_FP64, order=40):
    u, ux, uy = gpu_eval(w, order=order)
    if idx is None:
        idx = np.arange(w.n_nodes)
    ou, oux, ouy = oracle_eval(w, idx)
    errs = (rel_err(u[idx], ou), rel_err(ux[idx], oux), rel_err(uy[idx], ouy))
    assert max(errs) < tol, errs
    return errs


def test_nodes_match_the_layout():
    import torch
    w = I.star_adaptive_workload(seed=3, alpha=30.0, p=8, tol=1e-6, max_depth=6)
    vp = V.VolumePotential(w.kernel, w.alpha, w.p, w.tree)
    try:
        xy = vp.nodes().cpu().numpy()
    finally:
        vp.close()
    X, Y = I.node_coords(w.tree, w.p)
    assert np.abs(xy[0] - X).max() < 1e-14 and np.abs(xy[1] - Y).max() < 1e-14


def test_gaussian_uniform_depth3_all_nodes():
    # 64 leaves, p = 8, alpha = 10, G1: every one of the 4096 nodes
    _check(I.small_gaussian_workload())


@pytest.mark.parametrize("kernel,alpha", [(0, 10.0), (1, 30.0), (0, 300.0), (1, 300.0)])
def test_random_adaptive_trees(kernel, alpha):
    # mixed-level trees exercise the U (coarse/fine), W and X lists
    rng = np.random.default_rng(int(alpha) + kernel)
    tree = I.random_balanced_tree(rng, 40, 6, side=3.0, min_depth=2)
    p = 8
    X, Y = I.node_coords(tree, p)
    fn = I.gaussian_sum(rng.uniform(-0.8, 0.8, (4, 2)), rng.uniform(0.1, 0.4, 4), rng.uniform(-1, 1, 4))
    w = I.Workload("rand", kernel, alpha, p, tree, fn(X, Y))
    _check(w, sample_nodes(w, 400, 1))


def test_p16_modified_biharmonic_adaptive():
    rng = np.random.default_rng(12)
    tree = I.random_balanced_tree(rng, 12, 5, side=3.0, min_depth=2)
    p = 16
    X, Y = I.node_coords(tree, p)
    fn = I.gaussian_sum([[0.2, -0.1], [-0.5, 0.4]], [0.3, 0.15], [1.0, -0.7])
    w = I.Workload("p16", 1, 300.0, p, tree, fn(X, Y))
    _check(w, sample_nodes(w, 200, 2))


@pytest.mark.parametrize("depth", [0, 1, 2])
def test_shallow_trees(depth):
    # a single root leaf (near self only), 4 leaves (no far field), 16 leaves
    w = I.small_gaussian_workload(depth=depth, p=6)
    _check(w)


def test_minimum_p_and_order():
    w = I.small_gaussian_workload(depth=3, p=2)
    u, _, _ = gpu_eval(w, order=4)
    assert np.all(np.isfinite(u))


def test_linearity_and_host_path():
    import torch
    w = I.small_gaussian_workload()
    vp = V.VolumePotential(w.kernel, w.alpha, w.p, w.tree)
    try:
        rng = np.random.default_rng(0)
        f1 = torch.from_numpy(w.f).cuda()
        f2 = torch.from_numpy(rng.standard_normal(w.n_nodes)).cuda()
        u1, g1 = vp(f1)
        u2, g2 = vp(f2)
        u3, g3 = vp(2.0 * f1 - 3.0 * f2)
        assert rel_err((u3).cpu().numpy(), (2 * u1 - 3 * u2).cpu().numpy()) < 1e-13
        assert rel_err((g3).cpu().numpy(), (2 * g1 - 3 * g2).cpu().numpy()) < 1e-13
        # the host-buffer entry point gives the same bits as the device one
        uh = np.zeros(w.n_nodes); gh = np.zeros((2, w.n_nodes))
        V.vp_eval_host(vp.tree, np.ascontiguousarray(w.f), uh, gh)
        assert np.array_equal(uh, u1.cpu().numpy()) and np.array_equal(gh, g1.cpu().numpy())
        # repeated evaluation is deterministic
        u4, _ = vp(f1)
        assert torch.equal(u4, u1)
        ms = V.vp_eval_timed(vp.tree, f1, u4, g1)
        assert len(ms) == V.VP_NSTAGES and all(m >= 0 for m in ms)
        launches, flops = V.vp_tree_stats(vp.tree)
        assert launches > 0 and flops[4] > 0
    finally:
        vp.close()


def test_errors_from_the_device_entry_points():
    t = V.vp_tables_build(0, 10.0, 4, 3, 2.0, 8)
    try:
        with pytest.raises(V.VPError) as e:   # leaf deeper than the tables
            V.vp_tree_upload(t, 0, 0, [4] * 256, np.tile(np.arange(16), 16), np.repeat(np.arange(16), 16))
        assert e.value.code == -3
        # unbalanced: level-3 leaves touching level-1 leaves
        leaves = [(1, 0, 0), (1, 1, 0), (1, 0, 1), (2, 3, 2), (2, 2, 3), (2, 3, 3),
                  (3, 4, 4), (3, 5, 4), (3, 4, 5), (3, 5, 5)]
        lv, xx, yy = (np.array(c) for c in zip(*leaves))
        with pytest.raises(V.VPError) as e:
            V.vp_tree_upload(t, 0, 0, lv, xx, yy)
        assert e.value.code == -2
    finally:
        V.vp_tables_free(t)
    for bad in [dict(kernel=2), dict(alpha=-1.0), dict(p=1), dict(p=17), dict(order=3), dict(levels=-1)]:
        args = dict(kernel=0, alpha=10.0, p=4, levels=2, root_side=2.0, order=8)
        args.update(bad)
        with pytest.raises(V.VPError) as e:
            V.vp_tables_build(**args)
        assert e.value.code == -1


def _quarter_turn_symmetric_tree(seed):
    """An adaptive, 2:1-balanced tree that a quarter turn about the root centre maps onto itself:
    random level-2 and level-3 splits, closed under the rotation (l, ix, iy) -> (l, 2^l-1-iy, ix)."""
    rng = np.random.default_rng(seed)
    rot = lambda b: (b[0], (1 << b[0]) - 1 - b[2], b[1])
    leaves = {(2, x, y) for x in range(4) for y in range(4)}
    for level in (2, 3):
        cand = sorted(b for b in leaves if b[0] == level)
        for b in [cand[k] for k in rng.choice(len(cand), 2, replace=False)]:
            orbit = {b, rot(b), rot(rot(b)), rot(rot(rot(b)))}
            for o in orbit:
                if o in leaves:
                    leaves.discard(o)
                    leaves.update(I._children(*o))
        leaves = I.balance_21(leaves)
    assert leaves == {rot(b) for b in leaves}
    return I.tree_from_set(leaves, 0.0, 0.0, 2.0)


@pytest.mark.parametrize("shape,kernel,precision,tol", [
    ("uniform", 0, V.VP_PREC_FP64, 1e-12), ("uniform", 1, V.VP_PREC_FP64, 1e-12),
    ("uniform", 0, V.VP_PREC_SPLIT, 1e-9), ("uniform", 1, V.VP_PREC_SPLIT, 1e-9),
    ("adaptive", 1, V.VP_PREC_FP64, 1e-12), ("adaptive", 0, V.VP_PREC_SPLIT, 1e-9)])
def test_quarter_turn_symmetry(shape, kernel, precision, tol):
    # The kernels are rotation invariant and the tree, centred at the origin, maps onto itself under
    # a quarter turn R, so the source f(R^-1 x) has the potential u(R^-1 x) and the gradient
    # R grad u(R^-1 x) exactly: every relative-position table and expansion operator (near, V, and
    # on the adaptive tree the W and X lists) must agree with its rotated counterpart
    import torch
    p = 8
    tree = I.uniform_tree(3, side=2.0) if shape == "uniform" else _quarter_turn_symmetric_tree(4)
    X, Y = I.node_coords(tree, p)
    rng = np.random.default_rng(8)
    fn = I.gaussian_sum(rng.uniform(-0.6, 0.6, (3, 2)), rng.uniform(0.15, 0.3, 3), rng.uniform(-1, 1, 3))
    f = fn(X, Y)
    # m[k]: index of the node at R^-1 x_k = (y_k, -x_k)
    key = {(round(x, 9), round(y, 9)): k for k, (x, y) in enumerate(zip(X, Y))}
    m = np.array([key[(round(y, 9), round(-x, 9))] for x, y in zip(X, Y)])
    vp = V.VolumePotential(kernel, 10.0, p, tree, precision=precision)
    try:
        u1, g1 = vp(torch.from_numpy(f).cuda())
        u2, g2 = vp(torch.from_numpy(np.ascontiguousarray(f[m])).cuda())
        u1, g1, u2, g2 = (t.cpu().numpy() for t in (u1, g1, u2, g2))
    finally:
        vp.close()
    assert rel_err(u2, u1[m]) < tol
    # R (a, b) = (-b, a)
    assert rel_err(g2[0], -g1[1][m]) < tol and rel_err(g2[1], g1[0][m]) < tol


@pytest.mark.parametrize("kernel", [0, 1])
def test_single_basis_function_and_constant_sources(kernel):
    # f = one Lagrange basis function of one leaf: u at every node is that table column (near leaves)
    # or its expansion (far leaves); f = 1: the sum of all basis functions, the integral of 1
    rng = np.random.default_rng(17)
    tree = I.random_balanced_tree(rng, 6, 4, side=2.0, min_depth=2)
    p = 6
    N = tree.level.size * p * p
    k = int(rng.integers(N))
    for f in (np.eye(1, N, k)[0], np.ones(N)):
        w = I.Workload("basis", kernel, 12.0, p, tree, f)
        _check(w)


@pytest.mark.parametrize("kernel", [0, 1])
def test_far_field_truncation_follows_the_expansion_bound(kernel):
    # the only approximation beyond the tables is the expansion order P: the error against the
    # oracle falls with P like the separation ratio sqrt(2)/(4 - sqrt(2)) ~ 0.547 of the V lists
    rng = np.random.default_rng(23)
    tree = I.random_balanced_tree(rng, 40, 6, side=2.0, min_depth=3)
    p = 6
    X, Y = I.node_coords(tree, p)
    fn = I.gaussian_sum(rng.uniform(-0.6, 0.6, (3, 2)), rng.uniform(0.15, 0.3, 3), rng.uniform(-1, 1, 3))
    w = I.Workload("trunc", kernel, 3.0, p, tree, fn(X, Y))
    idx = sample_nodes(w, 300, 3)
    ou, oux, ouy = oracle_eval(w, idx)
    errs = {}
    for P in (8, 16, 24, 40):
        u, ux, uy = gpu_eval(w, order=P)
        errs[P] = max(rel_err(u[idx], ou), rel_err(ux[idx], oux), rel_err(uy[idx], ouy))
    ratio = np.sqrt(2) / (4 - np.sqrt(2))
    print("error by order", errs)
    for P, e in errs.items():
        assert e <= max(10 * ratio ** P, 1e-11), (P, e)
    assert errs[8] > errs[16] > errs[24]
