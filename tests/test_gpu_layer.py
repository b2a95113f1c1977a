"""The layer potential u^H = D[mu] at the volume nodes (vp_layer_*) through the C ABI.

Against the oracle's direct double-layer sum at every node (uniform and adaptive trees, the
latter with W and X lists; FP64 and split-precision tables), against the direct sum on the GPU
at a medium size, and against an exact solution: boundary data from exterior stokeslets, the
density from GMRES, u^H inside the star against the stokeslet field (Sec. 2.2)."""
import numpy as np
import pytest

import paper_1908_07392_gb300 as V
from paper_1908_07392_gb300 import inputs as I
from oracle import layer_oracle as LO
from gpu_util import TOL_FP64, TOL_SPLIT, rel_err

pytestmark = pytest.mark.gpu

STAR = dict(R=1.0, A=0.3, k=5, phase=0.4)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    V.load_library()


def density(t):
    return np.stack([np.cos(2 * t) + 0.3 * np.sin(t), np.sin(3 * t) - 0.2 + 0.1 * np.cos(t)], axis=-1)


def gpu_layer(tree, p, alpha, src, mu, precision, order=40):
    import torch
    vp = V.VolumePotential(V.VP_KERNEL_MBIHARMONIC, alpha, p, tree, order=order, precision=precision)
    layer = V.vp_layer_create(vp.tree, np.asarray(src))
    try:
        m = torch.from_numpy(np.ascontiguousarray(mu, dtype=np.float64)).cuda()
        u = torch.full((2, vp.N), float("nan"), dtype=torch.float64, device="cuda")
        V.vp_layer_eval(layer, m, u)
        u2 = torch.full_like(u, float("nan"))
        V.vp_layer_eval(layer, m, u2)  # a second call on the same buffers gives the same values
        torch.cuda.synchronize()
        assert torch.equal(u, u2)
        xy = vp.nodes().cpu().numpy()
        return u.cpu().numpy(), xy
    finally:
        V.vp_layer_free(layer)
        vp.close()


def check_against_oracle(tree, p, alpha, n_panels, precision, tol):
    x, y, nx, ny, w, t = LO.star_nodes(n_panels=n_panels, **STAR)
    src = np.stack([x, y, nx, ny, w])
    mu = density(t)
    u, xy = gpu_layer(tree, p, alpha, src, mu, precision)
    ref = LO.layer_potential(alpha, (x, y, nx, ny, w), mu, xy[0], xy[1])
    errs = [rel_err(u[a], ref[a]) for a in range(2)]
    assert max(errs) < tol, errs
    return errs


@pytest.mark.parametrize("precision,tol", [(V.VP_PREC_FP64, TOL_FP64), (V.VP_PREC_SPLIT, TOL_SPLIT)])
def test_uniform_tree_every_node(precision, tol):
    # depth 4, p = 8 (16,384 nodes), alpha h = 5.6: both channels of the far field active
    check_against_oracle(I.uniform_tree(4, side=3.0), 8, 30.0, 32, precision, tol)


@pytest.mark.parametrize("precision,tol", [(V.VP_PREC_FP64, TOL_FP64), (V.VP_PREC_SPLIT, TOL_SPLIT)])
def test_adaptive_tree_every_node(precision, tol):
    # random balanced tree (W and X lists), levels 2-5, p = 6
    rng = np.random.default_rng(11)
    tree = I.random_balanced_tree(rng, 60, 5, side=3.0, min_depth=2)
    check_against_oracle(tree, 6, 20.0, 24, precision, tol)


def test_coarse_tree_all_near():
    # leaves at levels 1-2 only: every pair is adjacent or handled at level 2
    check_against_oracle(I.uniform_tree(2, side=3.0), 6, 5.0, 16, V.VP_PREC_FP64, TOL_FP64)


def test_against_gpu_direct_sum():
    # the BIE object's own nodes and a GMRES-free density: the tree evaluation against the direct
    # sum over the boundary on the GPU (bie_eval) at every node of a depth-5 tree (262k nodes)
    import torch
    alpha = 316.0
    b = V.BIE(alpha, phase=STAR["phase"], n_panels=64)
    try:
        nodes = b.nodes.cpu().numpy()
        mu = density(nodes[6])
        tree = I.uniform_tree(5, side=3.0)
        for precision, tol in ((V.VP_PREC_FP64, TOL_FP64), (V.VP_PREC_SPLIT, TOL_SPLIT)):
            u, xy = gpu_layer(tree, 16, alpha, nodes[:5], mu, precision)
            m = torch.from_numpy(np.ascontiguousarray(mu).reshape(-1)).cuda()
            txy = torch.from_numpy(np.ascontiguousarray(xy)).cuda()
            ref = b.eval(m, txy).cpu().numpy()
            errs = [rel_err(u[a], ref[a]) for a in range(2)]
            assert max(errs) < tol, (precision, errs)
    finally:
        b.close()


def test_exact_solution_inside_the_star():
    # exterior stokeslets give boundary data g; GMRES gives mu; u^H = D[mu] must reproduce the
    # stokeslet field inside the star, away from the boundary (the plain quadrature's near-boundary
    # error is the subject of Sec. 4)
    import torch
    alpha, n_panels = 316.0, 256
    wl = I.step_workload(seed=5, depth=6)
    b = V.BIE(alpha, R=1.0, A=0.3, k=5, phase=wl.phi, n_panels=n_panels)
    try:
        forcing = I.moving_stokeslets(5)
        src_pts, strengths = forcing(0.0)
        nodes = b.nodes
        s = torch.from_numpy(np.ascontiguousarray(src_pts, dtype=np.float64)).cuda()
        f = torch.from_numpy(np.ascontiguousarray(strengths, dtype=np.float64)).cuda()
        gb = V.bie_stokeslets(alpha, s, f, nodes[:2].contiguous())
        g = gb.t().reshape(-1).contiguous()
        mu, it, rr = b.solve(g, None, 1e-13)
        assert rr < 1e-12
        vp = V.VolumePotential(V.VP_KERNEL_MBIHARMONIC, alpha, 16, wl.tree, precision=V.VP_PREC_SPLIT)
        layer = V.vp_layer_create(vp.tree, nodes[:5].cpu().numpy())
        try:
            u = torch.empty(2, vp.N, dtype=torch.float64, device="cuda")
            V.vp_layer_eval(layer, mu, u)
            xy = vp.nodes()
            exact = V.bie_stokeslets(alpha, s, f, xy)
            torch.cuda.synchronize()
        finally:
            V.vp_layer_free(layer)
            vp.close()
        X, Y = xy[0].cpu().numpy(), xy[1].cpu().numpy()
        rho, th = np.hypot(X, Y), np.arctan2(Y, X)
        inside = rho < 1.0 + 0.3 * np.cos(5 * th + wl.phi) - 0.05
        ue, uu = exact.cpu().numpy(), u.cpu().numpy()
        assert inside.sum() > 100000
        errs = [np.abs(uu[a][inside] - ue[a][inside]).max() / np.abs(ue[:, inside]).max() for a in range(2)]
        assert max(errs) < 1e-9, errs
    finally:
        b.close()
