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


def _near_nodes(xy, n_panels, factor, rng, n_pick):
    """Indices of nodes closer than factor panel lengths to the star (the closest ones and a seeded
    sample of the rest)."""
    x, y, nx, ny, w, t = LO.star_nodes(n_panels=n_panels, **STAR)
    ts = np.linspace(0, 2 * np.pi, 4096, endpoint=False)
    (sx, sy), _ = LO.star(STAR["R"], STAR["A"], STAR["k"], STAR["phase"], ts)
    h = w.reshape(n_panels, 16).sum(axis=1).mean()
    d = np.full(xy.shape[1], np.inf)
    for c0 in range(0, xy.shape[1], 4096):
        sl = slice(c0, c0 + 4096)
        d[sl] = np.sqrt(((xy[0, sl, None] - sx) ** 2 + (xy[1, sl, None] - sy) ** 2).min(axis=1))
    near = np.flatnonzero(d < factor * h)
    order = near[np.argsort(d[near])]
    pick = np.unique(np.concatenate([order[:12], rng.choice(near, min(n_pick, near.size), replace=False)]))
    return pick, d


@pytest.mark.parametrize("precision", [V.VP_PREC_FP64, V.VP_PREC_SPLIT])
def test_near_boundary_correction_against_accurate_oracle(precision):
    # nodes within a panel length of the boundary: the corrected layer potential against the oracle's
    # adaptive quadrature of the panel-interpolated density on the exact curve; the rest against the
    # plain sum (the correction leaves them to the panel rule's accuracy)
    import torch
    alpha, n_panels = 30.0, 48
    tree = I.uniform_tree(5, side=3.0)
    x, y, nx, ny, w, t = LO.star_nodes(n_panels=n_panels, **STAR)
    mu = density(t)
    vp = V.VolumePotential(V.VP_KERNEL_MBIHARMONIC, alpha, 8, tree, precision=precision)
    layer = V.vp_layer_create(vp.tree, np.stack([x, y, nx, ny, w]))
    try:
        npairs = V.vp_layer_near_star(layer, STAR["R"], STAR["A"], STAR["k"], STAR["phase"], n_panels, 1.2)
        assert npairs > 1000
        u = torch.empty(2, vp.N, dtype=torch.float64, device="cuda")
        V.vp_layer_eval(layer, torch.from_numpy(np.ascontiguousarray(mu)).cuda(), u)
        torch.cuda.synchronize()
        u = u.cpu().numpy()
        xy = vp.nodes().cpu().numpy()
    finally:
        V.vp_layer_free(layer)
        vp.close()
    pick, d = _near_nodes(xy, n_panels, 0.7, np.random.default_rng(3), 30)
    ref = LO.layer_potential_accurate(alpha, STAR, n_panels, mu, xy[0, pick], xy[1, pick], near=1.2)
    scale = np.abs(ref).max()
    errs = [np.abs(u[a, pick] - ref[a]).max() / scale for a in range(2)]
    tol = TOL_FP64 if precision == V.VP_PREC_FP64 else TOL_SPLIT
    assert max(errs) < tol, (errs, d[pick].min())
    far = np.flatnonzero(d > 2.0 * w.reshape(n_panels, 16).sum(axis=1).max())
    far = np.random.default_rng(5).choice(far, 400, replace=False)
    reff = LO.layer_potential(alpha, (x, y, nx, ny, w), mu, xy[0, far], xy[1, far])
    assert max(rel_err(u[a, far], reff[a]) for a in range(2)) < tol


def test_exact_solution_up_to_the_boundary():
    # with the near-boundary correction the exterior-stokeslet field is reproduced at every node inside
    # the star, however close to the boundary (alpha h_panel = 12 > 4.5); the plain sum is not
    import torch
    alpha, n_panels = 316.0, 256
    wl = I.step_workload(seed=5, depth=6)
    b = V.BIE(alpha, R=1.0, A=0.3, k=5, phase=wl.phi, n_panels=n_panels)
    try:
        src_pts, strengths = I.moving_stokeslets(5)(0.0)
        s = torch.from_numpy(np.ascontiguousarray(src_pts, dtype=np.float64)).cuda()
        f = torch.from_numpy(np.ascontiguousarray(strengths, dtype=np.float64)).cuda()
        nodes = b.nodes
        g = V.bie_stokeslets(alpha, s, f, nodes[:2].contiguous()).t().reshape(-1).contiguous()
        mu, it, rr = b.solve(g, None, 1e-13)
        vp = V.VolumePotential(V.VP_KERNEL_MBIHARMONIC, alpha, 16, wl.tree, precision=V.VP_PREC_SPLIT)
        plain = V.vp_layer_create(vp.tree, nodes[:5].cpu().numpy())
        corr = V.vp_layer_create(vp.tree, nodes[:5].cpu().numpy())
        try:
            V.vp_layer_near_star(corr, 1.0, 0.3, 5, wl.phi, n_panels, 1.2)
            up = torch.empty(2, vp.N, dtype=torch.float64, device="cuda")
            uc = torch.empty_like(up)
            V.vp_layer_eval(plain, mu, up)
            V.vp_layer_eval(corr, mu, uc)
            xy = vp.nodes()
            exact = V.bie_stokeslets(alpha, s, f, xy)
            torch.cuda.synchronize()
        finally:
            V.vp_layer_free(plain)
            V.vp_layer_free(corr)
            vp.close()
        X, Y = xy[0].cpu().numpy(), xy[1].cpu().numpy()
        inside = np.hypot(X, Y) < 1.0 + 0.3 * np.cos(5 * np.arctan2(Y, X) + wl.phi)
        ue, upl, uco = exact.cpu().numpy(), up.cpu().numpy(), uc.cpu().numpy()
        scale = np.abs(ue[:, inside]).max()
        err_c = max(np.abs(uco[a][inside] - ue[a][inside]).max() for a in range(2)) / scale
        err_p = max(np.abs(upl[a][inside] - ue[a][inside]).max() for a in range(2)) / scale
        assert err_c < 1e-9, (err_c, err_p)
        assert err_p > 1e3 * err_c
    finally:
        b.close()
