"""Leaf interpolation off the grid (vp_tree_interp) and the boundary trace of the particular solution."""
import numpy as np
import pytest

import oracle as O
import paper_1908_07392_gb300 as V
from paper_1908_07392_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    V.load_library()


def _poly(c, X, Y):
    return sum(c[a, b] * X ** a * Y ** b for a in range(c.shape[0]) for b in range(c.shape[1]))


def test_interp_reproduces_leaf_polynomials():
    # a polynomial of degree p-1 in each variable is its own leaf interpolant on every leaf, so the
    # interpolated values are exact up to rounding, on leaf edges and at the root corners too
    import torch
    p = 7
    rng = np.random.default_rng(3)
    tree = I.random_balanced_tree(rng, 40, 6, cx=0.3, cy=-0.2, side=2.5)
    vp = V.VolumePotential(I.KERNEL_MHELMHOLTZ, 10.0, p, tree)
    try:
        xy = vp.nodes().cpu().numpy()
        c1 = rng.uniform(-1, 1, (p, p)); c2 = rng.uniform(-1, 1, (p, p))
        F = np.stack([_poly(c1, xy[0], xy[1]), _poly(c2, xy[0], xy[1])])
        x0, y0 = tree.cx - tree.side / 2, tree.cy - tree.side / 2
        pts = [rng.uniform(0, 1, (2, 300))]
        # leaf corners and edge midpoints of the finest grid, and the four root corners
        g = rng.integers(0, 1 << tree.max_level + 1, (2, 100)) / float(1 << tree.max_level + 1)
        pts += [g, np.array([[0.0, 1.0, 0.0, 1.0], [0.0, 0.0, 1.0, 1.0]])]
        P = np.concatenate(pts, axis=1)
        P = np.stack([x0 + P[0] * tree.side, y0 + P[1] * tree.side])
        out = vp.interp(torch.tensor(F, device="cuda"), torch.tensor(P, device="cuda")).cpu().numpy()
        exact = np.stack([_poly(c1, P[0], P[1]), _poly(c2, P[0], P[1])])
        for k in range(2):
            assert np.abs(out[k] - exact[k]).max() <= 1e-12 * np.abs(exact[k]).max()
    finally:
        vp.close()


def test_interp_outside_root_box_is_nan():
    import torch
    tree = I.uniform_tree(2, side=2.0)
    vp = V.VolumePotential(I.KERNEL_MHELMHOLTZ, 10.0, 4, tree)
    try:
        F = torch.ones(1, vp.N, dtype=torch.float64, device="cuda")
        P = torch.tensor([[0.0, 1.5, -1.0, 0.2], [0.0, 0.0, -1.0000001, 1.0]], dtype=torch.float64, device="cuda")
        out = vp.interp(F, P).cpu().numpy()[0]
        assert out[0] == pytest.approx(1.0, abs=1e-14) and out[3] == pytest.approx(1.0, abs=1e-14)
        assert np.isnan(out[1]) and np.isnan(out[2])
    finally:
        vp.close()


def _lagrange(xi, t):
    return np.array([np.prod([(t - xi[k]) / (xi[i] - xi[k]) for k in range(len(xi)) if k != i])
                     for i in range(len(xi))])


def test_particular_solution_trace_against_the_oracle():
    # grad Psi at boundary nodes: the library's volume potential at the tree nodes carried to the
    # points by vp_tree_interp, against the oracle's values at the nodes of the leaves holding the
    # points, interpolated here on the CPU; then the right-hand side g = u_bc - (dPsi/dy, -dPsi/dx)
    import torch
    from paper_1908_07392_gb300 import warmstart as WS
    wl = I.step_workload(depth=4, p=8, re=100.0, dt=0.1)
    b = V.BIE(wl.alpha, R=1.0, A=0.3, k=5, phase=wl.phi, n_panels=8)
    prob = WS.StepProblem(wl, b)
    try:
        t = 0.37
        f = wl.source(prob.X, prob.Y, t)
        prob.vp(f, prob.u, prob.gradu)
        sel = np.arange(0, b.N, b.N // 6)
        bxy = prob.bxy[:, sel].contiguous()
        d = prob.vp.interp(prob.gradu, bxy).cpu().numpy()
        bx = bxy.cpu().numpy()
        tree, p = wl.tree, wl.p
        x0, y0 = tree.cx - tree.side / 2, tree.cy - tree.side / 2
        xi, _ = I.gl_nodes(p)
        X, Y = I.node_coords(tree, p)
        ref = np.zeros((2, bx.shape[1]))
        for m in range(bx.shape[1]):
            h = tree.side / 2.0 ** tree.level
            inside = np.flatnonzero((bx[0, m] >= x0 + tree.ix * h) & (bx[0, m] <= x0 + (tree.ix + 1) * h) &
                                    (bx[1, m] >= y0 + tree.iy * h) & (bx[1, m] <= y0 + (tree.iy + 1) * h))
            leaf = inside[0]
            idx = leaf * p * p + np.arange(p * p)
            _, ux, uy = O.volume_potential(I.KERNEL_MBIHARMONIC, wl.alpha, p, tree, f.cpu().numpy(), X[idx], Y[idx])
            lx = _lagrange(xi, 2 * ((bx[0, m] - x0) / h[leaf] - tree.ix[leaf]) - 1)
            ly = _lagrange(xi, 2 * ((bx[1, m] - y0) / h[leaf] - tree.iy[leaf]) - 1)
            ref[0, m] = ly @ ux.reshape(p, p) @ lx
            ref[1, m] = ly @ uy.reshape(p, p) @ lx
        for k in range(2):
            assert np.abs(d[k] - ref[k]).max() <= 1e-9 * np.abs(ref[k]).max()
        g, _ = prob.rhs(t)
        src, fs = wl.boundary(t)
        ubc = V.bie_stokeslets(wl.alpha, torch.tensor(src, device="cuda"), torch.tensor(fs, device="cuda"),
                               bxy).cpu().numpy()
        gg = g.reshape(-1, 2)[torch.tensor(sel, device="cuda")].cpu().numpy().T
        scale = max(np.abs(ubc).max(), np.abs(ref).max())
        assert np.abs(gg[0] - (ubc[0] - ref[1])).max() <= 1e-9 * scale
        assert np.abs(gg[1] - (ubc[1] + ref[0])).max() <= 1e-9 * scale
    finally:
        prob.close()
        b.close()
