"""Pins of the oracle against facts fixed by the mathematics, not by itself.

Each case is chosen so that a plausible mistake in the oracle fails it:
a wrong kernel sign or normalisation (kernel tables vs scipy, manufactured
solutions), a wrong gradient direction (manufactured, off-centre), a dropped
singular contribution of the self leaf or a near-singular neighbour (constant
source, brute force), a wrong log part of the modified-biharmonic kernel
(radial Gaussian with G2, manufactured G2), a transposed node order (the
off-centre manufactured solution is not symmetric in x and y).
"""
import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp

import oracle as O
from paper_1908_07392_gb300 import inputs as I
from conftest import rel_max_err


def test_gauss_legendre_matches_numpy():
    for n in (1, 2, 5, 8, 16, 20):
        x, w = O.gauss_legendre(n)
        xr, wr = np.polynomial.legendre.leggauss(n)
        assert np.abs(x - xr).max() < 1e-15
        assert np.abs(w - wr).max() < 1e-14


@pytest.mark.parametrize("alpha", [1.0, 10.0, 300.0])
def test_kernels_match_scipy(alpha):
    r = np.geomspace(1e-6, 2.0, 57)
    g1, d1 = O.kernel(0, alpha, r)
    assert rel_max_err(g1, sp.k0(alpha * r) / (2 * np.pi)) < 1e-14
    assert rel_max_err(d1, -alpha * sp.k1(alpha * r) / (2 * np.pi)) < 1e-14
    g2, d2 = O.kernel(1, alpha, r)
    ref2 = (sp.k0(alpha * r) + np.log(r)) / (2 * np.pi * alpha ** 2)
    assert np.abs(g2 - ref2).max() < 1e-14 * np.abs(ref2).max()
    # dG2/dr by 30-digit numerical differentiation of the closed form (sign check of the
    # derivative of Eq. Q0), independent of any Bessel derivative identity
    import mpmath as mp
    mp.mp.dps = 30
    for rv in r[::4]:
        ref = mp.diff(lambda t: (mp.besselk(0, alpha * t) + mp.log(t)) / (2 * mp.pi * alpha ** 2), mp.mpf(rv))
        got = O.kernel(1, alpha, np.array([rv]))[1][0]
        assert abs(got - float(ref)) <= 1e-12 * abs(float(ref)) + 1e-13 / (2 * np.pi * alpha ** 2) / rv


def _targets(tree, p, n, seed):
    X, Y = I.node_coords(tree, p)
    rng = np.random.default_rng(seed)
    idx = rng.choice(X.size, n, replace=False)
    return X[idx], Y[idx]


def test_constant_source_gives_inverse_alpha_squared():
    # f = 1 on the whole box; (alpha^2 - Laplacian) u = 1 has u = 1/alpha^2 away from the
    # box edge; here alpha * dist(edge) > 40, so the truncation is below e^-40.
    alpha, p = 80.0, 6
    tree = I.random_balanced_tree(np.random.default_rng(3), 6, 4, min_depth=2)
    f = np.ones(tree.n_leaves * p * p)
    X, Y = I.node_coords(tree, p)
    sel = np.flatnonzero(np.maximum(np.abs(X), np.abs(Y)) < 0.45)
    sel = sel[:: max(1, sel.size // 24)]
    u, ux, uy = O.volume_potential(0, alpha, p, tree, f, X[sel], Y[sel])
    assert np.abs(u * alpha ** 2 - 1).max() < 1e-12
    assert np.abs(ux).max() * alpha ** 2 < 1e-11 and np.abs(uy).max() * alpha ** 2 < 1e-11


def _radial_exact(kind, alpha, w, r):
    """u(r), du/dr for f = exp(-|x|^2/w^2) by angular averaging of the kernel:
    mean of K0(alpha|x-y|) over |y| = rho is I0(alpha r_<) K0(alpha r_>), mean of
    log|x-y| is log max(r, rho)."""
    f = lambda s: np.exp(-s * s / (w * w))
    top = 12 * w
    out_u, out_d = [], []
    for R in r:
        aR = alpha * R
        # inner: rho < R
        i_in = si.quad(lambda s: s * f(s) * sp.i0e(alpha * s) * np.exp(alpha * (s - R)), 0, R,
                       epsabs=0, epsrel=2e-14, limit=200)[0]
        d_in = si.quad(lambda s: s * f(s) * sp.i0e(alpha * s) * np.exp(alpha * (s - R)), 0, R,
                       epsabs=0, epsrel=2e-14, limit=200)[0]
        i_out = si.quad(lambda s: s * f(s) * sp.k0e(alpha * s) * np.exp(-alpha * (s - R)), R, max(top, R + 1e-3),
                        epsabs=0, epsrel=2e-14, limit=200)[0]
        u1 = i_in * sp.k0e(aR) + i_out * sp.i0e(aR)
        du1 = -alpha * d_in * sp.k1e(aR) + alpha * i_out * sp.i1e(aR)
        if kind == 0:
            out_u.append(u1); out_d.append(du1)
        else:
            m_in = si.quad(lambda s: s * f(s), 0, R, epsabs=0, epsrel=2e-14)[0]
            l_out = si.quad(lambda s: s * f(s) * np.log(s), R, max(top, R + 1e-3), epsabs=0, epsrel=2e-14)[0]
            u2 = (u1 + m_in * np.log(R) + l_out) / alpha ** 2
            du2 = (du1 + m_in / R) / alpha ** 2
            out_u.append(u2); out_d.append(du2)
    return np.array(out_u), np.array(out_d)


@pytest.mark.parametrize("kind,alpha", [(0, 10.0), (1, 10.0), (0, 200.0)])
def test_radial_gaussian_closed_form(kind, alpha):
    w, p = 0.15, 20
    tree = I.uniform_tree(3)
    X, Y = I.node_coords(tree, p)
    f = np.exp(-(X ** 2 + Y ** 2) / w ** 2)
    r = np.hypot(X, Y)
    rng = np.random.default_rng(5)
    near = np.flatnonzero(r < 0.5)
    sel = np.concatenate([np.argsort(r)[:4], rng.choice(near, 8, replace=False)])
    u, ux, uy = O.volume_potential(kind, alpha, p, tree, f, X[sel], Y[sel])
    ue, de = _radial_exact(kind, alpha, w, r[sel])
    assert rel_max_err(u, ue) < 1e-11
    gx, gy = de * X[sel] / r[sel], de * Y[sel] / r[sel]
    assert rel_max_err(ux, gx) < 1e-10
    assert rel_max_err(uy, gy) < 1e-10


def test_manufactured_mhelmholtz():
    # phi = exp(-|x-c|^2/w^2);  (alpha^2 - Laplacian) phi = f  =>  u = phi, grad u = grad phi.
    alpha, w, p = 10.0, 0.17, 14
    c = np.array([0.13, -0.21])
    tree = I.uniform_tree(3)
    X, Y = I.node_coords(tree, p)
    s = (X - c[0]) ** 2 + (Y - c[1]) ** 2
    phi = np.exp(-s / w ** 2)
    f = (alpha ** 2 + 4 / w ** 2 - 4 * s / w ** 4) * phi
    tx, ty = _targets(tree, p, 14, 7)
    u, ux, uy = O.volume_potential(0, alpha, p, tree, f, tx, ty)
    st = (tx - c[0]) ** 2 + (ty - c[1]) ** 2
    pe = np.exp(-st / w ** 2)
    assert rel_max_err(u, pe) < 1e-10 * np.abs(phi).max() / np.abs(pe).max()
    assert np.abs(ux - (-2 * (tx - c[0]) / w ** 2 * pe)).max() < 1e-9
    assert np.abs(uy - (-2 * (ty - c[1]) / w ** 2 * pe)).max() < 1e-9


def test_manufactured_mbiharmonic():
    # Laplacian (alpha^2 - Laplacian) phi = f  =>  G2 * f = phi  (derived with sympy).
    import sympy as S
    x, y = S.symbols("x y", real=True)
    alpha, w, p = 10.0, 0.12, 20  # log tail: the Gaussian must vanish to e^-34 at the box edge
    c = (0.11, 0.19)
    phi = S.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2) / w ** 2)
    lap = lambda e: S.diff(e, x, 2) + S.diff(e, y, 2)
    fexpr = lap(alpha ** 2 * phi - lap(phi))
    fnum = S.lambdify((x, y), fexpr, "numpy")
    gx = S.lambdify((x, y), S.diff(phi, x), "numpy")
    gy = S.lambdify((x, y), S.diff(phi, y), "numpy")
    pn = S.lambdify((x, y), phi, "numpy")
    tree = I.uniform_tree(3)
    X, Y = I.node_coords(tree, p)
    f = fnum(X, Y)
    tx, ty = _targets(tree, p, 14, 8)
    u, ux, uy = O.volume_potential(1, alpha, p, tree, f, tx, ty)
    assert np.abs(u - pn(tx, ty)).max() < 1e-12
    assert np.abs(ux - gx(tx, ty)).max() < 1e-10
    assert np.abs(uy - gy(tx, ty)).max() < 1e-10


@pytest.mark.parametrize("kind", [0, 1])
def test_brute_force_single_leaf(kind):
    # One leaf, p = 4, a random polynomial source; adaptive scipy quadrature split at the
    # target for the singular point; targets inside and just outside the leaf.
    alpha, p = 7.0, 4
    tree = I.Tree(0.0, 0.0, 1.0, np.array([0], np.int32), np.array([0], np.int32), np.array([0], np.int32))
    rng = np.random.default_rng(11)
    f = rng.uniform(-1, 1, p * p)
    xi, _ = np.polynomial.legendre.leggauss(p)
    # monomial coefficients of the tensor interpolant (Vandermonde solve, p = 4)
    V = np.vander(xi, p, increasing=True)
    Cm = np.linalg.solve(V, np.linalg.solve(V, f.reshape(p, p)).T)   # Cm[a, b] for x^a y^b
    def ftilde(yv, xv):
        return float(np.polynomial.polynomial.polyval2d(2 * xv, 2 * yv, Cm))
    def G(r):
        if kind == 0:
            return sp.k0(alpha * r) / (2 * np.pi)
        return (sp.k0(alpha * r) + np.log(r)) / (2 * np.pi * alpha ** 2)
    targets = [(0.1234, -0.2711), (-0.4712, 0.3), (0.5 + 0.013, 0.07)]
    for (x0, y0) in targets:
        u, _, _ = O.volume_potential(kind, alpha, p, tree, f, np.array([x0]), np.array([y0]))
        total = 0.0
        xs = sorted({-0.5, 0.5, min(max(x0, -0.5), 0.5)})
        ys = sorted({-0.5, 0.5, min(max(y0, -0.5), 0.5)})
        for a, b in zip(xs[:-1], xs[1:]):
            for cc, d in zip(ys[:-1], ys[1:]):
                total += si.dblquad(lambda yv, xv: G(np.hypot(x0 - xv, y0 - yv)) * ftilde(yv, xv),
                                    a, b, cc, d, epsabs=1e-14, epsrel=1e-12)[0]
        assert abs(u[0] - total) <= 1e-10 * max(abs(total), 1e-3)


def _diff_matrix(x):
    """First-derivative matrix of the Lagrange interpolant on the nodes x (barycentric form)."""
    n = len(x)
    w = np.array([1.0 / np.prod([x[j] - x[k] for k in range(n) if k != j]) for j in range(n)])
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (w[j] / w[i]) / (x[i] - x[j])
        D[i, i] = -D[i].sum()
    return D


@pytest.mark.parametrize("kind,tol", [(I.KERNEL_MHELMHOLTZ, 5e-7), (I.KERNEL_MBIHARMONIC, 3e-5)])
def test_pde_applied_back_by_spectral_differentiation(kind, tol):
    # On a leaf away from the box edge, the potential solves (alpha^2 - Lap) u = f (G1) or
    # Lap (alpha^2 - Lap) u = f (G2): apply the operator to the oracle's u at the leaf's nodes with
    # the p x p Lagrange differentiation matrices and compare with f (the source there is smooth, so
    # the leaf polynomial of u is accurate to the tolerance)
    p, alpha = 14, 4.0
    tree = I.uniform_tree(2, side=2.0)                 # 16 leaves of side 0.5
    fn = I.gaussian_sum([[0.1, -0.05]], [0.35], [1.0])
    X, Y = I.node_coords(tree, p)
    f = fn(X, Y)
    leaf = 5                                            # interior leaf (level 2, ix = 1, iy = 1)
    assert tree.ix[leaf] == 1 and tree.iy[leaf] == 1
    idx = leaf * p * p + np.arange(p * p)
    u, _, _ = O.volume_potential(kind, alpha, p, tree, f, X[idx], Y[idx])
    xi, _ = I.gl_nodes(p)
    h = tree.side / 2 ** tree.level[leaf]
    D = _diff_matrix(xi) * (2.0 / h)
    U = u.reshape(p, p)                                 # [j (y)][i (x)]

    def lap(V):
        return V @ (D @ D).T + (D @ D) @ V

    op = alpha ** 2 * U - lap(U)
    if kind == I.KERNEL_MBIHARMONIC:
        op = lap(op)
    F = f[idx].reshape(p, p)
    assert np.abs(op - F).max() <= tol * np.abs(F).max()


def test_brute_force_four_leaves():
    # Four leaves (uniform depth 1, side 1), p = 4, a random source per leaf: targets next to the
    # corner the leaves share and inside one leaf, against adaptive scipy quadrature of each leaf's
    # interpolant, split at the target's coordinates
    alpha, p = 5.0, 4
    tree = I.uniform_tree(1, side=1.0)
    rng = np.random.default_rng(21)
    f = rng.uniform(-1, 1, tree.level.size * p * p)
    xi, _ = np.polynomial.legendre.leggauss(p)
    V = np.vander(xi, p, increasing=True)

    def G(r):
        return sp.k0(alpha * r) / (2 * np.pi)

    targets = [(0.011, -0.023), (-0.31, 0.17)]
    for (x0, y0) in targets:
        u, _, _ = O.volume_potential(0, alpha, p, tree, f, np.array([x0]), np.array([y0]))
        total = 0.0
        for leaf in range(tree.level.size):
            h = 0.5
            lx, ly = -0.5 + tree.ix[leaf] * h, -0.5 + tree.iy[leaf] * h
            F = f[leaf * p * p:(leaf + 1) * p * p].reshape(p, p)
            Cm = np.linalg.solve(V, np.linalg.solve(V, F).T)
            cx, cy = lx + h / 2, ly + h / 2

            def integrand(yv, xv, Cm=Cm, cx=cx, cy=cy):
                s = np.polynomial.polynomial.polyval2d(2 * (xv - cx) / h, 2 * (yv - cy) / h, Cm)
                return G(np.hypot(x0 - xv, y0 - yv)) * s

            xs = sorted({lx, lx + h} | ({x0} if lx < x0 < lx + h else set()))
            ys = sorted({ly, ly + h} | ({y0} if ly < y0 < ly + h else set()))
            for a, b in zip(xs[:-1], xs[1:]):
                for c, d in zip(ys[:-1], ys[1:]):
                    total += si.dblquad(integrand, a, b, c, d, epsabs=1e-14, epsrel=1e-12)[0]
        assert abs(u[0] - total) <= 1e-10 * max(abs(total), 1e-3)
