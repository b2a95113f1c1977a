"""Pins of the layer-potential oracle (oracle/layer_oracle.py) by facts other than itself:
the FP64 kernel against the 40-digit closed-form stresslet (itself pinned by its definition in
test_bie_oracle_pins), the boundary discretisation against adaptive quadrature of the continuous
boundary integral, and the double-layer velocity against incompressibility (the stresslet's
velocity is divergence free, Sec. 2)."""
import numpy as np
import pytest
import scipy.integrate as si

from oracle import bie_oracle as BO
from oracle import layer_oracle as LO

STAR = dict(R=1.0, A=0.3, k=5, phase=0.4)


def density(t):
    """A smooth density on the boundary parameter (two components)."""
    return np.stack([np.cos(2 * t) + 0.3 * np.sin(t), np.sin(3 * t) - 0.2 + 0.1 * np.cos(t)], axis=-1)


def test_kernel_matches_closed_form_at_40_digits():
    rng = np.random.default_rng(7)
    alpha = 12.0
    for z in np.concatenate([np.geomspace(0.02, 1.9, 6), np.geomspace(2.1, 60.0, 8)]):
        th, phi = rng.uniform(0, 2 * np.pi, 2)
        r = z / alpha
        rx, ry, nx, ny = r * np.cos(th), r * np.sin(th), np.cos(phi), np.sin(phi)
        D = LO.kernel(alpha, np.array([rx]), np.array([ry]), np.array([nx]), np.array([ny]))[:, :, 0]
        Dm = BO.double_layer_kernel(alpha, rx, ry, nx, ny)
        for a in range(2):
            for b in range(2):
                ref = float(Dm[a][b])
                scale = max(abs(float(Dm[0][0])), abs(float(Dm[0][1])), abs(float(Dm[1][0])), abs(float(Dm[1][1])))
                assert abs(D[a, b] - ref) <= 2e-13 * scale, (z, a, b, D[a, b], ref)


@pytest.mark.parametrize("target", [(0.1, 0.05), (-0.4, 0.3)])
def test_boundary_quadrature_against_adaptive_integration(target):
    # the continuous integral int D(x - y(t)) mu(t) |y'(t)| dt by adaptive quadrature on the
    # parametrisation, against the panel rule of the oracle (spectrally accurate for a target
    # well inside the curve)
    alpha = 10.0
    x0, y0 = target

    def integrand(t, a):
        (yx, yy), (dx, dy) = LO.star(STAR["R"], STAR["A"], STAR["k"], STAR["phase"], np.array([t]))
        sp_ = np.hypot(dx, dy)
        nx, ny = -dy / sp_, dx / sp_
        D = LO.kernel(alpha, x0 - yx, y0 - yy, nx, ny)[:, :, 0]
        mu = density(np.array([t]))[0]
        return float((D[a, 0] * mu[0] + D[a, 1] * mu[1]) * sp_[0])

    ref = [si.quad(integrand, 0.0, 2 * np.pi, args=(a,), epsabs=1e-14, epsrel=1e-13, limit=400)[0] for a in range(2)]
    x, y, nx, ny, w, t = LO.star_nodes(n_panels=32, **STAR)
    u = LO.layer_potential(alpha, (x, y, nx, ny, w), density(t), np.array([x0]), np.array([y0]))
    scale = max(abs(ref[0]), abs(ref[1]))
    for a in range(2):
        assert abs(u[a, 0] - ref[a]) <= 1e-12 * scale, (a, u[a, 0], ref[a])


def test_nodes_describe_the_star():
    x, y, nx, ny, w, t = LO.star_nodes(n_panels=40, **STAR)
    # the weights integrate arc length; the normals are unit and point inward (toward the origin for
    # this star); the enclosed area by the divergence theorem matches the polar formula
    L = w.sum()
    Lref = si.quad(lambda s: np.hypot(*LO.star(STAR["R"], STAR["A"], STAR["k"], STAR["phase"], np.array([s]))[1])[0],
                   0, 2 * np.pi, epsabs=1e-14, limit=200)[0]
    assert abs(L - Lref) < 1e-12 * Lref
    assert np.allclose(np.hypot(nx, ny), 1.0)
    assert np.all(x * nx + y * ny < 0)
    area = -0.5 * np.sum((x * nx + y * ny) * w)  # inward normal: area = -1/2 int x.n ds
    area_ref = 0.5 * si.quad(lambda s: (STAR["R"] + STAR["A"] * np.cos(STAR["k"] * s + STAR["phase"])) ** 2, 0,
                             2 * np.pi)[0]
    assert abs(area - area_ref) < 1e-12 * area_ref


def test_velocity_is_divergence_free():
    # the double-layer velocity solves the modified Stokes equations inside: div u = 0, checked by
    # fourth-order central differences relative to |grad u|
    alpha, h = 8.0, 1e-3
    x, y, nx, ny, w, t = LO.star_nodes(n_panels=32, **STAR)
    src, mu = (x, y, nx, ny, w), density(t)
    x0, y0 = 0.15, -0.2
    off = np.array([-2, -1, 1, 2]) * h
    cw = np.array([1, -8, 8, -1]) / (12 * h)
    ux = LO.layer_potential(alpha, src, mu, x0 + off, np.full(4, y0))
    uy = LO.layer_potential(alpha, src, mu, np.full(4, x0), y0 + off)
    dudx = ux[0] @ cw
    dvdy = uy[1] @ cw
    grad = max(abs(dudx), abs(dvdy), abs(ux[1] @ cw), abs(uy[0] @ cw))
    assert abs(dudx + dvdy) < 1e-9 * grad, (dudx, dvdy)


def test_lagrange_reproduces_polynomials():
    g, _ = np.polynomial.legendre.leggauss(16)
    t = np.concatenate([np.linspace(-1.0, 1.0, 41), g[:3]])  # also exactly at nodes
    L = LO.lagrange(g, t)
    for deg in (0, 5, 15):
        c = np.random.default_rng(deg).standard_normal(deg + 1)
        assert np.abs(L @ np.polynomial.polynomial.polyval(g, c) - np.polynomial.polynomial.polyval(t, c)).max() < 1e-12 * max(1.0, np.abs(c).sum())


def test_accurate_sum_matches_panel_rule_away_from_the_boundary():
    # at targets far from every panel both the accurate and the plain sums are the panel rule
    alpha = 10.0
    x, y, nx, ny, w, t = LO.star_nodes(n_panels=24, **STAR)
    mu = density(t)
    tx, ty = np.array([0.1, -0.3]), np.array([0.05, 0.2])
    ua = LO.layer_potential_accurate(alpha, STAR, 24, mu, tx, ty, near=1.2)
    up = LO.layer_potential(alpha, (x, y, nx, ny, w), mu, tx, ty)
    assert np.abs(ua - up).max() < 1e-14 * np.abs(up).max()


def test_accurate_sum_near_the_boundary_converges_with_panels():
    # close to the boundary the plain rule fails; the accurate sum with the density given by a smooth
    # function of t converges to the continuous integral as the panels are refined (spectrally)
    alpha = 10.0
    (bx, by), (dx, dy) = LO.star(STAR["R"], STAR["A"], STAR["k"], STAR["phase"], np.array([1.1]))
    sp_ = np.hypot(dx, dy)
    tx, ty = bx - 0.004 * (dy / sp_), by + 0.004 * (dx / sp_)  # inward normal step of 0.004
    vals = []
    for npnl in (20, 40):
        x, y, nx, ny, w, t = LO.star_nodes(n_panels=npnl, **STAR)
        vals.append(LO.layer_potential_accurate(alpha, STAR, npnl, density(t), tx, ty, near=1.2)[:, 0])
        plain = LO.layer_potential(alpha, (x, y, nx, ny, w), density(t), tx, ty)[:, 0]
    assert np.abs(vals[1] - vals[0]).max() < 1e-9 * np.abs(vals[1]).max()
    assert np.abs(plain - vals[1]).max() > 1e-6 * np.abs(vals[1]).max()  # the plain rule is far off there
