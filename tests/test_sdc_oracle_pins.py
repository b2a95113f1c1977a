"""Pins of the SISDC oracle (oracle/sdc_oracle.py) by facts other than itself: the quadrature weights
against closed-form integrals of Lagrange polynomials, the Taylor-Green vortex (an exact solution of
the Navier-Stokes equations, u(t) = u(0) exp(-2 t / Re) on [0, 2 pi)^2) reached with the global
order K of Sec. 3.3, and the order K on a flow whose nonlinear term is not a gradient (against a
much finer run), so that a dropped or mis-signed term of Eq. rhs_correction lowers the order."""
import numpy as np
import pytest

from oracle import sdc_oracle as SO
from paper_1908_07392_gb300 import inputs as I

L = 2 * np.pi


def taylor_green(n):
    return I.taylor_green(n)


def interacting_modes(n):
    return I.interacting_modes(n)


def test_quadrature_weights():
    assert np.allclose(SO.weights(1), [[0.5, 0.5]], atol=1e-15)
    # Simpson-type closed forms for three equispaced nodes
    assert np.allclose(SO.weights(2), [[5 / 12, 8 / 12, -1 / 12], [-1 / 12, 8 / 12, 5 / 12]], atol=1e-15)
    rng = np.random.default_rng(0)
    for p in (1, 2, 3):
        w = SO.weights(p)
        assert np.allclose(w.sum(axis=1), 1.0, atol=1e-14)
        c = rng.standard_normal(p + 1)                 # a polynomial of degree p
        ci = np.polyint(c)
        for m in range(p):
            exact = np.polyval(ci, m + 1.0) - np.polyval(ci, float(m))
            assert abs(w[m] @ np.polyval(c, np.arange(p + 1.0)) - exact) < 1e-13


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_taylor_green_reaches_order(order):
    re, T, n = 1.0, 0.2, 16
    u0, g0, l0 = taylor_green(n)
    exact = u0 * np.exp(-2 * T / re)
    errs = []
    for ns in (4, 8, 16):
        u, _ = SO.run(u0, g0, l0, re, T / ns, ns, order, L)
        errs.append(np.abs(u - exact).max())
    rate = np.log2(errs[1] / errs[2])
    assert rate > order - 0.2, (errs, rate)
    assert errs[2] < [4e-3, 3e-5, 7e-8, 1e-10][order - 1], errs


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_interacting_modes_reach_order(order):
    re, T, n = 10.0, 0.2, 64
    u0, g0, l0 = interacting_modes(n)
    ref, _ = SO.run(u0, g0, l0, re, T / 64, 64, 4, L)
    errs = []
    for ns in (4, 8, 16):
        u, _ = SO.run(u0, g0, l0, re, T / ns, ns, order, L)
        errs.append(np.abs(u - ref).max())
    rate = np.log2(errs[1] / errs[2])
    assert rate > order - 0.3, (errs, rate)


def test_velocity_stays_divergence_free():
    # every substep is a projected solve: the result has no divergence (spectral derivative)
    re, n = 10.0, 64
    u0, g0, l0 = interacting_modes(n)
    u, g = SO.run(u0, g0, l0, re, 0.05, 2, 3, L)
    div = g[0, 0] + g[1, 1]
    assert np.abs(div).max() < 1e-12 * np.abs(g).max()
