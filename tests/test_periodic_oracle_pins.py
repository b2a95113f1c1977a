"""Pins of the periodic-solution oracle (oracle/periodic_oracle.py) by exact solutions of the
periodic modified Stokes equations (Sec. 2.1): a manufactured divergence-free velocity with an
added pressure gradient, a constant force, and a pure gradient force (taken up by the pressure)."""
import numpy as np

from oracle import periodic_oracle as PO


def grid(n, L):
    x = np.arange(n) * L / n
    Y, X = np.meshgrid(x, x, indexing="ij")
    return X, Y


def test_manufactured_divergence_free_velocity():
    # psi = sin(a x + p1) cos(b y + p2): u = (dpsi/dy, -dpsi/dx) is divergence free;
    # F = (alpha^2 - Lap) u + grad p with p = cos(c x) sin(d y) must give u back exactly
    n, L, alpha = 64, 3.0, 7.0
    X, Y = grid(n, L)
    w = 2 * np.pi / L
    a, b, c, d, p1, p2 = 3 * w, 2 * w, 1 * w, 4 * w, 0.3, -0.7
    s1, c1 = np.sin(a * X + p1), np.cos(a * X + p1)
    s2, c2 = np.sin(b * Y + p2), np.cos(b * Y + p2)
    u = np.stack([-b * s1 * s2, -a * c1 * c2])
    lap = -(a * a + b * b)
    px = -c * np.sin(c * X) * np.sin(d * Y)
    py = d * np.cos(c * X) * np.cos(d * Y)
    F = (alpha ** 2 - lap) * u + np.stack([px, py])
    uo, go = PO.periodic_stokes(alpha, L, F)
    assert np.abs(uo - u).max() < 1e-13 * np.abs(u).max()
    gx = np.stack([[-a * b * c1 * s2, -b * b * s1 * c2], [a * a * s1 * c2, a * b * c1 * s2]])
    assert np.abs(go - gx).max() < 1e-12 * np.abs(gx).max()


def test_constant_force():
    n, L, alpha = 32, 2.0, 3.0
    F = np.stack([np.full((n, n), 1.5), np.full((n, n), -0.25)])
    u, g = PO.periodic_stokes(alpha, L, F)
    assert np.allclose(u[0], 1.5 / alpha ** 2, rtol=1e-14) and np.allclose(u[1], -0.25 / alpha ** 2, rtol=1e-14)
    assert np.abs(g).max() < 1e-15


def test_gradient_force_is_absorbed_by_the_pressure():
    n, L, alpha = 64, 3.0, 5.0
    X, Y = grid(n, L)
    w = 2 * np.pi / L
    phi_x = 2 * w * np.cos(2 * w * X) * np.sin(3 * w * Y)
    phi_y = 3 * w * np.sin(2 * w * X) * np.cos(3 * w * Y)
    u, g = PO.periodic_stokes(alpha, L, np.stack([phi_x, phi_y]))
    assert np.abs(u).max() < 1e-14 * np.abs(phi_x).max()
