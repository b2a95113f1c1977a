"""Oracle of the layer potential at volume points (test infrastructure only).

u^H = D[mu] (Sec. 2.2, Eqs. uH_dbl, dbl_lyr_pot) discretised by the boundary quadrature of
Sec. 3.2 (Eq. dbl_lyr_quad: panels of equal parameter length, 16-point Gauss-Legendre on each),
summed directly over every boundary node for every target:

    u_a(x) = sum_j D_ab(x - y_j) mu_b(y_j) w_j,   D_ab = -T_bak n_k   (Eq. dbl_lyr_ker),

T the modified Stokes stresslet of App. B (Eq. app_stresslet) with the scalar functions T1, T2, T3
in closed form through K0, K1. In FP64 the closed forms lose digits to cancellation for small
z = alpha r, so pairs with z < 2 are evaluated with the 40-digit mpmath stresslet of bie_oracle;
the rest with scipy's k0, k1. The boundary is the star r(t) = R + A cos(k t + phase) traversed
counter-clockwise, the unit normal pointing into the enclosed domain. Nothing here is shared with
the CUDA path.
"""
from __future__ import annotations

import numpy as np
import scipy.special as sp

from . import bie_oracle as BO

Z_SMALL = 2.0


def star(R, A, k, phase, t):
    """Point, first and second derivative of the star at parameters t (arrays)."""
    r = R + A * np.cos(k * t + phase)
    dr = -A * k * np.sin(k * t + phase)
    c, s = np.cos(t), np.sin(t)
    return (r * c, r * s), (dr * c - r * s, dr * s + r * c)


def star_nodes(R, A, k, phase, n_panels, q=16):
    """Boundary nodes of n_panels equal parameter panels with q-point Gauss-Legendre each:
    x, y, n_x, n_y (unit normal into the domain), w (arc-length weight), t."""
    g, gw = np.polynomial.legendre.leggauss(q)
    h = 2 * np.pi / n_panels
    t = (np.arange(n_panels)[:, None] * h + 0.5 * h * (1.0 + g[None, :])).ravel()
    wt = np.tile(0.5 * h * gw, n_panels)
    (x, y), (dx, dy) = star(R, A, k, phase, t)
    sp_ = np.hypot(dx, dy)
    # counter-clockwise traversal: the interior lies to the left of the tangent
    nx, ny = -dy / sp_, dx / sp_
    return x, y, nx, ny, wt * sp_, t


def _scalars_fp64(z):
    """T1, T2, T3 (App. B) for z >= Z_SMALL, vectorised."""
    K0, K1 = sp.k0(z), sp.k1(z)
    z2 = z * z
    T1 = -(2 * z2 * K0 + (z2 + 4) * z * K1 - 4) / (2 * np.pi * z2 * z2)
    T2 = (4 * z2 * K0 + (z2 + 8) * z * K1 - 8) / (np.pi * z2 ** 3)
    T3 = (z * K1 - 1) / (2 * np.pi * z2)
    return T1, T2, T3


def kernel(alpha, rx, ry, nx, ny):
    """D_ab(r) for arrays of displacements r = x - y and source normals; returns D[2][2][...]."""
    rx, ry, nx, ny = np.broadcast_arrays(np.asarray(rx, float), np.asarray(ry, float),
                                         np.asarray(nx, float), np.asarray(ny, float))
    r = np.hypot(rx, ry)
    z = alpha * r
    T1 = np.empty_like(z); T2 = np.empty_like(z); T3 = np.empty_like(z)
    big = z >= Z_SMALL
    T1[big], T2[big], T3[big] = _scalars_fp64(z[big])
    for idx in zip(*np.nonzero(~big)):
        t1, t2, t3, _, _ = BO.scalars(z[idx])
        T1[idx], T2[idx], T3[idx] = float(t1), float(t2), float(t3)
    a2 = alpha * alpha
    rn = rx * nx + ry * ny
    rr, nn = (rx, ry), (nx, ny)
    D = np.empty((2, 2) + z.shape)
    for a in range(2):
        for b in range(2):
            D[a, b] = (-a2 * T1 * (nn[a] * rr[b] + nn[b] * rr[a] + (rn if a == b else 0.0))
                       - a2 * a2 * T2 * rr[a] * rr[b] * rn - a2 * T3 * rr[a] * nn[b])
    return D


def layer_potential(alpha, src, mu, tx, ty, chunk=2048):
    """u [2][M] at targets (tx, ty) of the double layer with boundary nodes src = (x, y, n_x, n_y, w)
    and density mu [n][2]."""
    x, y, nx, ny, w = (np.asarray(a, float) for a in src)
    mu = np.asarray(mu, float).reshape(-1, 2)
    tx = np.asarray(tx, float); ty = np.asarray(ty, float)
    u = np.zeros((2, tx.size))
    for m0 in range(0, tx.size, chunk):
        sl = slice(m0, m0 + chunk)
        D = kernel(alpha, tx[sl, None] - x[None, :], ty[sl, None] - y[None, :], nx[None, :], ny[None, :])
        for a in range(2):
            u[a, sl] = (D[a, 0] * (mu[:, 0] * w)[None, :] + D[a, 1] * (mu[:, 1] * w)[None, :]).sum(axis=1)
    return u


def lagrange(x_nodes, t):
    """Lagrange basis of the nodes at points t (barycentric form): L[len(t)][len(x_nodes)]."""
    x_nodes = np.asarray(x_nodes, float)
    t = np.atleast_1d(np.asarray(t, float))
    w = np.array([1.0 / np.prod([x_nodes[j] - x_nodes[m] for m in range(x_nodes.size) if m != j])
                  for j in range(x_nodes.size)])
    L = np.empty((t.size, x_nodes.size))
    for i, ti in enumerate(t):
        d = ti - x_nodes
        hit = np.flatnonzero(d == 0.0)
        if hit.size:
            L[i] = 0.0
            L[i, hit[0]] = 1.0
        else:
            v = w / d
            L[i] = v / v.sum()
    return L


def layer_potential_accurate(alpha, geom, n_panels, mu, tx, ty, near=1.2, q=16):
    """u [2][M] at targets of the double layer with the density given at the panel nodes (mu [n][2],
    panel order) and interpolated on each panel by its Lagrange basis in the parameter: panels farther
    than `near` panel lengths from a target by the panel rule, nearer ones by adaptive quadrature
    (scipy quad, split at the closest parameter) of the interpolated density on the exact curve."""
    import scipy.integrate as si
    R, A, k, ph = geom["R"], geom["A"], geom["k"], geom["phase"]
    x, y, nx, ny, w, t = star_nodes(R, A, k, ph, n_panels, q)
    mu = np.asarray(mu, float).reshape(-1, 2)
    g, _ = np.polynomial.legendre.leggauss(q)
    h = 2 * np.pi / n_panels
    plen = w.reshape(n_panels, q).sum(axis=1)
    tx = np.atleast_1d(np.asarray(tx, float)); ty = np.atleast_1d(np.asarray(ty, float))
    u = np.zeros((2, tx.size))
    for m in range(tx.size):
        for pnl in range(n_panels):
            sl = slice(pnl * q, (pnl + 1) * q)
            ta = pnl * h
            ts = np.linspace(ta, ta + h, 129)
            (sx, sy), _ = star(R, A, k, ph, ts)
            dist = np.hypot(sx - tx[m], sy - ty[m])
            if dist.min() >= near * plen[pnl]:
                D = kernel(alpha, tx[m] - x[sl], ty[m] - y[sl], nx[sl], ny[sl])
                for a in range(2):
                    u[a, m] += np.sum((D[a, 0] * mu[sl, 0] + D[a, 1] * mu[sl, 1]) * w[sl])
                continue
            t0 = ts[int(np.argmin(dist))]

            def f(s, a):
                (yx, yy), (dx, dy) = star(R, A, k, ph, np.array([s]))
                sp_ = np.hypot(dx, dy)
                D = kernel(alpha, tx[m] - yx, ty[m] - yy, -dy / sp_, dx / sp_)[:, :, 0]
                L = lagrange(g, 2 * (s - ta) / h - 1)[0]
                return float((D[a, 0] * (L @ mu[sl, 0]) + D[a, 1] * (L @ mu[sl, 1])) * sp_[0])

            pts = [t0] if ta < t0 < ta + h else None
            for a in range(2):
                u[a, m] += si.quad(f, ta, ta + h, args=(a,), points=pts, epsabs=1e-15, epsrel=1e-13, limit=500)[0]
    return u
