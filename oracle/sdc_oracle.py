"""Oracle of semi-implicit spectral deferred correction time stepping (test infrastructure only).

Sec. 3.3 (Eqs. sisdc_initial, sisdc_formula, rhs_initial, rhs_correction,
rhs_correction_integral) for the Navier-Stokes equations u_t + (u . grad) u = Delta u / Re - grad p,
div u = 0, on a periodic box, each implicit substep solved by the periodic modified Stokes solution
of periodic_oracle (Sec. 2.1, Eq. uhat): (alpha^2 - Delta) u + Re grad p = F, alpha^2 = Re / dt.

Order K >= 2: p = K - 1 equal substeps dt = Delta t / p on [t_a, t_b], a first pass of IMEX Euler
substeps (Eq. rhs_initial) and K - 1 correction passes (Eq. rhs_correction), final value u^{K-1}_p.
Order 1: one IMEX Euler step of length Delta t. Per node j of a pass the method keeps u_j, the
nonlinear term N_j = (u_j . grad) u_j formed pointwise from u and its gradient, and the implicit term
L_j = Delta u_j - Re grad p_j, recovered from the substep's own equation as alpha^2 u_j - F_j (at the
first time the caller supplies Delta u; a gradient added to F does not change u). The quadrature
I_m^{m+1} integrates the polynomial through the p + 1 nodes: weights q_j^m / dt = the integral over
[m, m + 1] of the j-th Lagrange polynomial on the integer nodes 0..p. Arrays are [component][row j
(y)][column i (x)], gradients [component a][direction m] = d u_a / d x_m. Nothing here is shared with
the CUDA path.
"""
from __future__ import annotations

import numpy as np

from .periodic_oracle import periodic_stokes


def weights(p):
    """w[m][j] = (1 / dt) q_j^m for equispaced nodes 0..p: the integral over [m, m + 1] of the
    Lagrange polynomial of node j."""
    nodes = np.arange(p + 1, dtype=float)
    w = np.zeros((p, p + 1))
    for j in range(p + 1):
        others = np.delete(nodes, j)
        c = np.poly(others) / np.prod(nodes[j] - others)   # coefficients, highest power first
        ci = np.polyint(c)
        for m in range(p):
            w[m, j] = np.polyval(ci, m + 1.0) - np.polyval(ci, float(m))
    return w


def nonlinear(u, g):
    """(u . grad) u: component a is u_x du_a/dx + u_y du_a/dy."""
    return np.stack([u[0] * g[a, 0] + u[1] * g[a, 1] for a in range(2)])


def step(u, g, L, re, dt_step, order, side):
    """One step of length dt_step from (u, grad u, L) at t_a; returns (u, grad u, L) at t_b."""
    if order == 1:
        alpha = np.sqrt(re / dt_step)
        F = alpha ** 2 * u - re * nonlinear(u, g)
        un, gn = periodic_stokes(alpha, side, F)
        return un, gn, alpha ** 2 * un - F
    p = order - 1
    dt = dt_step / p
    alpha = np.sqrt(re / dt)
    w = weights(p)
    # first pass (Eq. rhs_initial)
    U, G, Ls = [u], [g], [L]
    for m in range(p):
        F = alpha ** 2 * U[m] - re * nonlinear(U[m], G[m])
        un, gn = periodic_stokes(alpha, side, F)
        U.append(un); G.append(gn); Ls.append(alpha ** 2 * un - F)
    # correction passes (Eqs. rhs_correction, rhs_correction_integral)
    for _ in range(order - 1):
        Nold = [nonlinear(U[j], G[j]) for j in range(p + 1)]
        V, H, Lv = [u], [g], [L]
        for m in range(p):
            quad = sum(w[m, j] * (Ls[j] - re * Nold[j]) for j in range(p + 1))
            F = (alpha ** 2 * V[m] - re * (nonlinear(V[m], H[m]) - Nold[m]) - Ls[m + 1] + quad)
            un, gn = periodic_stokes(alpha, side, F)
            V.append(un); H.append(gn); Lv.append(alpha ** 2 * un - F)
        U, G, Ls = V, H, Lv
    return U[p], G[p], Ls[p]


def run(u0, g0, lap0, re, dt_step, n_steps, order, side):
    """n_steps steps from u0 (with its gradient g0 and Laplacian lap0); returns (u, grad u)."""
    u, g, L = (np.asarray(a, float) for a in (u0, g0, lap0))
    for _ in range(n_steps):
        u, g, L = step(u, g, L, re, dt_step, order, side)
    return u, g
