"""Oracle of the boundary-integral pieces (test infrastructure only).

* The scalar functions of the modified Stokes stokeslet and stresslet (App. B, Eqs.
  app_stokeslet_S1/S2, app_stresslet_T1/T2/T3) from their closed forms in K0, K1, evaluated with
  mpmath at 40 digits, which removes the cancellation the closed forms suffer for small arguments.
* The stokeslet tensor S_ij(r) = S1 d_ij + a^2 S2 r_i r_j and the pressure vector phi_i = r_i/(2 pi r^2)
  (App. B), the stresslet T_ijk = a^2 T1 (d_jk r_i + d_ik r_j + d_ij r_k) + a^4 T2 r_i r_j r_k
  + a^2 T3 d_ik r_j (Eq. app_stresslet), and sums of stokeslets (exact solutions of the homogeneous
  modified Stokes equation inside any domain that excludes the sources).
These are pinned in the tests by the equations the paper derives them from (divergence free,
a^2 u - Lap u + grad p = 0 away from the source, T from its definition through S and phi).
"""
from __future__ import annotations

import mpmath as mp
import numpy as np

mp.mp.dps = 40


def scalars(z):
    """(T1, T2, T3, S1, S2) at z > 0 as mpmath numbers."""
    z = mp.mpf(z)
    K0, K1 = mp.besselk(0, z), mp.besselk(1, z)
    z2 = z * z
    T1 = -(2 * z2 * K0 + (z2 + 4) * z * K1 - 4) / (2 * mp.pi * z2 * z2)
    T2 = (4 * z2 * K0 + (z2 + 8) * z * K1 - 8) / (mp.pi * z2 ** 3)
    T3 = (z * K1 - 1) / (2 * mp.pi * z2)
    S1 = (z2 * K0 + z * K1 - 1) / (2 * mp.pi * z2)
    S2 = -(z2 * K0 + 2 * z * K1 - 2) / (2 * mp.pi * z2 * z2)
    return T1, T2, T3, S1, S2


def stokeslet(alpha, rx, ry):
    """S_ij at r = (rx, ry) (mpmath 2x2)."""
    a = mp.mpf(alpha)
    r = mp.sqrt(mp.mpf(rx) ** 2 + mp.mpf(ry) ** 2)
    _, _, _, S1, S2 = scalars(a * r)
    rr = [mp.mpf(rx), mp.mpf(ry)]
    return [[S1 * (1 if i == j else 0) + a * a * S2 * rr[i] * rr[j] for j in range(2)] for i in range(2)]


def pressure(rx, ry):
    r2 = mp.mpf(rx) ** 2 + mp.mpf(ry) ** 2
    return [mp.mpf(rx) / (2 * mp.pi * r2), mp.mpf(ry) / (2 * mp.pi * r2)]


def stresslet(alpha, rx, ry):
    """T_ijk at r (mpmath 2x2x2) from the closed form."""
    a = mp.mpf(alpha)
    r = mp.sqrt(mp.mpf(rx) ** 2 + mp.mpf(ry) ** 2)
    T1, T2, T3, _, _ = scalars(a * r)
    rr = [mp.mpf(rx), mp.mpf(ry)]
    d = lambda i, j: 1 if i == j else 0
    return [[[a * a * T1 * (d(j, k) * rr[i] + d(i, k) * rr[j] + d(i, j) * rr[k]) + a ** 4 * T2 * rr[i] * rr[j] * rr[k]
              + a * a * T3 * d(i, k) * rr[j] for k in range(2)] for j in range(2)] for i in range(2)]


def double_layer_kernel(alpha, rx, ry, nx, ny):
    """D_ij = -T_jik n_k (Eq. dbl_lyr_ker), r = x - y, n = n(y)."""
    T = stresslet(alpha, rx, ry)
    n = [mp.mpf(nx), mp.mpf(ny)]
    return [[-sum(T[j][i][k] * n[k] for k in range(2)) for j in range(2)] for i in range(2)]


def stokeslet_sum(alpha, src, f, x, y):
    """u (2 x M, float64) at points (x, y) of stokeslets at src [K][2] with strengths f [K][2]."""
    u = np.zeros((2, len(x)))
    for m in range(len(x)):
        for (sx, sy), (fx, fy) in zip(src, f):
            S = stokeslet(alpha, x[m] - sx, y[m] - sy)
            u[0, m] += float(S[0][0] * fx + S[0][1] * fy)
            u[1, m] += float(S[1][0] * fx + S[1][1] * fy)
    return u
