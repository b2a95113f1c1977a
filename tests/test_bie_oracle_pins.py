"""Pins of the boundary-integral oracles against the equations they come from (CPU only)."""
import mpmath as mp
import numpy as np
import pytest

from oracle import bie_oracle as B
from oracle import ws_oracle as W


@pytest.mark.parametrize("alpha,r", [(10.0, (0.31, -0.17)), (3.0, (-0.8, 0.45)), (50.0, (0.02, 0.013))])
def test_stokeslet_solves_modified_stokes(alpha, r):
    # div S = 0 and alpha^2 S - Lap S + grad phi = 0 away from the source (App. B derivation)
    h = mp.mpf("1e-8")
    x, y = mp.mpf(r[0]), mp.mpf(r[1])
    S = lambda a, b: B.stokeslet(alpha, a, b)
    Sxp, Sxm, Syp, Sym, S0 = S(x + h, y), S(x - h, y), S(x, y + h), S(x, y - h), S(x, y)
    for j in range(2):
        div = (Sxp[0][j] - Sxm[0][j]) / (2 * h) + (Syp[1][j] - Sym[1][j]) / (2 * h)
        assert abs(div) < mp.mpf("1e-12") * (1 + abs(S0[0][j]) / abs(x))
    # pressure of a stokeslet with unit force e_j is phi_j
    php, phm = B.pressure(x + h, y), B.pressure(x - h, y)
    pyp, pym = B.pressure(x, y + h), B.pressure(x, y - h)
    for i in range(2):
        for j in range(2):
            lap = (Sxp[i][j] + Sxm[i][j] + Syp[i][j] + Sym[i][j] - 4 * S0[i][j]) / h ** 2
            # d_i phi_j
            dphi = ((php[j] - phm[j]) / (2 * h)) if i == 0 else ((pyp[j] - pym[j]) / (2 * h))
            res = alpha ** 2 * S0[i][j] - lap + dphi
            assert abs(res) < mp.mpf("1e-6") * (1 + abs(alpha ** 2 * S0[i][j]))


@pytest.mark.parametrize("alpha,r", [(10.0, (0.31, -0.17)), (2.0, (-0.5, 0.9))])
def test_stresslet_matches_its_definition(alpha, r):
    # T_ijk = -d_ik phi_j + d_k S_ij + d_i S_kj (Sec. 2, Eq. stresslet), by 30-digit differences
    h = mp.mpf("1e-10")
    x, y = mp.mpf(r[0]), mp.mpf(r[1])
    T = B.stresslet(alpha, x, y)
    phi = B.pressure(x, y)
    def dS(k):
        if k == 0:
            a, b = B.stokeslet(alpha, x + h, y), B.stokeslet(alpha, x - h, y)
        else:
            a, b = B.stokeslet(alpha, x, y + h), B.stokeslet(alpha, x, y - h)
        return [[(a[i][j] - b[i][j]) / (2 * h) for j in range(2)] for i in range(2)]
    D = [dS(0), dS(1)]
    for i in range(2):
        for j in range(2):
            for k in range(2):
                ref = -(1 if i == k else 0) * phi[j] + D[k][i][j] + D[i][k][j]
                assert abs(T[i][j][k] - ref) < mp.mpf("1e-15") * (1 + abs(ref))


def test_stokeslet_sum_symmetry():
    u = B.stokeslet_sum(5.0, [(2.0, 0.0)], [(1.0, 0.0)], np.array([0.0, 0.0]), np.array([0.3, -0.3]))
    assert abs(u[0, 0] - u[0, 1]) < 1e-15 and abs(u[1, 0] + u[1, 1]) < 1e-15


def test_warm_start_oracle_gradient_by_finite_differences():
    rng = np.random.default_rng(0)
    chans, K, n, Bt = [3, 5, 4, 2], 5, 23, 2
    npar = sum(chans[l + 1] * chans[l] * K + chans[l + 1] for l in range(3))
    p = rng.standard_normal(npar) * 0.3
    x = rng.standard_normal((Bt, 3, n))
    t = rng.standard_normal((Bt, 2, n))
    loss, g = W.loss_and_grad(p, chans, K, x, t)
    eps = 1e-6
    for idx in rng.choice(npar, 25, replace=False):
        pp = p.copy(); pp[idx] += eps
        pm = p.copy(); pm[idx] -= eps
        fd = (W.loss_and_grad(pp, chans, K, x, t)[0] - W.loss_and_grad(pm, chans, K, x, t)[0]) / (2 * eps)
        assert abs(fd - g[idx]) < 1e-7 * (1 + abs(fd))


def test_warm_start_oracle_conv_is_circular():
    # a kernel with a single tap at offset k moves the signal by k - K/2, wrapping around
    x = np.arange(7, dtype=float)[None, None, :]
    Wt = np.zeros((1, 1, 3)); Wt[0, 0, 2] = 1.0
    y = W.conv(x, Wt, np.zeros(1))
    assert np.array_equal(y[0, 0], np.roll(x[0, 0], -1))
