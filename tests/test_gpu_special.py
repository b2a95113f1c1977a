"""The device special functions (vp_special) against 40-digit mpmath values."""
import numpy as np
import pytest

import paper_1908_07392_gb300 as V

pytestmark = pytest.mark.gpu

mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 40


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    V.load_library()


def _args(lo, hi, n, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([np.geomspace(lo, hi, n), np.exp(rng.uniform(np.log(lo), np.log(hi), n // 2)),
                                     [2.0, 2.0000001, 25.0, 25.0000001]]))


def _rel(a, b):
    return abs(a - b) / abs(b)


def test_k0_k1_scaled():
    # the three regimes (series z <= 2, trapezoid 2 < z <= 25, Hankel beyond) over [1e-8, 800]
    import torch
    z = _args(1e-8, 800.0, 80, 1)
    z = z[z <= 800.0]
    out = V.vp_special(0, torch.tensor(z, device="cuda")).cpu().numpy()
    worst = [0.0, 0.0]
    for m, x in enumerate(z):
        for k in range(2):
            ref = float(mpmath.besselk(k, x) * mpmath.exp(x))
            worst[k] = max(worst[k], _rel(out[k, m], ref))
    print("K0, K1 scaled: worst relative error", worst)
    assert worst[0] < 2e-15 and worst[1] < 2e-15, worst


def test_normalised_multipole_basis():
    # e^z Khat_n(z), Khat_n = K_n (z/2)^n 2/(n-1)!, n <= 60, at the arguments the expansions use
    import torch
    nmax = 60
    z = _args(1e-3, 200.0, 24, 2)
    out = V.vp_special(1, torch.tensor(z, device="cuda"), nmax).cpu().numpy()
    worst = 0.0
    for m, x in enumerate(z):
        xm = mpmath.mpf(x)
        for n in range(nmax + 1):
            k = mpmath.besselk(n, xm) * mpmath.exp(xm)
            ref = k if n == 0 else k * (xm / 2) ** n * 2 / mpmath.factorial(n - 1)
            worst = max(worst, _rel(out[n, m], float(ref)))
    print("Khat scaled: worst relative error", worst)
    assert worst < 1e-14, worst


def test_normalised_local_basis():
    # Ihat_n(z) = I_n(z) n!/(z/2)^n, n <= 60, z up to 45
    import torch
    nmax = 60
    z = _args(1e-6, 45.0, 24, 3)
    out = V.vp_special(2, torch.tensor(z, device="cuda"), nmax).cpu().numpy()
    worst = 0.0
    for m, x in enumerate(z):
        xm = mpmath.mpf(x)
        for n in range(nmax + 1):
            ref = mpmath.besseli(n, xm) * mpmath.factorial(n) / (xm / 2) ** n
            worst = max(worst, _rel(out[n, m], float(ref)))
    print("Ihat: worst relative error", worst)
    assert worst < 1e-14, worst


def test_argument_checks():
    import torch
    z = torch.ones(3, dtype=torch.float64, device="cuda")
    with pytest.raises(V.VPError):
        V.vp_special(3, z)
    with pytest.raises(V.VPError):
        V.vp_special(1, z, 65)
