"""The periodic particular solution by FFT (vp_periodic_*) through the C ABI: against the numpy
oracle at every grid point for several sizes, and against the tree's free-space volume potential
for a compact divergence-free force (then u = G1 * F componentwise and the periodic images decay
like exp(-alpha d))."""
import numpy as np
import pytest

import paper_1908_07392_gb300 as V
from paper_1908_07392_gb300 import inputs as I
from oracle import periodic_oracle as PO

pytestmark = pytest.mark.gpu

TOL = 1e-12  # relative max-norm, FP64 transforms (rounding grows like log n)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    V.load_library()


def random_force(n, L, seed):
    """A smooth periodic force: random Fourier modes with decaying amplitudes (seeded)."""
    rng = np.random.default_rng(seed)
    x = np.arange(n) * L / n
    Y, X = np.meshgrid(x, x, indexing="ij")
    F = np.zeros((2, n, n))
    w = 2 * np.pi / L
    for _ in range(24):
        kx, ky = rng.integers(-min(12, n // 4), min(12, n // 4) + 1, 2)
        amp = rng.standard_normal(2) / (1.0 + kx * kx + ky * ky)
        ph = rng.uniform(0, 2 * np.pi, 2)
        F[0] += amp[0] * np.cos(w * (kx * X + ky * Y) + ph[0])
        F[1] += amp[1] * np.cos(w * (kx * X + ky * Y) + ph[1])
    return F


@pytest.mark.parametrize("n,alpha", [(32, 3.0), (256, 40.0), (1024, 316.0)])
def test_against_oracle_every_point(n, alpha):
    import torch
    L = 3.0
    F = random_force(n, L, n)
    P = V.PeriodicStokes(alpha, n, L)
    try:
        u, g = P(torch.from_numpy(F).cuda())
        u2, g2 = P(torch.from_numpy(F).cuda())  # the work arrays are reused
        torch.cuda.synchronize()
        assert torch.equal(u, u2) and torch.equal(g, g2)
        u, g = u.cpu().numpy(), g.cpu().numpy()
    finally:
        P.close()
    uo, go = PO.periodic_stokes(alpha, L, F)
    for a in range(2):
        assert np.abs(u[a] - uo[a]).max() <= TOL * np.abs(uo[a]).max()
        for m in range(2):
            assert np.abs(g[a, m] - go[a, m]).max() <= TOL * np.abs(go[a, m]).max()


@pytest.mark.parametrize("n", [32, 64])
def test_white_noise_with_nyquist_content(n):
    # every mode present, the Nyquist row, column and corner included: the multiplier of a real field
    # must stay even there (the oracle transforms each component separately and keeps the real part)
    import torch
    L, alpha = 2 * np.pi, 5.0
    F = np.random.default_rng(n + 7).standard_normal((2, n, n))
    P = V.PeriodicStokes(alpha, n, L)
    try:
        u, g = P(torch.from_numpy(F).cuda())
        torch.cuda.synchronize()
        u, g = u.cpu().numpy(), g.cpu().numpy()
    finally:
        P.close()
    uo, go = PO.periodic_stokes(alpha, L, F)
    assert np.abs(u - uo).max() <= TOL * np.abs(uo).max()
    assert np.abs(g - go).max() <= TOL * np.abs(go).max()


def test_against_the_tree_for_a_compact_divergence_free_force():
    # F = perp grad phi, phi a Gaussian well inside the box: u = (alpha^2 - Lap)^-1 F = G1 * F
    import torch
    L, n, alpha = 3.0, 512, 60.0
    c, wdt = np.array([0.2, -0.1]), 0.15
    def force(X, Y):
        e = np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2) / wdt ** 2)
        return np.stack([-2 * (Y - c[1]) / wdt ** 2 * e, 2 * (X - c[0]) / wdt ** 2 * e])
    x = -1.5 + np.arange(n) * L / n
    Yg, Xg = np.meshgrid(x, x, indexing="ij")
    P = V.PeriodicStokes(alpha, n, L)
    try:
        u_fft, _ = P(torch.from_numpy(np.ascontiguousarray(force(Xg, Yg))).cuda())
        u_fft = u_fft.cpu().numpy()
    finally:
        P.close()
    tree = I.uniform_tree(5, side=3.0)
    vp = V.VolumePotential(V.VP_KERNEL_MHELMHOLTZ, alpha, 16, tree)
    try:
        xy = vp.nodes().cpu().numpy()
        Fn = force(xy[0], xy[1])
        u_tree = []
        for a in range(2):
            ua, _ = vp(torch.from_numpy(np.ascontiguousarray(Fn[a])).cuda())
            u_tree.append(ua.clone())
        pts = torch.from_numpy(np.ascontiguousarray(np.stack([Xg.ravel(), Yg.ravel()]))).cuda()
        ut = vp.interp(torch.stack(u_tree), pts).cpu().numpy().reshape(2, n, n)
    finally:
        vp.close()
    err = np.abs(ut - u_fft).max() / np.abs(u_fft).max()
    assert err < 1e-10, err
