"""SISDC time stepping on the periodic box (vp_sdc_*) against the numpy oracle element by element, and
its properties at full size: the Taylor-Green exact solution, the order K, a divergence-free result."""
import numpy as np
import pytest

import paper_1908_07392_gb300 as V
from paper_1908_07392_gb300 import inputs as I
from oracle import sdc_oracle as SO

pytestmark = pytest.mark.gpu

L = 2 * np.pi


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    V.load_library()


def _run_gpu(fields, re, dt, n_steps, order, n):
    import torch
    u0, g0, l0 = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in fields)
    s = V.SISDC(re, dt, order, n, L)
    try:
        s.set(u0, g0, l0)
        s.step(n_steps)
        u, g = s.get()
        torch.cuda.synchronize()
        return u.cpu().numpy(), g.cpu().numpy()
    finally:
        s.close()


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("order", [1, 2, 3, 4])
@pytest.mark.parametrize("n", [32, 128])
def test_against_oracle(order, n):
    fields = I.interacting_modes(n)
    re, dt, steps = 10.0, 0.02, 3
    u, g = _run_gpu(fields, re, dt, steps, order, n)
    uo, go = SO.run(*fields, re, dt, steps, order, L)
    assert _rel(u, uo) < 1e-12 and _rel(g, go) < 1e-12, (_rel(u, uo), _rel(g, go))


@pytest.mark.parametrize("order", [2, 4])
def test_taylor_green_full_size(order):
    # 2048^2 grid, the exact decay reached at the scheme's accuracy, and order K against the exact
    # solution
    n, re, T = 2048, 1.0, 0.2
    fields = I.taylor_green(n)
    exact = fields[0] * np.exp(-2 * T / re)
    errs = []
    for ns in (4, 8):
        u, g = _run_gpu(fields, re, T / ns, ns, order, n)
        errs.append(np.abs(u - exact).max())
        div = g[0, 0] + g[1, 1]
        assert np.abs(div).max() < 1e-12 * np.abs(g).max()
    rate = np.log2(errs[0] / errs[1])
    assert rate > order - 0.4, (errs, rate)


def test_order_on_interacting_modes():
    # order 3 on a flow whose nonlinear term matters, against a finer order-4 run on the GPU itself
    n, re, T = 64, 10.0, 0.2
    fields = I.interacting_modes(n)
    ref, _ = _run_gpu(fields, re, T / 64, 64, 4, n)
    errs = [np.abs(_run_gpu(fields, re, T / ns, ns, 3, n)[0] - ref).max() for ns in (8, 16)]
    assert np.log2(errs[0] / errs[1]) > 2.7, errs


def test_bad_arguments():
    s = V.SISDC(10.0, 0.01, 2, 64, L)
    try:
        with pytest.raises(V.VPError):      # no state set yet
            s.step(1)
        with pytest.raises(V.VPError):
            s.get()
    finally:
        s.close()
    with pytest.raises(V.VPError):
        V.SISDC(10.0, 0.01, 5, 64, L)
    with pytest.raises(V.VPError):
        V.SISDC(10.0, -0.01, 2, 64, L)
    with pytest.raises(V.VPError):
        V.SISDC(10.0, 0.01, 2, 48, L)
