"""Boundary integral equation, GMRES and the learned warm start on the GPU, against the oracles."""
import numpy as np
import pytest

import paper_1908_07392_gb300 as V
from oracle import bie_oracle as BO
from oracle import ws_oracle as WO

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    V.load_library()


def test_kernel_scalars_against_mpmath():
    import torch
    z = np.concatenate([np.geomspace(1e-3, 1.49, 25), [1.5, 1.51], np.geomspace(1.6, 40.0, 15)])
    got = V.bie_kernel_scalars(torch.tensor(z, device="cuda")).cpu().numpy()
    for m, zz in enumerate(z):
        ref = [float(v) for v in BO.scalars(zz)]
        for k in range(5):
            assert abs(got[k, m] - ref[k]) <= 1e-12 * abs(ref[k]) + 1e-300, (k, zz, got[k, m], ref[k])


def test_nullspace_of_half_plus_double_layer():
    # Nullspace lemma (Sec. 2.2 / App. A): 1/2 + D has a one-dimensional nullspace whose element xi has
    # int xi.n != 0, and adding W makes the system invertible.
    import torch
    b = V.BIE(10.0, n_panels=32)
    try:
        n2 = 2 * b.N
        A = torch.stack([b.apply(torch.eye(n2, dtype=torch.float64, device="cuda")[k]) for k in range(n2)], 1)
        nx, ny, w = b.nodes[2], b.nodes[3], b.nodes[4]
        nvec = torch.stack([nx, ny], 1).reshape(-1)                 # n at the nodes, interleaved
        wn = (torch.stack([nx, ny], 1) * w[:, None]).reshape(-1)    # n w
        Wm = torch.outer(nvec, wn) / b.length
        s_full = torch.linalg.svdvals(A)
        U, s, Vh = torch.linalg.svd(A - Wm)
        assert float(s[-1]) < 1e-9 * float(s[0])          # one (numerically) zero singular value
        assert float(s[-2]) > 1e-3 * float(s[0])          # only one
        xi = Vh[-1]
        assert abs(float(xi @ wn)) > 1e-3                   # int xi.n != 0
        assert float(s_full[-1]) > 1e-3 * float(s_full[0])  # with W the system is invertible
    finally:
        b.close()


@pytest.mark.parametrize("alpha,n_panels", [(10.0, 96), (40.0, 128)])
def test_exact_solution_from_exterior_stokeslets(alpha, n_panels):
    # homogeneous problem with the trace of exterior stokeslets as data: D[mu] reproduces them inside
    import torch
    b = V.BIE(alpha, R=1.0, A=0.3, k=5, phase=0.4, n_panels=n_panels)
    try:
        rng = np.random.default_rng(1)
        ang = rng.uniform(0, 2 * np.pi, 5)
        src = np.stack([1.7 * np.cos(ang), 1.7 * np.sin(ang)], 1)
        f = rng.uniform(-1, 1, (5, 2))
        S = torch.tensor(src, device="cuda"); F = torch.tensor(f, device="cuda")
        xy = b.nodes[0:2].contiguous()
        g = V.bie_stokeslets(alpha, S, F, xy).t().contiguous().reshape(-1)
        mu, it, rr = b.solve(g, None, 1e-13)
        assert rr < 1e-12 and it < 150
        r = rng.uniform(0, 0.45, 12); th = rng.uniform(0, 2 * np.pi, 12)
        tx = np.stack([r * np.cos(th), r * np.sin(th)])
        u = b.eval(mu, torch.tensor(tx, device="cuda")).cpu().numpy()
        ue = BO.stokeslet_sum(alpha, src, f, tx[0], tx[1])
        assert np.abs(u - ue).max() < 1e-9 * np.abs(ue).max()
        # the library's stokeslet sum agrees with the oracle's
        ul = V.bie_stokeslets(alpha, S, F, torch.tensor(tx, device="cuda")).cpu().numpy()
        assert np.abs(ul - ue).max() < 1e-13 * np.abs(ue).max()
    finally:
        b.close()


def test_network_forward_and_gradient_against_the_oracle():
    import torch
    chans, K, n, B = [8, 16, 16, 2], 5, 64, 3
    net = V.WarmStartNet(in_ch=8, width=16, out_ch=2, n_layers=3, ksize=K, n=n, max_batch=4, seed=3)
    try:
        rng = np.random.default_rng(2)
        x = rng.standard_normal((B, 8, n)).astype(np.float32)
        t = rng.standard_normal((B, 2, n)).astype(np.float32)
        p = net.params().cpu().numpy().astype(np.float64)
        y = net.forward(torch.tensor(x, device="cuda")).cpu().numpy()
        yo = WO.forward(p, chans, K, x.astype(np.float64))[-1]
        assert np.abs(y - yo).max() < 1e-5 * np.abs(yo).max()
        g, loss = net.grad(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"))
        lo, go = WO.loss_and_grad(p, chans, K, x.astype(np.float64), t.astype(np.float64))
        assert abs(loss - lo) < 1e-5 * lo
        g = g.cpu().numpy()
        assert np.abs(g - go).max() < 1e-4 * np.abs(go).max()
        # training lowers the loss
        first = net.train_step(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"), 3e-3)
        for _ in range(60):
            last = net.train_step(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"), 3e-3)
        assert last < 0.5 * first
    finally:
        net.close()


def test_warm_start_reduces_gmres_iterations():
    from paper_1908_07392_gb300 import warmstart as WS
    r = WS.experiment(alpha=50.0, n_panels=48, n_train=96, n_test=12, dt=2e-3, tol=1e-11, epochs=20, batch=8,
                      lr=2e-3, width=32, n_layers=4, ksize=9)
    ev = r["held_out"]
    net, ext = ev["network"], ev["extrapolation"]
    print(f"GMRES iterations: cold {ev['cold']['mean_iters']:.2f}, extrapolation {ext['mean_iters']:.2f}, "
          f"network {net['mean_iters']:.2f}; network residual / extrapolation residual "
          f"{net['residual_ratio_vs_extrapolation']:.3f}, kept {net['kept_fraction']:.2f}")
    assert ext["mean_iters"] < ev["cold"]["mean_iters"]
    assert r["final_train_loss"] < r["first_train_loss"]
    # what training adds over the method without it: the trained network's guess (before the
    # safeguard that falls back to the extrapolation) has a smaller residual than the quadratic
    # extrapolation it corrects (geometric mean over the held-out steps), and it is kept on some
    # steps; the guess never costs iterations over the extrapolation
    assert net["residual_ratio_vs_extrapolation"] < 1.0
    assert net["kept_fraction"] > 0.0
    assert net["mean_iters"] <= ext["mean_iters"] + 0.5


def test_augmented_gmres():
    # one augmentation direction: the exact correction solves the system in the least-squares step;
    # an arbitrary direction still converges to the same density; a zero direction is plain GMRES
    import torch
    b = V.BIE(30.0, R=1.0, A=0.3, k=5, phase=0.2, n_panels=32)
    try:
        gen = torch.Generator(device="cuda").manual_seed(3)
        g = torch.randn(2 * b.N, dtype=torch.float64, device="cuda", generator=gen)
        ref, it0, rr0 = b.solve(g, None, 1e-13)
        x0 = 0.9 * ref + 1e-3 * torch.randn(2 * b.N, dtype=torch.float64, device="cuda", generator=gen)
        mu, it, rr = b.solve(g, x0, 1e-13, aug=ref - x0)
        assert rr < 1e-12 and it <= 1
        assert float((mu - ref).abs().max()) < 1e-10 * float(ref.abs().max())
        d = torch.randn(2 * b.N, dtype=torch.float64, device="cuda", generator=gen)
        mu2, it2, rr2 = b.solve(g, x0, 1e-13, aug=d)
        assert rr2 < 1e-12 and float((mu2 - ref).abs().max()) < 1e-10 * float(ref.abs().max())
        mu3, it3, rr3 = b.solve(g, x0, 1e-13, aug=torch.zeros_like(d))
        mu4, it4, rr4 = b.solve(g, x0, 1e-13)
        assert it3 == it4 and torch.equal(mu3, mu4)
    finally:
        b.close()


def test_gmres_reports_non_convergence():
    # an iteration cap below what the tolerance needs: the solver stops there and reports the
    # iterations and the true residual, which the caller compares with the tolerance
    import torch
    b = V.BIE(30.0, n_panels=16)
    try:
        g = torch.ones(2 * b.N, dtype=torch.float64, device="cuda")
        mu, it, rr = b.solve(g, None, 1e-13, max_iter=2)
        assert it == 2 and rr > 1e-13 and bool(torch.isfinite(mu).all())
        mu2, it2, rr2 = b.solve(g, mu, 1e-13)
        assert rr2 < 1e-12
    finally:
        b.close()
