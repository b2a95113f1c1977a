"""Learned warm start for the per-step boundary integral equation.

A sequence of steps n = 0, 1, ... each solves (1/2 + D + W) mu_n = g_n by GMRES (library). The
network (library kernels) sees the last density, its first and second backward differences, the
current boundary data and the residual of the quadratic extrapolation 3 mu_{n-1} - 3 mu_{n-2} +
mu_{n-3} (one operator apply), each over a fixed scale, and predicts the correction to that
extrapolation. The correction is used either added to the extrapolation as the initial guess (kept
only if its residual is smaller) or as an augmentation direction of GMRES started at the
extrapolation (bie_solve_aug). The network is trained on densities that plain (cold-start) GMRES
solves produce. Plain GMRES to the same residual stays the solver and decides when the result is
accurate enough: the network only changes where, and along which extra direction, GMRES starts.
"""
from __future__ import annotations

import time

import numpy as np

from . import BIE, VP_PREC_FP64, VolumePotential, WarmStartNet, bie_stokeslets
from . import inputs as I


def boundary_data(bie, forcing, times):
    """g_n at the boundary nodes for each time (device, [steps][2N] interleaved per node)."""
    import torch
    xy = bie.nodes[0:2].contiguous()
    out = []
    for t in times:
        src, f = forcing(t)
        u = bie_stokeslets(bie.alpha, torch.tensor(src, device="cuda"), torch.tensor(f, device="cuda"), xy)
        out.append(u.t().contiguous().reshape(-1))    # (x, y) per node
    return torch.stack(out)


def plain_solves(bie, G, tol):
    import torch
    mus, its = [], []
    for g in G:
        mu, it, rr = bie.solve(g, None, tol)
        if not rr <= 10 * tol:
            raise RuntimeError(f"GMRES did not reach the tolerance ({rr:.2e})")
        mus.append(mu); its.append(it)
    return torch.stack(mus), its


def _extrapolation(mus, n):
    return 3 * mus[n - 1] - 3 * mus[n - 2] + mus[n - 3]


def residuals(bie, mus, G, idx):
    """r_n = g_n - A (3 mu_{n-1} - 3 mu_{n-2} + mu_{n-3}) for the steps idx ([len(idx)][2N])."""
    import torch
    return torch.stack([G[n] - bie.apply(_extrapolation(mus, n)) for n in idx])


def _features(mus, G, R, n, scale):
    """Network inputs [B][10][N] for steps n (index tensor), formed in FP64 and then rounded to FP32:
    the last density, its first and second backward differences, the boundary data and the residual
    R of the quadratic extrapolation (rows matching n), each over its own fixed scale (differences are
    scaled separately so that FP32 keeps them); and the extrapolation itself [B][2N]."""
    import torch
    N = mus.shape[1] // 2
    m1, m2, m3 = mus[n - 1], mus[n - 2], mus[n - 3]
    parts = [(m1, "s_mu"), (m1 - m2, "s_d1"), (m1 - 2 * m2 + m3, "s_d2"), (G[n], "s_g"), (R, "s_r")]
    ch = [(v / scale[k]).reshape(-1, N, 2).permute(0, 2, 1) for v, k in parts]
    x = torch.cat(ch, dim=1).float().contiguous()
    return x, _extrapolation(mus, n)


IN_CHANNELS = 10


def train(bie, net, mus, G, train_idx, epochs=40, batch=16, lr=1e-3, seed=0):
    import torch
    N = mus.shape[1] // 2
    R = torch.zeros_like(mus)
    R[train_idx] = residuals(bie, mus, G, train_idx)
    err = mus[train_idx] - _extrapolation(mus, train_idx)
    d1 = mus[train_idx - 1] - mus[train_idx - 2]
    d2 = mus[train_idx - 1] - 2 * mus[train_idx - 2] + mus[train_idx - 3]
    scale = {k: (float(v.std()) or 1.0) for k, v in
             (("s_mu", mus[train_idx]), ("s_d1", d1), ("s_d2", d2), ("s_g", G[train_idx]), ("s_r", R[train_idx]),
              ("s_err", err))}
    rng = np.random.default_rng(seed)
    losses = []
    for ep in range(epochs):
        order = rng.permutation(train_idx)
        for k in range(0, len(order) - batch + 1, batch):
            n = torch.tensor(order[k:k + batch], device="cuda")
            x, ext = _features(mus, G, R[n], n, scale)
            t = ((mus[n] - ext).reshape(-1, N, 2).permute(0, 2, 1) / scale["s_err"]).float().contiguous()
            losses.append(net.train_step(x, t, lr))
    return dict(scale, losses=losses)


def correction(bie, net, scale, mus, G, n):
    """The extrapolation for step n, the network's correction to it (device [2N] each) and the
    extrapolation's residual."""
    import torch
    idx = torch.tensor([n], device="cuda")
    r = residuals(bie, mus, G, [n])
    x, ext = _features(mus, G, r, idx, scale)
    y = net.forward(x)[0]                                   # [2][N]
    return ext[0], scale["s_err"] * y.permute(1, 0).reshape(-1).double(), r[0]


def guess(bie, net, scale, mus, G, n):
    """Network guess for step n, kept only if its residual is below that of the extrapolation
    (one extra operator apply); returns (guess, whether the network's guess was kept, the ratio of
    the two residual norms)."""
    ext, d, r = correction(bie, net, scale, mus, G, n)
    cand = ext + d
    rc = G[n] - bie.apply(cand)
    ratio = float(rc.norm()) / max(float(r.norm()), 1e-300)
    if ratio < 1.0:
        return cand, True, ratio
    return ext, False, ratio


def evaluate(bie, net, scale, mus, G, test_idx, tol, rhs=None):
    """GMRES iterations and solve times from each initial guess on the held-out steps. With rhs
    (n -> (g_n, ms)), the right-hand side is recomputed per step and its time added to every method."""
    import torch
    res = {k: {"iters": [], "ms": []} for k in ("cold", "previous", "extrapolation", "network", "network_aug")}
    kept, ratios = 0, []
    # one untimed pass through every path first (library and torch kernels load on first use)
    n0 = test_idx[0]
    (G[n0], 0.0) if rhs is None else rhs(n0)
    g0, _, _ = guess(bie, net, scale, mus, G, n0)
    bie.solve(G[n0], g0, tol)
    e0, d0, _ = correction(bie, net, scale, mus, G, n0)
    bie.solve(G[n0], e0, tol, aug=d0)
    torch.cuda.synchronize()
    for n in test_idx:
        g, t_rhs = (G[n], 0.0) if rhs is None else rhs(n)
        guesses = {
            "cold": None,
            "previous": mus[n - 1],
            "extrapolation": _extrapolation(mus, n),
        }
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        guesses["network"], used, ratio = guess(bie, net, scale, mus, G, n)
        kept += int(used)
        ratios.append(ratio)
        torch.cuda.synchronize()
        t_net = time.perf_counter() - t0
        for k, x0 in guesses.items():
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            mu, it, rr = bie.solve(g, x0, tol)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0 + (t_net if k == "network" else 0.0) + t_rhs / 1000.0
            if not rr <= 10 * tol:
                raise RuntimeError(f"GMRES from the {k} guess did not reach the tolerance ({rr:.2e})")
            res[k]["iters"].append(it)
            res[k]["ms"].append(1000 * dt)
        # the network's correction as an augmentation direction of GMRES started at the extrapolation
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ext, d, _ = correction(bie, net, scale, mus, G, n)
        mu, it, rr = bie.solve(g, ext, tol, aug=d)
        torch.cuda.synchronize()
        if not rr <= 10 * tol:
            raise RuntimeError(f"augmented GMRES did not reach the tolerance ({rr:.2e})")
        res["network_aug"]["iters"].append(it)
        res["network_aug"]["ms"].append(1000 * (time.perf_counter() - t0) + t_rhs)
    out = {k: {"mean_iters": float(np.mean(v["iters"])), "max_iters": int(np.max(v["iters"])),
               "mean_ms": float(np.mean(v["ms"]))} for k, v in res.items()}
    out["network"]["kept_fraction"] = kept / max(1, len(test_idx))
    out["network"]["residual_ratio_vs_extrapolation"] = float(np.exp(np.mean(np.log(ratios))))
    return out


def experiment(alpha, n_panels=256, n_train=2000, n_test=200, dt=1e-3, tol=1e-11, epochs=40, batch=16,
               lr=1e-3, seed=5, width=64, n_layers=4, ksize=9):
    """Plain solves for n_train + n_test + 3 steps of a star with moving exterior forcing, network
    training on the first n_train, iterations and times from each initial guess on the rest."""
    rng = np.random.default_rng(seed)
    bie = BIE(alpha, R=1.0, A=0.3, k=5, phase=float(rng.uniform(0, 2 * np.pi)), n_panels=n_panels, max_krylov=300)
    try:
        forcing = I.moving_stokeslets(seed)
        steps = n_train + n_test + 3
        times = dt * np.arange(steps)
        t0 = time.perf_counter()
        G = boundary_data(bie, forcing, times)
        mus, its = plain_solves(bie, G, tol)
        t_plain = time.perf_counter() - t0
        net = WarmStartNet(in_ch=IN_CHANNELS, width=width, out_ch=2, n_layers=n_layers, ksize=ksize, n=bie.N,
                           max_batch=batch, seed=seed)
        try:
            t0 = time.perf_counter()
            scale = train(bie, net, mus, G, np.arange(3, 3 + n_train), epochs=epochs, batch=batch, lr=lr, seed=seed)
            t_train = time.perf_counter() - t0
            test_idx = np.arange(3 + n_train, steps)
            ev = evaluate(bie, net, scale, mus, G, test_idx, tol)
        finally:
            net.close()
        return {"nodes": bie.N, "alpha": alpha, "n_train": n_train, "n_test": n_test, "tol": tol,
                "plain_mean_iters": float(np.mean(its)), "plain_seconds": t_plain, "train_seconds": t_train,
                "final_train_loss": float(np.mean(scale["losses"][-20:])), "first_train_loss": float(scale["losses"][0]),
                "held_out": ev}
    finally:
        bie.close()


# --------------------------------------------------------------------------- coupled steps

class StepProblem:
    """Per-step right-hand side of the homogeneous problem (Sec. 2.2): the boundary velocity minus
    the particular solution u^P = (d Psi/dy, -d Psi/dx), Psi the volume potential (modified-
    biharmonic kernel) of the step's vorticity source, carried to the boundary nodes through the
    leaf interpolants."""

    def __init__(self, wl, bie, precision=VP_PREC_FP64):
        import torch
        self.wl, self.bie = wl, bie
        self.vp = VolumePotential(I.KERNEL_MBIHARMONIC, wl.alpha, wl.p, wl.tree, precision=precision)
        xy = self.vp.nodes()
        self.X, self.Y = xy[0], xy[1]
        self.bxy = bie.nodes[0:2].contiguous()
        self.u = torch.empty(self.vp.N, dtype=torch.float64, device="cuda")
        self.gradu = torch.empty(2, self.vp.N, dtype=torch.float64, device="cuda")

    def rhs(self, t):
        """g at time t (device [2N], interleaved per node) and the time of the volume part (ms)."""
        import torch
        f = self.wl.source(self.X, self.Y, t)
        src, fs = self.wl.boundary(t)
        ubc = bie_stokeslets(self.bie.alpha, torch.tensor(src, device="cuda"), torch.tensor(fs, device="cuda"),
                             self.bxy)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        self.vp(f, self.u, self.gradu)
        d = self.vp.interp(self.gradu, self.bxy)
        g = (ubc - torch.stack([d[1], -d[0]])).t().contiguous().reshape(-1)
        e1.record()
        e1.synchronize()
        return g, e0.elapsed_time(e1)

    def close(self):
        self.vp.close()


def step_experiment(wl, n_panels=256, n_train=2000, n_test=200, tol=1e-11, precision=VP_PREC_FP64, epochs=40,
                    batch=16, lr=1e-3, seed=5, width=64, n_layers=4, ksize=9, log=None):
    """Steps of the coupled problem: plain solves for n_train + n_test + 3 steps, network training on
    the first n_train, then per held-out step the volume potential, its boundary trace and GMRES from
    each initial guess (step time = volume part + guess + GMRES)."""
    import torch
    bie = BIE(wl.alpha, R=1.0, A=0.3, k=5, phase=wl.phi, n_panels=n_panels, max_krylov=300)
    prob = None
    try:
        prob = StepProblem(wl, bie, precision)
        steps = n_train + n_test + 3
        times = wl.dt * np.arange(steps)
        t0 = time.perf_counter()
        G, vp_ms = [], []
        for k, t in enumerate(times):
            g, ms = prob.rhs(float(t))
            G.append(g); vp_ms.append(ms)
            if log and k % 500 == 0:
                log(f"rhs {k}/{steps}")
        G = torch.stack(G)
        t_rhs = time.perf_counter() - t0
        t0 = time.perf_counter()
        mus, its = plain_solves(bie, G, tol)
        t_plain = time.perf_counter() - t0
        if log:
            log(f"plain solves: mean {np.mean(its):.1f} iterations, {t_plain:.1f} s")
        net = WarmStartNet(in_ch=IN_CHANNELS, width=width, out_ch=2, n_layers=n_layers, ksize=ksize, n=bie.N,
                           max_batch=batch, seed=seed)
        try:
            t0 = time.perf_counter()
            scale = train(bie, net, mus, G, np.arange(3, 3 + n_train), epochs=epochs, batch=batch, lr=lr, seed=seed)
            t_train = time.perf_counter() - t0
            if log:
                log(f"training: {t_train:.1f} s, loss {scale['losses'][0]:.3e} -> {np.mean(scale['losses'][-20:]):.3e}")
            test_idx = np.arange(3 + n_train, steps)
            ev = evaluate(bie, net, scale, mus, G, test_idx, tol, rhs=lambda n: prob.rhs(float(times[n])))
        finally:
            net.close()
        return {"nodes": bie.N, "volume_nodes": prob.vp.N, "alpha": wl.alpha, "n_train": n_train, "n_test": n_test,
                "tol": tol, "plain_mean_iters": float(np.mean(its)), "rhs_seconds": t_rhs,
                "volume_ms_mean": float(np.mean(vp_ms[3:])), "plain_seconds": t_plain, "train_seconds": t_train,
                "final_train_loss": float(np.mean(scale["losses"][-20:])), "first_train_loss": float(scale["losses"][0]),
                "held_out": ev}
    finally:
        if prob is not None:
            prob.close()
        bie.close()


def interior_error(bie, forcing, t, n_targets=64, seed=0, tol=1e-13):
    """Accuracy of the discretisation: data from exterior stokeslets, whose field solves the
    homogeneous problem inside; D[mu] against it at interior targets (radius <= 0.45)."""
    import torch
    src, f = forcing(t)
    S, F = torch.tensor(src, device="cuda"), torch.tensor(f, device="cuda")
    g = bie_stokeslets(bie.alpha, S, F, bie.nodes[0:2].contiguous()).t().contiguous().reshape(-1)
    mu, it, rr = bie.solve(g, None, tol)
    rng = np.random.default_rng(seed)
    r = rng.uniform(0, 0.45, n_targets); th = rng.uniform(0, 2 * np.pi, n_targets)
    tx = torch.tensor(np.stack([r * np.cos(th), r * np.sin(th)]), device="cuda")
    u = bie.eval(mu, tx)
    ue = bie_stokeslets(bie.alpha, S, F, tx)
    return float((u - ue).abs().max() / ue.abs().max()), it
