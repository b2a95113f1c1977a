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

from . import (BIE, VP_PREC_FP64, VolumePotential, WarmStartNet, bie_stokeslets, vp_autotune, vp_layer_create,
               vp_layer_eval, vp_layer_free, vp_layer_near_star)
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


# weights of mu_{n-1}, mu_{n-2}, ... in the extrapolation through the last `order` densities
_EXTRAP = {3: (3.0, -3.0, 1.0), 4: (4.0, -6.0, 4.0, -1.0), 5: (5.0, -10.0, 10.0, -5.0, 1.0)}


def _extrapolation(mus, n, order=3):
    return sum(c * mus[n - 1 - k] for k, c in enumerate(_EXTRAP[order]))


def in_channels(lags=3):
    """Network inputs: the last density, its backward differences up to lags - 1, g_n and r_n."""
    return 2 * (lags + 2)


def residuals(bie, mus, G, idx, order=3):
    """r_n = g_n - A (extrapolation of mu_n from the last `order` densities) for the steps idx."""
    import torch
    return torch.stack([G[n] - bie.apply(_extrapolation(mus, n, order)) for n in idx])


def _differences(mus, n, order):
    """mu_{n-1} and its backward differences of order 1 .. order-1 (FP64)."""
    lags = [mus[n - 1 - k] for k in range(order)]
    out = [lags[0]]
    cur = lags
    for _ in range(order - 1):
        cur = [cur[k] - cur[k + 1] for k in range(len(cur) - 1)]
        out.append(cur[0])
    return out


def _features(mus, G, R, n, scale):
    """Network inputs [B][2 (lags + 2)][N] for steps n (index tensor), formed in FP64 and then
    rounded to FP32: the last density, its backward differences over the last `lags` densities, the
    boundary data and the residual R of the extrapolation (rows matching n), each over its own fixed
    scale (differences are scaled separately so that FP32 keeps them); and the extrapolation through
    the last `order` densities itself [B][2N]."""
    import torch
    order, lags = scale["order"], scale["lags"]
    N = mus.shape[1] // 2
    parts = [(v, f"s_d{k}") for k, v in enumerate(_differences(mus, n, lags))] + [(G[n], "s_g"), (R, "s_r")]
    ch = [(v / scale[k]).reshape(-1, N, 2).permute(0, 2, 1) for v, k in parts]
    x = torch.cat(ch, dim=1).float().contiguous()
    return x, _extrapolation(mus, n, order)


IN_CHANNELS = in_channels(3)


def train(bie, net, mus, G, train_idx, epochs=40, batch=16, lr=1e-3, seed=0, order=3, lags=None):
    """Adam on the network's correction to the extrapolation through the last `order` densities, from
    features of the last `lags` densities (default `order`; train_idx >= both)."""
    import torch
    lags = order if lags is None else lags
    N = mus.shape[1] // 2
    R = torch.zeros_like(mus)
    R[train_idx] = residuals(bie, mus, G, train_idx, order)
    err = mus[train_idx] - _extrapolation(mus, train_idx, order)
    scale = {"order": order, "lags": lags}
    for k, v in enumerate(_differences(mus, train_idx, lags)):
        scale[f"s_d{k}"] = float(v.std()) or 1.0
    for k, v in (("s_g", G[train_idx]), ("s_r", R[train_idx]), ("s_err", err)):
        scale[k] = float(v.std()) or 1.0
    rng = np.random.default_rng(seed)
    losses = []
    for ep in range(epochs):
        perm = rng.permutation(train_idx)
        for k in range(0, len(perm) - batch + 1, batch):
            n = torch.tensor(perm[k:k + batch], device="cuda")
            x, ext = _features(mus, G, R[n], n, scale)
            t = ((mus[n] - ext).reshape(-1, N, 2).permute(0, 2, 1) / scale["s_err"]).float().contiguous()
            losses.append(net.train_step(x, t, lr))
    return dict(scale, losses=losses)


def correction(bie, net, scale, mus, G, n):
    """The extrapolation for step n, the network's correction to it (device [2N] each) and the
    extrapolation's residual."""
    import torch
    idx = torch.tensor([n], device="cuda")
    r = residuals(bie, mus, G, [n], scale["order"])
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


def evaluate(bie, nets, mus, G, test_idx, tol, rhs=None, post=None):
    """GMRES iterations and solve times from each initial guess on the held-out steps: cold, previous
    density, extrapolation through the last 3, 4 and 5 densities, and for every (name -> (net, scale))
    in nets the network's guess ("name") and its correction as an augmentation direction
    ("name_aug"). With rhs (n -> (g_n, ms)), the right-hand side is recomputed per step and its time
    added to every method; with post (mu -> ms), the step's velocity is formed from each solution and
    its time added as well."""
    import torch
    names = ["cold", "previous", "extrapolation", "cubic", "quartic"]
    for nm in nets:
        names += [nm, nm + "_aug"]
    res = {k: {"iters": [], "ms": [], "post_ms": []} for k in names}
    kept = {nm: 0 for nm in nets}
    ratios = {nm: [] for nm in nets}
    # one untimed pass through every path first (library and torch kernels load on first use)
    n0 = test_idx[0]
    (G[n0], 0.0) if rhs is None else rhs(n0)
    for net, scale in nets.values():
        g0, _, _ = guess(bie, net, scale, mus, G, n0)
        bie.solve(G[n0], g0, tol)
        e0, d0, _ = correction(bie, net, scale, mus, G, n0)
        bie.solve(G[n0], e0, tol, aug=d0)
    torch.cuda.synchronize()

    def solve(name, x0, extra_s, t_rhs, aug=None):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mu, it, rr = bie.solve(g, x0, tol, aug=aug)
        torch.cuda.synchronize()
        if not rr <= 10 * tol:
            raise RuntimeError(f"GMRES ({name}) did not reach the tolerance ({rr:.2e})")
        solve_s = time.perf_counter() - t0
        t_post = post(mu) if post is not None else 0.0
        res[name]["iters"].append(it)
        res[name]["ms"].append(1000 * (solve_s + extra_s) + t_rhs + t_post)
        res[name]["post_ms"].append(t_post)

    for n in test_idx:
        g, t_rhs = (G[n], 0.0) if rhs is None else rhs(n)
        solve("cold", None, 0.0, t_rhs)
        solve("previous", mus[n - 1], 0.0, t_rhs)
        solve("extrapolation", _extrapolation(mus, n, 3), 0.0, t_rhs)
        solve("cubic", _extrapolation(mus, n, 4), 0.0, t_rhs)
        solve("quartic", _extrapolation(mus, n, 5), 0.0, t_rhs)
        for nm, (net, scale) in nets.items():
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x0, used, ratio = guess(bie, net, scale, mus, G, n)
            torch.cuda.synchronize()
            kept[nm] += int(used)
            ratios[nm].append(ratio)
            solve(nm, x0, time.perf_counter() - t0, t_rhs)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ext, d, _ = correction(bie, net, scale, mus, G, n)
            torch.cuda.synchronize()
            solve(nm + "_aug", ext, time.perf_counter() - t0, t_rhs, aug=d)
    out = {k: {"mean_iters": float(np.mean(v["iters"])), "max_iters": int(np.max(v["iters"])),
               "mean_ms": float(np.mean(v["ms"])), "velocity_ms": float(np.mean(v["post_ms"]))} for k, v in res.items()}
    for nm in nets:
        out[nm]["kept_fraction"] = kept[nm] / max(1, len(test_idx))
        out[nm]["residual_ratio_vs_extrapolation"] = float(np.exp(np.mean(np.log(ratios[nm]))))
    return out


# (name, extrapolation order corrected, past densities seen, layers, kernel width, channels)
SPEC_NETWORK = ("network", 3, 3, 4, 9, 64)            # the configuration's network
STEP_SPECS = (SPEC_NETWORK,
              ("network4", 4, 4, 4, 9, 64),           # the same one order up
              ("network8", 5, 8, 4, 9, 64),           # eight past densities, correcting the quartic
              ("temporal8", 5, 8, 1, 1, 1))           # a learned linear filter over eight past densities


def _train_nets(bie, mus, G, n_train, specs, epochs, batch, lr, seed):
    """One network per spec (name, order, lags, layers, ksize, width), trained on steps
    max(order, lags) .. n_train + 2. Returns ({name: (net, scale)}, seconds, the first scale)."""
    nets = {}
    t0 = time.perf_counter()
    try:
        for name, order, lags, n_layers, ksize, width in specs:
            net = WarmStartNet(in_ch=in_channels(lags), width=width, out_ch=2, n_layers=n_layers, ksize=ksize,
                               n=bie.N, max_batch=batch, seed=seed)
            nets[name] = (net, None)
            scale = train(bie, net, mus, G, np.arange(max(order, lags), 3 + n_train), epochs=epochs, batch=batch,
                          lr=lr, seed=seed, order=order, lags=lags)
            nets[name] = (net, scale)
    except Exception:
        for net, _ in nets.values():
            net.close()
        raise
    first = next(iter(nets.values()))[1]
    return nets, time.perf_counter() - t0, first


def experiment(alpha, n_panels=256, n_train=2000, n_test=200, dt=1e-3, tol=1e-11, epochs=40, batch=16,
               lr=1e-3, seed=5, width=64, n_layers=4, ksize=9, specs=None):
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
        if specs is None:
            specs = (("network", 3, 3, n_layers, ksize, width),)
        nets, t_train, scale = _train_nets(bie, mus, G, n_train, specs, epochs, batch, lr, seed)
        try:
            test_idx = np.arange(3 + n_train, steps)
            ev = evaluate(bie, nets, mus, G, test_idx, tol)
        finally:
            for net, _ in nets.values():
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
        if precision != VP_PREC_FP64:
            # contraction engine per launch shape, chosen once for this tree
            vp_autotune(self.vp.tree, self.wl.source(self.X, self.Y, 0.0), self.u, self.gradu)
        # the homogeneous part at the volume nodes: the double layer of the boundary density, with the
        # near-boundary correction for the nodes within 1.2 panel lengths of the boundary
        self.layer = vp_layer_create(self.vp.tree, bie.nodes[0:5].cpu().numpy())
        self.near_pairs = vp_layer_near_star(self.layer, 1.0, 0.3, 5, wl.phi, bie.N // 16, 1.2)
        self.uh = torch.empty(2, self.vp.N, dtype=torch.float64, device="cuda")
        self.vel = torch.empty(2, self.vp.N, dtype=torch.float64, device="cuda")

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

    def velocity(self, mu):
        """The step's velocity at every volume node, u = u^P + u^H (Sec. 2.2): u^P = (dPsi/dy, -dPsi/dx)
        from the last rhs() and u^H = D[mu] by the layer potential on the tree; returns the time (ms)."""
        import torch
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        vp_layer_eval(self.layer, mu, self.uh)
        self.vel[0] = self.gradu[1] + self.uh[0]
        self.vel[1] = self.uh[1] - self.gradu[0]
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1)

    def close(self):
        vp_layer_free(self.layer)
        self.vp.close()


def step_experiment(wl, n_panels=256, n_train=2000, n_test=200, tol=1e-11, precision=VP_PREC_FP64, epochs=40,
                    batch=16, lr=1e-3, seed=5, width=64, n_layers=4, ksize=9, log=None, specs=STEP_SPECS):
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
        if specs is None:
            specs = (("network", 3, 3, n_layers, ksize, width),)
        nets, t_train, scale = _train_nets(bie, mus, G, n_train, specs, epochs, batch, lr, seed)
        try:
            if log:
                log(f"training: {t_train:.1f} s, loss {scale['losses'][0]:.3e} -> {np.mean(scale['losses'][-20:]):.3e}")
            test_idx = np.arange(3 + n_train, steps)
            ev = evaluate(bie, nets, mus, G, test_idx, tol, rhs=lambda n: prob.rhs(float(times[n])), post=prob.velocity)
        finally:
            for net, _ in nets.values():
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
