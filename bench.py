"""Benchmark: volume-potential leaf-nodes/s on one GB300 (or N replicas).

Workload (the single-GPU configuration the metric is quoted on): modified-
biharmonic kernel G2 = (K0(alpha r) + log r)/(2 pi alpha^2), alpha = 300, box
[-1.5, 1.5]^2, p = 16 Gauss-Legendre nodes per leaf side, tree refined until
the leaf Legendre tail is below 1e-11 (max depth 10) for a seeded star-shaped
source with a C-infinity blend of width 0.05 plus 20 narrow Gaussians.

A step is one vp_eval (every stage of the volume potential) over the resident
source. L2 is flushed (a 512 MB write) before every timed step. By default the
headline value is the split-precision form (sliced bf16 tensor-core
contractions, 1e-9 against the FP64 oracle) and the plain FP64 form (1e-10) is
measured beside it in the same run ("plain_fp64", "split_speedup_vs_fp64").
The dominant kernel (the near-field table contraction) is timed live with CUDA
events on the launching stream (vp_eval_timed). The e2e figure runs
vp_eval_host from pinned host buffers (host-to-device copy of f and
device-to-host copy of u and grad u inside the timed region). The CPU baseline
is the FP64 oracle on a bounded sample of targets of the same workload.

Other workloads: --workload batched (64 trees in one CUDA graph),
--workload steps (coupled volume potential + boundary integral equation steps
with the learned GMRES warm start) and --workload periodic (the periodic FFT
solution and SISDC steps alone).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                       [--precision both|fp64|split] [--workload star|batched|steps|periodic]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP64_FLOPS_PER_CLK_PER_SM = 4.0   # 2 DFMA per clock per SM: 1.25 TFLOP/s nominal over 152 SMs at ~2.06 GHz
# DRAM bytes of one FP64 near-field launch on the default workload, NOT measured in this run: a past ncu
# capture of the same kernel at depth 8 (688 MB for 66.6k near pairs, profiles/near_f64_star_d8.md) scaled
# by pairs to the 356k pairs at depth 10.
TRAFFIC_FP64_NEAR = 3.68e9
TRAFFIC_FP64_NEAR_SOURCE = "constant from a past ncu capture (profiles/near_f64_star_d8.md, depth 8 scaled by near pairs)"
# DRAM bytes of the split-precision near-field launch (tcgen05 engine) per algorithmic GFLOP of the near
# stage, NOT measured in this run: the ncu capture of the same kernel at depth 8 (419.3 MB read + 419.2
# MB written for 29.33 GFLOP, profiles/near_tc_star_d8.md); traffic grows with the near pairs, i.e. with
# the stage's flops.
TRAFFIC_SPLIT_NEAR_PER_GFLOP = 838.5e6 / 29.33
TRAFFIC_SPLIT_NEAR_SOURCE = ("constant from an ncu capture (profiles/near_tc_star_d8.md, depth 8, 838.5 MB for 29.33 "
                             "GFLOP) scaled by the near stage's flops")
N_SM = 152
ENGINE_NAMES = {-1: "-", 0: "mma.sync 128x64", 1: "tcgen05 128x128", 2: "mma.sync 64x32", 3: "tcgen05 128x64",
                4: "tcgen05 transposed 128x128"}


def launch_list_engine(launch_list, table):
    """Engine of the (first) split contraction on operator table `table` in a launch list, or -1."""
    for x in launch_list:
        if x["kind"] == 4 and x["table"] == table:
            return x["engine"]
    return -1
SLICE_PRODUCTS = 21  # S (S + 1) / 2 slice products per contraction, S = 6 bf16 slices


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--alpha", type=float, default=300.0)
    ap.add_argument("--precision", default="both", choices=["both", "fp64", "split"],
                    help="both (default): split-precision headline plus the plain FP64 form beside it")
    ap.add_argument("--order", type=int, default=40)
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched workload that the default run measures beside the headline")
    ap.add_argument("--max-depth", type=int, default=10, help="tree depth cap (10 = the stated workload)")
    ap.add_argument("--workload", default="star", choices=["star", "batched", "steps", "periodic"],
                    help="star: one adaptive tree (default); batched: 64 trees in one CUDA graph; "
                         "steps: coupled volume potential + boundary solve with the learned warm start")
    ap.add_argument("--train-steps", type=int, default=2000, help="steps workload: plain solves to train on")
    ap.add_argument("--test-steps", type=int, default=200, help="steps workload: held-out steps")
    ap.add_argument("--epochs", type=int, default=40, help="steps workload: training epochs")
    ap.add_argument("--streams", type=int, default=64, help="graph branches for the batched workload")
    ap.add_argument("--engine", default="auto", choices=["auto", "mma", "tcgen05"],
                    help="split-precision GEMM engine: autotuned per launch, mma.sync, or tcgen05")
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def job_totals(units, total_ms, world, device):
    """Whole-job totals over the ranks: units summed, timed milliseconds maxed (value = units / max)."""
    if world <= 1:
        return float(units), float(total_ms)
    import torch
    import torch.distributed as dist
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    m = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return float(u.item()), float(m.item())


def barrier(world):
    """Barrier over the ranks (if any) and a device synchronise."""
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    if torch.cuda.is_available():
        torch.cuda.synchronize()


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def workload(alpha, max_depth=10):
    from paper_1908_07392_gb300 import inputs as I
    return I.star_adaptive_workload(seed=2, alpha=alpha, p=16, tol=1e-11, max_depth=max_depth)


def workload_desc(w):
    import numpy as np
    return {"workload": f"star_adaptive_p{w.p}_a{w.alpha:g}", "kernel": "modified-biharmonic G2",
            "alpha": w.alpha, "p": w.p, "leaves": int(w.tree.n_leaves), "nodes": int(w.n_nodes),
            "max_depth": int(w.tree.max_level), "box": "[-1.5,1.5]^2",
            "levels": {int(l): int(c) for l, c in enumerate(np.bincount(w.tree.level)) if c}}


def cpu_sample(w, budget_s, seed=0):
    """Time the oracle on a bounded random sample of targets; returns (targets/s, n, cores, seconds)."""
    import numpy as np
    import oracle
    from paper_1908_07392_gb300 import inputs as I
    oracle.build()
    X, Y = I.node_coords(w.tree, w.p)
    rng = np.random.default_rng(seed)
    cores = oracle.num_threads()
    one = getattr(cpu_sample, "one", None)
    if one is None:
        # seconds of one target on one thread, probed once per process
        t0 = time.perf_counter()
        idx = rng.choice(w.n_nodes, 1, replace=False)
        oracle.volume_potential(w.kernel, w.alpha, w.p, w.tree, w.f, X[idx], Y[idx], nthreads=1)
        one = cpu_sample.one = max(time.perf_counter() - t0, 1e-3)
    n = int(max(cores, min(4096, budget_s / one * cores * 0.8)))
    idx = rng.choice(w.n_nodes, n, replace=False)
    t0 = time.perf_counter()
    vals = oracle.volume_potential(w.kernel, w.alpha, w.p, w.tree, w.f, X[idx], Y[idx])
    dt = time.perf_counter() - t0
    cpu_sample.last = (idx, vals)   # sampled nodes and the oracle's (u, du/dx, du/dy) there
    return n / dt, n, cores, dt


def sampled_errors(idx, vals, u, g):
    """Per-field relative max-norm error of the GPU result on the sampled nodes (u, gradu host)."""
    import numpy as np
    out = {}
    for name, a, b in (("u", u[idx], vals[0]), ("dudx", g[0][idx], vals[1]), ("dudy", g[1][idx], vals[2])):
        out[name] = float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
    out["nodes"] = int(len(idx))
    return out


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(os.environ.get("BENCH_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"vp_bench_clocks_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            # start timing only once the sampler is producing lines
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < 3.0 and os.path.getsize(self.path) == 0:
                time.sleep(0.05)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1])); mx.append(float(r[2]))
            except Exception:
                continue
            for k, name in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(name)
        if sm:
            out["sm_mhz"] = statistics.median(sm)
            out["sm_max_mhz"] = max(mx)
            out["samples"] = len(sm)
        out["reasons"] = sorted(reasons)
        return out


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    w = workload(args.alpha, args.max_depth)
    per_step = []
    for _ in range(args.warmup):
        cpu_sample(w, min(args.cpu_seconds, 5.0), seed=1)
    n_total = 0
    budget = max(2.0, args.cpu_seconds * 4 / max(1, args.steps))
    t_total = 0.0
    cores = 1
    for k in range(args.steps):
        rate, n, cores, dt = cpu_sample(w, budget, seed=100 + k)
        per_step.append(dt)
        n_total += n
        t_total += dt
    value = n_total / t_total
    line = {"impl": "reference", "metric": "volume-potential leaf-nodes/s at stated rel err, split/batched vs plain FP64",
            "value": value, "unit": "nodes/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * t_total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_desc(w),
            "cpu_baseline": {"value": value, "unit": "nodes/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n_total} random target nodes over {args.steps} steps (direct quadrature per target)"},
            "e2e": {"value": value, "unit": "nodes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def choose_engine(V, args, tree, f, u, g):
    """Engine of the split-precision contractions; returns the number of launches on tcgen05."""
    if args.engine == "mma":
        V.vp_tree_set_engine(tree, V.ENGINE_MMA_SYNC)
        return 0
    if args.engine == "tcgen05":
        V.vp_tree_set_engine(tree, V.ENGINE_TCGEN05)
        return -1
    return V.vp_autotune(tree, f, u, g)


def batched_form(args, V, ws, prec, local, world=1):
    """One form (FP64 or split) of the batched workload: graph replay timed per step, L2 flushed."""
    import torch
    t0 = time.perf_counter()
    vps = [V.VolumePotential(w.kernel, w.alpha, w.p, w.tree, order=args.order, precision=prec) for w in ws]
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    batch = None
    try:
        fs = [torch.from_numpy(w.f).cuda() for w in ws]
        us = [torch.empty_like(f) for f in fs]
        gs = [torch.empty(2, f.numel(), dtype=torch.float64, device="cuda") for f in fs]
        trees = [vp.tree for vp in vps]
        n_tc = sum(choose_engine(V, args, vp.tree, f, u, g) for vp, f, u, g in zip(vps, fs, us, gs)) \
            if prec == V.VP_PREC_SPLIT else 0
        batch = V.vp_batch_create(trees, fs, us, gs, n_streams=args.streams)
        nodes, launches = V.vp_batch_stats(batch)
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        stream = torch.cuda.current_stream()

        def timed(fn):
            for _ in range(args.warmup):
                fn()
            barrier(world)
            total = 0.0
            for _ in range(args.steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream); fn(); e1.record(stream); e1.synchronize()
                total += e0.elapsed_time(e1)
            barrier(world)
            return total

        sampler = ClockSampler(local)
        with sampler:
            graph_ms = timed(lambda: V.vp_batch_run(batch))
        serial_ms = timed(lambda: V.vp_eval_batched(trees, fs, us, gs, use_graph=0))
        nodes_all, graph_ms = job_totals(nodes, graph_ms, world, "cuda")
        _, serial_ms = job_totals(nodes, serial_ms, world, "cuda")
        # dominant kernel: the near-field contraction of the largest tree, timed with events
        big = max(range(len(ws)), key=lambda k: ws[k].n_nodes)
        ms = [V.vp_eval_timed(vps[big].tree, fs[big], us[big], gs[big]) for _ in range(3)]
        _, sf = V.vp_tree_stats(vps[big].tree)
        near_ms = statistics.mean(m[4] for m in ms)
        if prec == V.VP_PREC_FP64:
            achieved = sf[4] / (near_ms / 1e3) / 1e12
            peak = N_SM * 2070.0e6 * FP64_FLOPS_PER_CLK_PER_SM / 1e12
            roof = {"kernel": "k_gemm_gather_f64<1> (near tables, largest tree)", "bound": "alu"}
        else:
            achieved = sf[4] * 21 / (near_ms / 1e3) / 1e12
            peak = measured_peaks().get("bf16_tflops", 1900.0)
            roof = {"kernel": "split-precision near GEMM, engine per launch (largest tree)", "bound": "tensor",
                    "peak_source": "measured dense bf16 burst, of measured"}
        return {"nodes": int(nodes), "nodes_all": nodes_all, "launches": int(launches), "graph_ms": graph_ms,
                "serial_ms": serial_ms,
                "setup_s": setup_s, "n_tc": n_tc, "clocks": sampler.summary(),
                "roofline": dict(roof, achieved=achieved, peak=peak, unit="TFLOP/s", frac=achieved / peak,
                                 traffic=None)}
    finally:
        if batch is not None:
            V.vp_batch_free(batch)
        for vp in vps:
            vp.close()


def batched_pair(args, V, local, world):
    """Both forms of the batched workload with fewer steps than the headline (its own L2 flush and clock
    record per form), as an extra object of the headline line."""
    from paper_1908_07392_gb300 import inputs as I
    import copy
    rank = int(os.environ.get("RANK", "0"))
    a = copy.copy(args)
    a.steps = max(3, min(args.steps, 10))
    a.warmup = max(3, min(args.warmup, 3))
    ws = I.batched_workloads(seed=4 + rank)
    sp = batched_form(a, V, ws, V.VP_PREC_SPLIT, local, world)
    fp = batched_form(a, V, ws, V.VP_PREC_FP64, local, world)
    sv = sp["nodes_all"] * a.steps / (sp["graph_ms"] / 1000.0)
    fv = fp["nodes_all"] * a.steps / (fp["graph_ms"] / 1000.0)
    return {"workload": "batched: 64 trees, nodes log-uniform [1e4, 5e5], alpha log-uniform [10, 1000], "
                        "p in {8, 12, 16}, modified-Helmholtz kernel, Gaussian-sum sources, one CUDA graph",
            "trees": len(ws), "nodes": sp["nodes"], "steps": a.steps, "warmup": a.warmup, "streams": a.streams,
            "l2": "flushed before every timed step (512 MB write)",
            "split": {"value": sv, "unit": "nodes/s", "ms_per_step": sp["graph_ms"] / a.steps,
                      "serial_ms_per_step": sp["serial_ms"] / a.steps, "gpu_launches_per_step": sp["launches"],
                      "tcgen05_launches": sp["n_tc"], "stated_rel_err": 1e-9, "roofline": sp["roofline"],
                      "clocks": sp["clocks"], "setup_s": round(sp["setup_s"], 1)},
            "plain_fp64": {"value": fv, "unit": "nodes/s", "ms_per_step": fp["graph_ms"] / a.steps,
                           "serial_ms_per_step": fp["serial_ms"] / a.steps, "gpu_launches_per_step": fp["launches"],
                           "stated_rel_err": 1e-10, "roofline": fp["roofline"], "clocks": fp["clocks"],
                           "setup_s": round(fp["setup_s"], 1)},
            "split_speedup_vs_fp64": sv / fv}


def timed_steps(fn, steps, warmup, flush, stream):
    """Milliseconds of each of `steps` calls of fn (CUDA events on `stream`, L2 flushed before each)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    out = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream); fn(); e1.record(stream); e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def layer_and_periodic(args, V):
    """The two other paths to the velocity, measured beside the headline:
    * the layer potential u^H = D[mu] at every node of the coupled-step tree (uniform depth 7, p = 16,
      4.19M nodes, alpha = sqrt(Re/dt) = 316, split-precision tables) from the GMRES density of 256 x 16
      boundary nodes, with its error against the exterior-stokeslet exact solution inside the star;
    * the periodic particular solution by FFT (u and grad u) on a 4096^2 grid of the same box, with its
      error against a manufactured exact solution."""
    import numpy as np
    import torch
    from paper_1908_07392_gb300 import inputs as I
    steps, warmup = max(3, min(args.steps, 10)), 3
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    out = {}
    wl = I.step_workload(seed=5)
    b = V.BIE(wl.alpha, R=1.0, A=0.3, k=5, phase=wl.phi, n_panels=256)
    vp = layer = None
    try:
        src, f = I.moving_stokeslets(5)(0.0)
        S = torch.tensor(src, device="cuda"); Fs = torch.tensor(f, device="cuda")
        g = V.bie_stokeslets(wl.alpha, S, Fs, b.nodes[0:2].contiguous()).t().contiguous().reshape(-1)
        mu, it, rr = b.solve(g, None, 1e-13)
        t0 = time.perf_counter()
        vp = V.VolumePotential(I.KERNEL_MBIHARMONIC, wl.alpha, wl.p, wl.tree, precision=V.VP_PREC_SPLIT)
        layer = V.vp_layer_create(vp.tree, b.nodes[0:5].cpu().numpy())
        setup_s = time.perf_counter() - t0
        u = torch.empty(2, vp.N, dtype=torch.float64, device="cuda")
        ms = timed_steps(lambda: V.vp_layer_eval(layer, mu, u), steps, warmup, flush, stream)
        xy = vp.nodes()
        ue = V.bie_stokeslets(wl.alpha, S, Fs, xy).cpu().numpy()
        X, Y = xy[0].cpu().numpy(), xy[1].cpu().numpy()
        inside = np.hypot(X, Y) < 1.0 + 0.3 * np.cos(5 * np.arctan2(Y, X) + wl.phi) - 0.05
        uu = u.cpu().numpy()
        err = max(float(np.abs(uu[a][inside] - ue[a][inside]).max() / np.abs(ue[:, inside]).max()) for a in range(2))
        flush.zero_(); torch.cuda.synchronize()
        launches = V.vp_layer_steps(layer, mu, u)
        kinds = {0: "fp64 gemm", 1: "fp64 reduce", 2: "memset", 3: "slice", 4: "split gemm", 5: "df reduce",
                 6: "point operator"}
        top = sorted(launches, key=lambda x: -x["ms"])[:6]
        med = statistics.median(ms)
        out["layer_potential"] = {
            "workload": "coupled-step tree: uniform depth 7, p = 16, box [-1.5,1.5]^2, alpha 316, split tables; "
                        "4096 boundary nodes (256 panels x 16), GMRES density for exterior stokeslets",
            "value": vp.N / (med / 1e3), "unit": "nodes/s", "ms_per_eval": med, "steps": steps, "setup_s": setup_s,
            "gmres_iterations": it,
            "rel_err_vs_exact_inside": err, "inside_nodes": int(inside.sum()),
            "launches": len(launches), "in_order_ms": sum(x["ms"] for x in launches),
            "top_launches": [{"ms": round(x["ms"], 4), "kind": kinds.get(x["kind"], "?"),
                              "stage": V.STAGE_NAMES[x["stage"]], "gflop": round(x["flops"] / 1e9, 3),
                              "gbytes": round(x["bytes"] / 1e9, 3)} for x in top]}
    finally:
        if layer:
            V.vp_layer_free(layer)
        if vp is not None:
            vp.close()
        b.close()
    out.update(periodic_and_sdc(args, V, steps, warmup, flush, stream))
    return out


def periodic_and_sdc(args, V, steps, warmup, flush, stream):
    """The periodic FFT solution (u and grad u) on a 4096^2 grid against a manufactured exact solution,
    and SISDC steps of orders 2 and 4 on a 2048^2 Taylor-Green vortex against its exact decay."""
    import numpy as np
    import torch
    from paper_1908_07392_gb300 import inputs as I
    out = {}
    # periodic FFT solution: manufactured divergence-free velocity with a pressure gradient added
    n, L, alpha = 4096, 3.0, 316.0
    x = torch.arange(n, dtype=torch.float64, device="cuda") * (L / n)
    Yg, Xg = torch.meshgrid(x, x, indexing="ij")
    w = 2 * np.pi / L
    a_, b_ = 7 * w, 5 * w
    s1, c1, s2, c2 = torch.sin(a_ * Xg + 0.3), torch.cos(a_ * Xg + 0.3), torch.sin(b_ * Yg - 0.7), torch.cos(b_ * Yg - 0.7)
    u_ex = torch.stack([-b_ * s1 * s2, -a_ * c1 * c2])
    F = (alpha ** 2 + a_ * a_ + b_ * b_) * u_ex + torch.stack([-w * torch.sin(w * Xg) * torch.sin(3 * w * Yg),
                                                            3 * w * torch.cos(w * Xg) * torch.cos(3 * w * Yg)])
    F = F.contiguous()
    P = V.PeriodicStokes(alpha, n, L)
    try:
        u = torch.empty(2, n, n, dtype=torch.float64, device="cuda")
        gu = torch.empty(2, 2, n, n, dtype=torch.float64, device="cuda")
        ms = timed_steps(lambda: P(F, u, gu), steps, warmup, flush, stream)
        err = float((u - u_ex).abs().max() / u_ex.abs().max())
    finally:
        P.close()
    med = statistics.median(ms)
    flops = 4 * 10.0 * n * n * np.log2(n)  # one forward and three inverse complex 2-D transforms (nominal count)
    fp64_peak = N_SM * 2070.0e6 * FP64_FLOPS_PER_CLK_PER_SM / 1e12
    out["periodic_fft"] = {
        "workload": f"periodic modified Stokes velocity and gradient on a {n}^2 grid, box side 3, alpha 316",
        "value": n * n / (med / 1e3), "unit": "grid points/s", "ms_per_eval": med, "steps": steps,
        "rel_err_vs_manufactured": err,
        "roofline": {"bound": "alu", "kernel": "k_fft_rows: FP64 radix-4 Stockham rows in shared memory",
                     "achieved": flops / (med / 1e3) / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": flops / (med / 1e3) / 1e12 / fp64_peak,
                     "flops_note": "10 n^2 log2 n per complex 2-D transform, 4 transforms"}}
    # SISDC time stepping on the periodic box: Taylor-Green vortex, exact decay exp(-2 t / Re)
    n, re, dt = 2048, 1.0, 0.01
    u0, g0, l0 = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in I.taylor_green(n))
    sdc = {}
    for order in (2, 4):
        st = V.SISDC(re, dt, order, n, 2 * np.pi)
        try:
            st.set(u0, g0, l0)
            ms = timed_steps(lambda: st.step(1), steps, warmup, flush, stream)
            u, _ = st.get()
            T = (steps + warmup) * dt
            err = float((u - u0 * np.exp(-2 * T / re)).abs().max() / u0.abs().max())
        finally:
            st.close()
        med = statistics.median(ms)
        solves = 1 if order == 1 else order * order - order
        sdc[f"order_{order}"] = {"ms_per_step": med, "solves_per_step": solves, "ms_per_solve": med / solves,
                                 "steps_per_s": 1e3 / med, "t_end": T, "rel_err_vs_exact": err}
    out["sisdc"] = {"workload": f"Navier-Stokes on the periodic box [0, 2 pi)^2, {n}^2 grid, Re {re:g}, "
                                f"Delta t {dt:g}, Taylor-Green vortex", **sdc}
    return out


def run_periodic(args):
    """The periodic FFT solution and SISDC steps alone (the parts of the default line that need no
    tree), as one JSON line: a small command for profiling these kernels."""
    import torch
    import paper_1908_07392_gb300 as V
    from paper_1908_07392_gb300 import build as B
    B.build()
    steps, warmup = max(1, min(args.steps, 10)), max(1, args.warmup)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    with ClockSampler(torch.cuda.current_device()) as sampler:
        res = periodic_and_sdc(args, V, steps, warmup, flush, torch.cuda.current_stream())
    p = res["periodic_fft"]
    line = {"metric": "periodic modified Stokes solution grid points/s", "value": p["value"], "unit": p["unit"],
            "n_gpus": 1, "steps": steps, "warmup": warmup, "ms_per_step": p["ms_per_eval"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": p["workload"]}, "roofline": p["roofline"], "sisdc": res["sisdc"],
            "rel_err_vs_manufactured": p["rel_err_vs_manufactured"], "clocks": sampler.summary()}
    print(json.dumps(line), flush=True)


def run_batched(args):
    import torch
    import paper_1908_07392_gb300 as V
    from paper_1908_07392_gb300 import build as B
    from paper_1908_07392_gb300 import inputs as I
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    B.build()
    # whole trees are sharded over the ranks (a different seeded batch per rank), no collective
    ws = I.batched_workloads(seed=4 + rank)
    head_prec = V.VP_PREC_FP64 if args.precision == "fp64" else V.VP_PREC_SPLIT
    head = batched_form(args, V, ws, head_prec, local, world)
    plain = batched_form(args, V, ws, V.VP_PREC_FP64, local, world) if args.precision == "both" else None
    split = head_prec == V.VP_PREC_SPLIT
    line = {"metric": "volume-potential leaf-nodes/s at stated rel err, split/batched vs plain FP64",
            "value": head["nodes_all"] * args.steps / (head["graph_ms"] / 1000.0), "unit": "nodes/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["graph_ms"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64+bf16-slices" if split else "f64", "data": "synthetic",
            "config": {"workload": "batched: 64 trees, nodes log-uniform [1e4, 5e5], alpha log-uniform [10, 1000], "
                                   "p in {8, 12, 16}, modified-Helmholtz kernel, Gaussian-sum sources",
                       "trees": len(ws), "nodes": head["nodes"], "max_depth": int(max(w.tree.max_level for w in ws)),
                       "precision": "split" if split else "fp64", "stated_rel_err": 1e-9 if split else 1e-10,
                       "streams": args.streams, "setup_s": round(head["setup_s"], 1),
                       "engine": args.engine if split else "fp64", "tcgen05_launches": head["n_tc"],
                       "l2": "flushed before every timed step (512 MB write)"},
            "serial_ms_per_step": head["serial_ms"] / args.steps,
            "graph_speedup_vs_serial": head["serial_ms"] / head["graph_ms"],
            "roofline": head["roofline"], "cpu_baseline": None, "e2e": None,
            "gpu_launches": head["launches"] * args.steps, "clocks": head["clocks"]}
    if plain is not None:
        pv = plain["nodes_all"] * args.steps / (plain["graph_ms"] / 1000.0)
        line["plain_fp64"] = {"value": pv, "unit": "nodes/s", "ms_per_step": plain["graph_ms"] / args.steps,
                              "roofline": plain["roofline"]}
        line["split_speedup_vs_fp64"] = line["value"] / pv
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_steps(args):
    """Coupled steps in the star (Re = 100, dt = 1e-3, alpha = sqrt(Re/dt)): per step the volume
    potential of the vorticity source on a uniform depth-7, p = 16 tree (4.19M nodes), its boundary
    trace, and GMRES (tol 1e-11) for 256 panels x 16 nodes from a cold, previous, extrapolated or
    network initial guess; the network is trained on the plain solves of the first steps."""
    import numpy as np
    import torch
    import paper_1908_07392_gb300 as V
    from paper_1908_07392_gb300 import build as B
    from paper_1908_07392_gb300 import inputs as I
    from paper_1908_07392_gb300 import warmstart as WS
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    B.build()
    wl = I.step_workload(seed=5 + rank)
    prec = V.VP_PREC_FP64 if args.precision == "fp64" else V.VP_PREC_SPLIT
    log = (lambda m: print(m, file=sys.stderr, flush=True)) if rank == 0 else None
    t0 = time.perf_counter()
    sampler = ClockSampler(local)
    with sampler:
        r = WS.step_experiment(wl, n_panels=256, n_train=args.train_steps, n_test=args.test_steps, tol=1e-11,
                               precision=prec, epochs=args.epochs, log=log)
    wall = time.perf_counter() - t0
    b = V.BIE(wl.alpha, R=1.0, A=0.3, k=5, phase=wl.phi, n_panels=256)
    try:
        err, _ = WS.interior_error(b, wl.boundary, 0.0)
        # the Krylov operator apply (dense FP64 matrix-vector product, HBM-bound), timed with events
        x = torch.randn(2 * b.N, dtype=torch.float64, device="cuda")
        yv = torch.empty_like(x)
        for _ in range(3):
            b.apply(x, yv)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream = torch.cuda.current_stream()
        e0.record(stream)
        for _ in range(20):
            b.apply(x, yv)
        e1.record(stream)
        e1.synchronize()
        gemv_ms = e0.elapsed_time(e1) / 20
        gemv_bytes = (2 * b.N) ** 2 * 8 + 2 * (2 * b.N) * 8
    finally:
        b.close()
    hbm = measured_peaks().get("hbm_gbs", 6800.0)
    ev = r["held_out"]
    line = {"metric": "coupled step time with the learned GMRES warm start", "value": ev["network"]["mean_ms"],
            "unit": "ms/step", "n_gpus": world, "steps": args.test_steps, "warmup": 3 + args.train_steps,
            "ms_per_step": ev["network"]["mean_ms"], "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 solve, f32 network", "data": "synthetic",
            "config": {"workload": wl.name, "alpha": wl.alpha, "boundary_nodes": r["nodes"],
                       "volume_nodes": r["volume_nodes"], "volume_precision": "fp64" if prec == V.VP_PREC_FP64 else "split",
                       "train_steps": args.train_steps, "test_steps": args.test_steps, "epochs": args.epochs,
                       "gmres_tol": 1e-11, "net": "circular conv1d, fp32: network 10-64-64-64-2 k9 (3 densities), network4 12-64-64-64-2 k9, "
                              "network8 20-64-64-64-2 k9 (8 densities), temporal8 20-2 k1 (linear filter)"},
            "held_out": ev,
            "iterations_saved_vs_cold": ev["cold"]["mean_iters"] - ev["network"]["mean_iters"],
            "iterations_saved_vs_extrapolation": ev["extrapolation"]["mean_iters"] - ev["network"]["mean_iters"],
            "augmented_iterations_saved_vs_cold": ev["cold"]["mean_iters"] - ev["network_aug"]["mean_iters"],
            "augmented_iterations_saved_vs_extrapolation":
                ev["extrapolation"]["mean_iters"] - ev["network_aug"]["mean_iters"],
            "network4_iterations_saved_vs_cubic": (ev["cubic"]["mean_iters"] - ev["network4"]["mean_iters"])
            if "network4" in ev else None,
            "eight_density_iterations_saved_vs_quartic": {
                k: ev["quartic"]["mean_iters"] - ev[k]["mean_iters"] for k in ("network8", "temporal8") if k in ev},
            "plain_mean_iters": r["plain_mean_iters"], "volume_ms_mean": r["volume_ms_mean"],
            "train_seconds": r["train_seconds"], "train_loss": [r["first_train_loss"], r["final_train_loss"]],
            "interior_rel_err_exact_solution": err, "wall_seconds": wall,
            "gmres_operator_roofline": {"kernel": "k_gemv (dense FP64 Nystrom matrix)", "bound": "hbm",
                                        "achieved": gemv_bytes / (gemv_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                                        "frac": gemv_bytes / (gemv_ms / 1e3) / 1e9 / hbm, "ms": gemv_ms},
            "clocks": sampler.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)


def measure(args, V, w, prec, world, local, with_e2e):
    """Time args.steps evaluations of one form (FP64 or split) of the workload; per-step L2 flush."""
    import torch
    t0 = time.perf_counter()
    vp = V.VolumePotential(w.kernel, w.alpha, w.p, w.tree, order=args.order, precision=prec)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    try:
        N = vp.N
        f = torch.from_numpy(w.f).cuda()
        u = torch.empty(N, dtype=torch.float64, device="cuda")
        g = torch.empty(2, N, dtype=torch.float64, device="cuda")
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        launches, stage_flops = V.vp_tree_stats(vp.tree)
        stream = torch.cuda.current_stream()
        n_tc = choose_engine(V, args, vp.tree, f, u, g) if prec == V.VP_PREC_SPLIT else 0
        for _ in range(args.warmup):
            V.vp_eval(vp.tree, f, u, g)
        torch.cuda.synchronize()

        stage_ms, step_ms = [], []
        sampler = ClockSampler(local)
        barrier(world)
        with sampler:
            # the timed steps: vp_eval as a user calls it (near field overlapped with the far field)
            for _ in range(args.steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                V.vp_eval(vp.tree, f, u, g)
                e1.record(stream)
                e1.synchronize()
                step_ms.append(e0.elapsed_time(e1))
        barrier(world)
        # per-stage times (and the near kernel's duration for the roofline): the same evaluation with
        # every stage in order on one stream, bracketed by CUDA events on that stream
        for _ in range(min(args.steps, 5)):
            flush.zero_()
            torch.cuda.synchronize()
            stage_ms.append(V.vp_eval_timed(vp.tree, f, u, g))
        units, total_ms = job_totals(N * args.steps, sum(step_ms), world, "cuda")
        value = units / (total_ms / 1000.0)

        # e2e: host buffers, copies inside the timed region
        e2e = None
        if with_e2e:
            fh = torch.from_numpy(w.f).pin_memory()
            uh = torch.empty(N, dtype=torch.float64).pin_memory()
            gh = torch.empty(2, N, dtype=torch.float64).pin_memory()
            V.vp_eval_host(vp.tree, fh, uh, gh)
            torch.cuda.synchronize()
            barrier(world)
            t0 = time.perf_counter()
            for _ in range(args.steps):
                V.vp_eval_host(vp.tree, fh, uh, gh)
            torch.cuda.synchronize()
            e2e = {"value": world * N * args.steps / (time.perf_counter() - t0), "unit": "nodes/s",
                   "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 24 * N}

        stage_bytes = V.vp_tree_bytes(vp.tree)
        # every launch timed in order (one evaluation, L2 flushed before it)
        flush.zero_()
        torch.cuda.synchronize()
        launch_list = V.vp_eval_steps(vp.tree, f, u, g)
        split = prec == V.VP_PREC_SPLIT
        hbm = measured_peaks().get("hbm_gbs", 6800.0)
        fp64_peak = N_SM * 2070.0e6 * FP64_FLOPS_PER_CLK_PER_SM / 1e12
        tc_peak = measured_peaks().get("bf16_tflops", 1900.0)
        near_ms = statistics.mean(m[4] for m in stage_ms)
        near_flops = stage_flops[4]
        near_gbs = stage_bytes[4] / (near_ms / 1000.0) / 1e9
        if not split:
            achieved = near_flops / (near_ms / 1000.0) / 1e12
            peak = fp64_peak
            roof = {"kernel": "k_gemm_gather_f64<1> (near-field tables)", "bound": "alu",
                    "peak_source": "FP64 pipe: 152 SMs x 2070 MHz x 4 flop/clk (derived; 1.20 TFLOP/s measured)"}
            traffic = TRAFFIC_FP64_NEAR if (args.max_depth == 10 and args.alpha == 300.0) else None
            if traffic is not None:
                roof["traffic_source"] = TRAFFIC_FP64_NEAR_SOURCE
        else:
            # tensor work: S(S+1)/2 slice products of the same shape as the FP64 contraction
            achieved = near_flops * SLICE_PRODUCTS / (near_ms / 1000.0) / 1e12
            peak = tc_peak
            roof = {"kernel": "split-precision near-field GEMM (6 bf16 slices, fp32 accumulation; engine per launch)",
                    "bound": "tensor", "peak_source": "measured dense bf16 burst (MEASURED_PEAKS.json), of measured",
                    "fp64_equivalent_tflops": near_flops / (near_ms / 1000.0) / 1e12}
            traffic = None
            if args.engine in ("auto", "tcgen05") and launch_list_engine(launch_list, 0) == 1:
                traffic = near_flops / 1e9 * TRAFFIC_SPLIT_NEAR_PER_GFLOP
                roof["traffic_source"] = TRAFFIC_SPLIT_NEAR_SOURCE
        roof.update(algorithmic_bytes=stage_bytes[4], achieved_gbs=near_gbs, hbm_frac_of_measured=near_gbs / hbm)

        def rate(flops, bytes_, ms):
            sec = max(ms, 1e-6) / 1000.0
            tf = flops * (SLICE_PRODUCTS if split else 1) / sec / 1e12
            gbs = bytes_ / sec / 1e9
            return {"ms": round(ms, 4), "tflops": round(tf, 3), "frac": round(tf / (tc_peak if split else fp64_peak), 4),
                    "gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4)}

        stage_roof = {}
        for k, name in enumerate(V.STAGE_NAMES):
            ms_k = statistics.mean(m[k] for m in stage_ms)
            stage_roof[name] = dict(rate(stage_flops[k], stage_bytes[k], ms_k), gflop=round(stage_flops[k] / 1e9, 2),
                                    gbytes=round(stage_bytes[k] / 1e9, 3))
        kinds = {0: "fp64 gemm", 1: "fp64 reduce", 2: "memset", 3: "slice", 4: "split gemm", 5: "df reduce"}
        tables = {-1: "-", 0: "near", 1: "s2m", 2: "l2t", 3: "m2m", 4: "l2l", 5: "m2l", 6: "m2t", 7: "s2l",
                  8: "m2m_lo", 9: "m2m_hi"}
        top = sorted(range(len(launch_list)), key=lambda i: -launch_list[i]["ms"])[:10]
        top_launches = [dict(rate(launch_list[i]["flops"], launch_list[i]["bytes"], launch_list[i]["ms"]),
                             index=i, kind=kinds.get(launch_list[i]["kind"], "?"),
                             stage=V.STAGE_NAMES[launch_list[i]["stage"]],
                             table=tables.get(launch_list[i]["table"], "?"),
                             engine=ENGINE_NAMES.get(launch_list[i]["engine"], "?"))
                        for i in top]
        return {"value": value, "total_ms": total_ms, "N": N, "setup_s": setup_s, "n_tc": n_tc,
                "u": u.cpu().numpy(), "g": g.cpu().numpy(),
                "launches": int(launches), "e2e": e2e, "clocks": sampler.summary(),
                "stage_ms": {name: round(statistics.mean(m[k] for m in stage_ms), 4)
                             for k, name in enumerate(V.STAGE_NAMES)},
                "stage_roofline": stage_roof,
                "launch_list": {"launches": len(launch_list), "in_order_ms": round(sum(x["ms"] for x in launch_list), 4),
                                "top": top_launches},
                "roofline": dict(roof, achieved=achieved, peak=peak, unit="TFLOP/s", frac=achieved / peak,
                                 traffic=traffic)}
    finally:
        vp.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "steps":
        run_steps(args)
        return
    if args.workload == "periodic":
        run_periodic(args)
        return
    import torch
    import paper_1908_07392_gb300 as V
    from paper_1908_07392_gb300 import build as B

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    B.build()
    w = workload(args.alpha, args.max_depth)
    # headline form: split precision unless only FP64 is asked for; "both" adds the FP64 form beside it
    # the CPU baseline (the oracle on a bounded sample of nodes) runs first; its values also give the
    # sampled error of every GPU form measured below
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, n, cores, dt = cpu_sample(w, args.cpu_seconds)
        cpu = {"value": rate, "unit": "nodes/s", "cores": cores, "kind": "oracle",
               "sample": f"{n} random target nodes of the same workload, {dt:.1f} s on {cores} threads"}
    head_prec = V.VP_PREC_FP64 if args.precision == "fp64" else V.VP_PREC_SPLIT
    head = measure(args, V, w, head_prec, world, local, not args.no_e2e)
    plain = measure(args, V, w, V.VP_PREC_FP64, world, local, False) if args.precision == "both" else None
    # the batched workload (64 trees in one CUDA graph), split and FP64, in the same run
    batched = None if (args.no_batched or args.precision != "both") else batched_pair(args, V, local, world)
    # the layer potential and the periodic FFT solution
    extras = None if (args.no_batched or args.precision != "both" or world > 1) else layer_and_periodic(args, V)
    errs = {}
    if cpu is not None:
        idx, vals = cpu_sample.last
        errs["split" if head_prec == V.VP_PREC_SPLIT else "fp64"] = sampled_errors(idx, vals, head["u"], head["g"])
        if plain is not None:
            errs["fp64"] = sampled_errors(idx, vals, plain["u"], plain["g"])

    if rank == 0:
        split = head_prec == V.VP_PREC_SPLIT
        line = {"metric": "volume-potential leaf-nodes/s at stated rel err, split/batched vs plain FP64",
                "value": head["value"], "unit": "nodes/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": head["total_ms"] / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64+bf16-slices" if split else "f64",
                "data": "synthetic",
                "config": dict(workload_desc(w), precision="split" if split else "fp64", order=args.order,
                               stated_rel_err=1e-9 if split else 1e-10,
                               engine=args.engine if split else "fp64", tcgen05_launches=head["n_tc"],
                               l2="flushed before every timed step (512 MB write)",
                               parallelism="replicas" if world > 1 else "single GPU",
                               setup_s=round(head["setup_s"], 2)),
                "stage_ms": head["stage_ms"],
                "stage_timing": "per-stage CUDA events, stages in order on one stream; the timed steps run "
                                "vp_eval, which overlaps the near field with the far-field chain",
                "stage_roofline": head["stage_roofline"],
                "stage_roofline_note": "per stage: algorithmic flops (split: x21 bf16 slice products) and bytes "
                                       "(operators and distinct source vectors once, outputs once) over the "
                                       "in-order stage time; frac of the measured bf16 burst (split) or the "
                                       "derived FP64 pipe (fp64); hbm_frac of the measured copy bandwidth",
                "launch_list": head["launch_list"],
                "roofline": head["roofline"],
                "cpu_baseline": cpu,
                "rel_err_vs_oracle_sampled": errs or None,
                "e2e": head["e2e"],
                "gpu_launches": head["launches"] * args.steps,
                "clocks": head["clocks"]}
        if plain is not None:
            line["plain_fp64"] = {"value": plain["value"], "unit": "nodes/s",
                                  "ms_per_step": plain["total_ms"] / args.steps, "stage_ms": plain["stage_ms"],
                                  "stage_roofline": plain["stage_roofline"], "launch_list": plain["launch_list"],
                                  "roofline": plain["roofline"], "clocks": plain["clocks"],
                                  "gpu_launches": plain["launches"] * args.steps}
            line["split_speedup_vs_fp64"] = head["value"] / plain["value"]
        if batched is not None:
            line["batched"] = batched
        if extras is not None:
            line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
