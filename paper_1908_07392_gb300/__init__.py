"""GB300 volume-potential library: thin Python binding of libvp.so.

The functions below carry the names of the C ABI in ``include/vp.h`` and only
marshal arguments (PyTorch supplies device memory and streams). Every step of
the computation runs in the library's CUDA kernels; there is no Python or CPU
fallback: if the compiled library is missing, importing the binding raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import inputs  # noqa: F401  (seeded input generators, no method arithmetic)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libvp.so")

VP_KERNEL_MHELMHOLTZ = 0
VP_KERNEL_MBIHARMONIC = 1
VP_PREC_FP64 = 0
VP_PREC_SPLIT = 1

_lib = None


class VPError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        msg = f"{vp_strerror(code)} ({code})"
        if code == -5:
            msg += f" [{load_library().vp_last_cuda_error().decode()}]"
        super().__init__(f"{what}: {msg}" if what else msg)


def load_library():
    """Load libvp.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libvp.so not built at {LIB_PATH}; run paper_1908_07392_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    c_int, c_double, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    i32p = ctypes.POINTER(ctypes.c_int32)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.vp_tables_build.argtypes = [c_int, c_double, c_int, c_int, c_double, c_int, c_int, c_void_p,
                                    ctypes.POINTER(c_void_p)]
    lib.vp_tree_upload.argtypes = [c_void_p, c_double, c_double, c_int, i32p, i32p, i32p, c_void_p,
                                   ctypes.POINTER(c_void_p)]
    lib.vp_tree_size.argtypes = [c_void_p, i64p, i64p]
    lib.vp_tree_nodes.argtypes = [c_void_p, c_void_p, c_void_p]
    lib.vp_tree_interp.argtypes = [c_void_p, c_int, c_void_p, c_int, c_void_p, c_void_p, c_void_p]
    lib.vp_special.argtypes = [c_int, c_int, c_int, c_void_p, c_void_p, c_void_p]
    lib.vp_eval.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.vp_eval_host.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.vp_tree_free.argtypes = [c_void_p]
    lib.vp_tree_free.restype = None
    lib.vp_tables_free.argtypes = [c_void_p]
    lib.vp_tables_free.restype = None
    lib.vp_strerror.argtypes = [c_int]
    lib.vp_strerror.restype = ctypes.c_char_p
    vpp = ctypes.POINTER(c_void_p)
    lib.bie_create.argtypes = [c_double, c_double, c_double, c_int, c_double, c_int, c_int, c_void_p, vpp]
    lib.bie_free.argtypes = [c_void_p]
    lib.bie_free.restype = None
    lib.bie_size.argtypes = [c_void_p, ctypes.POINTER(c_int), ctypes.POINTER(c_double)]
    lib.bie_nodes.argtypes = [c_void_p, c_void_p, c_void_p]
    lib.bie_apply.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
    lib.bie_solve.argtypes = [c_void_p, c_void_p, c_void_p, c_double, c_int, ctypes.POINTER(c_int),
                              ctypes.POINTER(c_double), c_void_p]
    lib.bie_solve_aug.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_double, c_int, ctypes.POINTER(c_int),
                                  ctypes.POINTER(c_double), c_void_p]
    lib.bie_eval.argtypes = [c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p]
    lib.bie_stokeslets.argtypes = [c_double, c_int, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p]
    lib.bie_kernel_scalars.argtypes = [c_int, c_void_p, c_void_p, c_void_p]
    lib.ws_create.argtypes = [c_int, c_int, c_int, c_int, c_int, c_int, c_int, ctypes.c_uint64, c_void_p, vpp]
    lib.ws_free.argtypes = [c_void_p]
    lib.ws_free.restype = None
    lib.ws_num_params.argtypes = [c_void_p, i64p]
    lib.ws_params.argtypes = [c_void_p, c_void_p, c_int, c_void_p]
    lib.ws_forward.argtypes = [c_void_p, c_void_p, c_int, c_void_p, c_void_p]
    lib.ws_grad.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_void_p, ctypes.POINTER(ctypes.c_float), c_void_p]
    lib.ws_train_step.argtypes = [c_void_p, c_void_p, c_void_p, c_int, ctypes.c_float,
                                  ctypes.POINTER(ctypes.c_float), c_void_p]
    lib.vp_tree_set_engine.argtypes = [c_void_p, c_int]
    lib.vp_autotune.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, ctypes.c_char_p, c_void_p,
                                ctypes.POINTER(c_int)]
    lib.vp_device_status.argtypes = []
    lib.vp_selftest_timeout.argtypes = [c_void_p]
    lib.vp_last_cuda_error.argtypes = []
    lib.vp_last_cuda_error.restype = ctypes.c_char_p
    lib.vp_plan_pairs.argtypes = [c_int, i32p, i32p, i32p, i64p, i32p, i32p, i32p]
    lib.vp_eval_timed.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, ctypes.POINTER(ctypes.c_float)]
    lib.vp_tree_stats.argtypes = [c_void_p, i64p, ctypes.POINTER(c_double)]
    lib.vp_tree_bytes.argtypes = [c_void_p, ctypes.POINTER(c_double)]
    lib.vp_layer_create.argtypes = [c_void_p, c_int, c_void_p, c_void_p, ctypes.POINTER(c_void_p)]
    lib.vp_layer_eval.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
    lib.vp_layer_steps.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int, ctypes.POINTER(c_int),
                                   ctypes.POINTER(ctypes.c_float), ctypes.POINTER(c_int), ctypes.POINTER(c_double),
                                   ctypes.POINTER(c_double)]
    lib.vp_layer_free.argtypes = [c_void_p]
    lib.vp_layer_free.restype = None
    lib.vp_layer_near_star.argtypes = [c_void_p, c_double, c_double, c_int, c_double, c_int, c_double, c_void_p, i64p]
    lib.vp_periodic_create.argtypes = [c_double, c_int, c_double, c_void_p, ctypes.POINTER(c_void_p)]
    lib.vp_periodic_eval.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.vp_periodic_free.argtypes = [c_void_p]
    lib.vp_periodic_free.restype = None
    lib.vp_sdc_create.argtypes = [c_double, c_double, c_int, c_int, c_double, c_void_p, ctypes.POINTER(c_void_p)]
    lib.vp_sdc_set.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.vp_sdc_step.argtypes = [c_void_p, c_int, c_void_p]
    lib.vp_sdc_get.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
    lib.vp_sdc_free.argtypes = [c_void_p]
    lib.vp_sdc_free.restype = None
    lib.vp_eval_steps.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int, ctypes.POINTER(c_int),
                                  ctypes.POINTER(ctypes.c_float), ctypes.POINTER(c_int), ctypes.POINTER(c_double),
                                  ctypes.POINTER(c_double)]
    pp = ctypes.POINTER(c_void_p)
    lib.vp_batch_create.argtypes = [c_int, pp, pp, pp, pp, c_int, c_void_p, ctypes.POINTER(c_void_p)]
    lib.vp_batch_run.argtypes = [c_void_p, c_void_p]
    lib.vp_batch_stats.argtypes = [c_void_p, i64p, i64p]
    lib.vp_batch_free.argtypes = [c_void_p]
    lib.vp_batch_free.restype = None
    lib.vp_eval_batched.argtypes = [c_int, pp, pp, pp, pp, c_int, c_void_p]
    _lib = lib
    return lib


def exported_symbols():
    """Names declared in include/vp.h (the ABI surface)."""
    return ["vp_tables_build", "vp_tree_upload", "vp_tree_size", "vp_tree_nodes", "vp_tree_interp", "vp_special", "vp_eval", "vp_eval_host",
            "vp_eval_timed", "vp_tree_stats", "vp_tree_bytes", "vp_eval_steps", "vp_layer_create", "vp_layer_eval",
            "vp_layer_steps", "vp_layer_free", "vp_layer_near_star", "vp_periodic_create", "vp_periodic_eval", "vp_periodic_free", "vp_sdc_create", "vp_sdc_set", "vp_sdc_step", "vp_sdc_get", "vp_sdc_free", "vp_tree_free", "vp_tables_free", "vp_strerror", "vp_plan_pairs",
            "vp_eval_static", "vp_batch_create", "vp_batch_run", "vp_batch_stats", "vp_batch_free",
            "vp_eval_batched", "vp_last_cuda_error", "vp_tree_set_engine", "vp_autotune", "vp_device_status", "vp_selftest_timeout",
            "bie_create", "bie_free", "bie_size", "bie_nodes", "bie_apply", "bie_solve", "bie_solve_aug", "bie_eval",
            "bie_stokeslets", "bie_kernel_scalars", "ws_create", "ws_free", "ws_num_params", "ws_params",
            "ws_forward", "ws_grad", "ws_train_step"]


ENGINE_MMA_SYNC = 0
ENGINE_TCGEN05 = 1
ENGINE_MMA_SMALL = 2
ENGINE_TCGEN05_N64 = 3
ENGINE_TCGEN05_T = 4


def vp_tree_set_engine(tree: int, engine: int):
    _check(load_library().vp_tree_set_engine(ctypes.c_void_p(tree), int(engine)), "vp_tree_set_engine")


def vp_selftest_timeout(stream=None) -> int:
    """Status code of the bounded-wait self test (VP_ERR_TIMEOUT = -7 when the give-up path works)."""
    return int(load_library().vp_selftest_timeout(_stream_ptr(stream)))


def vp_device_status():
    _check(load_library().vp_device_status(), "vp_device_status")


def vp_autotune(tree: int, f, u, gradu, cache_path=None, stream=None) -> int:
    """Pick the faster split-precision engine per launch; returns how many launches use tcgen05."""
    n = ctypes.c_int()
    _check(load_library().vp_autotune(ctypes.c_void_p(tree), ctypes.c_void_p(f.data_ptr()),
                                      ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(gradu.data_ptr()),
                                      cache_path.encode() if cache_path else None, _stream_ptr(stream),
                                      ctypes.byref(n)), "vp_autotune")
    return n.value


VP_NSTAGES = 6
STAGE_NAMES = ["upward", "m2l", "downward", "targets", "near", "output"]


def _check(rc, what):
    if rc != 0:
        raise VPError(rc, what)


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream))


def vp_strerror(code: int) -> str:
    return load_library().vp_strerror(int(code)).decode()


def vp_tables_build(kernel: int, alpha: float, p: int, levels: int, root_side: float, order: int = 40,
                    precision: int = VP_PREC_FP64, stream=None) -> int:
    out = ctypes.c_void_p()
    rc = load_library().vp_tables_build(int(kernel), float(alpha), int(p), int(levels), float(root_side),
                                        int(order), int(precision), _stream_ptr(stream), ctypes.byref(out))
    _check(rc, "vp_tables_build")
    return out.value


def vp_tree_upload(tables: int, cx: float, cy: float, level, ix, iy, stream=None) -> int:
    lv, plv = _i32(level)
    xx, pix = _i32(ix)
    yy, piy = _i32(iy)
    out = ctypes.c_void_p()
    rc = load_library().vp_tree_upload(ctypes.c_void_p(tables), float(cx), float(cy), int(lv.size), plv, pix, piy,
                                       _stream_ptr(stream), ctypes.byref(out))
    _check(rc, "vp_tree_upload")
    return out.value


def vp_tree_size(tree: int):
    a = ctypes.c_int64(); b = ctypes.c_int64()
    _check(load_library().vp_tree_size(ctypes.c_void_p(tree), ctypes.byref(a), ctypes.byref(b)), "vp_tree_size")
    return a.value, b.value


def vp_tree_nodes(tree: int, xy, stream=None):
    _check(load_library().vp_tree_nodes(ctypes.c_void_p(tree), ctypes.c_void_p(xy.data_ptr()), _stream_ptr(stream)),
           "vp_tree_nodes")


def vp_special(which: int, z, nmax: int = 1, stream=None):
    """Device special functions at z (device float64 [M]); see include/vp.h. Returns [rows][M]."""
    import torch
    rows = 2 if which == 0 else nmax + 1
    out = torch.empty(rows, z.numel(), dtype=torch.float64, device=z.device)
    _check(load_library().vp_special(int(which), int(nmax), int(z.numel()), ctypes.c_void_p(z.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)), "vp_special")
    return out


def vp_tree_interp(tree: int, fields, xy, out, stream=None):
    """fields: device float64 [F, N]; xy: [2, M]; out: [F, M]."""
    _check(load_library().vp_tree_interp(ctypes.c_void_p(tree), int(fields.shape[0]), ctypes.c_void_p(fields.data_ptr()),
                                         int(xy.shape[1]), ctypes.c_void_p(xy.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)), "vp_tree_interp")


def vp_eval(tree: int, f, u, gradu, stream=None):
    """f, u: device float64 [N]; gradu: device float64 [2, N] (torch tensors, contiguous)."""
    for t in (f, u, gradu):
        if not (t.is_cuda and t.is_contiguous()) or str(t.dtype) != "torch.float64":
            raise ValueError("vp_eval expects contiguous float64 CUDA tensors")
    _check(load_library().vp_eval(ctypes.c_void_p(tree), ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                  ctypes.c_void_p(gradu.data_ptr()), _stream_ptr(stream)), "vp_eval")


def vp_eval_timed(tree: int, f, u, gradu, stream=None):
    """vp_eval with CUDA events between stages; returns milliseconds per stage (list of VP_NSTAGES)."""
    ms = (ctypes.c_float * VP_NSTAGES)()
    _check(load_library().vp_eval_timed(ctypes.c_void_p(tree), ctypes.c_void_p(f.data_ptr()),
                                        ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(gradu.data_ptr()),
                                        _stream_ptr(stream), ms), "vp_eval_timed")
    return list(ms)


def vp_tree_stats(tree: int):
    """(launches per evaluation, algorithmic flops per stage)."""
    n = ctypes.c_int64()
    fl = (ctypes.c_double * VP_NSTAGES)()
    _check(load_library().vp_tree_stats(ctypes.c_void_p(tree), ctypes.byref(n), fl), "vp_tree_stats")
    return n.value, list(fl)


def vp_tree_bytes(tree: int):
    """Algorithmic device-memory bytes per stage (list of VP_NSTAGES)."""
    b = (ctypes.c_double * VP_NSTAGES)()
    _check(load_library().vp_tree_bytes(ctypes.c_void_p(tree), b), "vp_tree_bytes")
    return list(b)


def vp_eval_steps(tree: int, f, u, gradu, stream=None):
    """Every launch of one evaluation timed in order: list of dicts (ms, kind, stage, table, engine, flops,
    bytes), one per launch."""
    lib = load_library()
    n = ctypes.c_int()
    _check(lib.vp_eval_steps(ctypes.c_void_p(tree), None, None, None, _stream_ptr(stream), 0, ctypes.byref(n),
                             None, None, None, None), "vp_eval_steps")
    k = n.value
    ms = (ctypes.c_float * k)(); info = (ctypes.c_int * (4 * k))()
    fl = (ctypes.c_double * k)(); by = (ctypes.c_double * k)()
    _check(lib.vp_eval_steps(ctypes.c_void_p(tree), ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                             ctypes.c_void_p(gradu.data_ptr()), _stream_ptr(stream), k, ctypes.byref(n), ms, info,
                             fl, by), "vp_eval_steps")
    return [{"ms": ms[i], "kind": info[4 * i], "stage": info[4 * i + 1], "table": info[4 * i + 2],
             "engine": info[4 * i + 3], "flops": fl[i], "bytes": by[i]} for i in range(k)]


def vp_layer_create(tree: int, src, stream=None) -> int:
    """Layer potential operators of boundary points on a tree. src: host array [5][n] (x, y, n_x, n_y, w)."""
    a = np.ascontiguousarray(src, dtype=np.float64)
    if a.ndim != 2 or a.shape[0] != 5:
        raise ValueError("src must be [5][n]: x, y, n_x, n_y, w")
    out = ctypes.c_void_p()
    _check(load_library().vp_layer_create(ctypes.c_void_p(tree), int(a.shape[1]), a.ctypes.data_as(ctypes.c_void_p),
                                          _stream_ptr(stream), ctypes.byref(out)), "vp_layer_create")
    return out.value


def vp_layer_eval(layer: int, mu, u, stream=None):
    """mu: device float64 [n][2] (or [2n], (mu_x, mu_y) per point); u: device float64 [2, N]."""
    _check(load_library().vp_layer_eval(ctypes.c_void_p(layer), ctypes.c_void_p(mu.data_ptr()),
                                        ctypes.c_void_p(u.data_ptr()), _stream_ptr(stream)), "vp_layer_eval")


def vp_layer_steps(layer: int, mu, u, stream=None):
    """Every launch of one layer evaluation timed in order (as vp_eval_steps)."""
    lib = load_library()
    n = ctypes.c_int()
    _check(lib.vp_layer_steps(ctypes.c_void_p(layer), None, None, _stream_ptr(stream), 0, ctypes.byref(n),
                              None, None, None, None), "vp_layer_steps")
    k = n.value
    ms = (ctypes.c_float * k)(); info = (ctypes.c_int * (4 * k))()
    fl = (ctypes.c_double * k)(); by = (ctypes.c_double * k)()
    _check(lib.vp_layer_steps(ctypes.c_void_p(layer), ctypes.c_void_p(mu.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                              _stream_ptr(stream), k, ctypes.byref(n), ms, info, fl, by), "vp_layer_steps")
    return [{"ms": ms[i], "kind": info[4 * i], "stage": info[4 * i + 1], "table": info[4 * i + 2],
             "engine": info[4 * i + 3], "flops": fl[i], "bytes": by[i]} for i in range(k)]


class PeriodicStokes:
    """Periodic particular solution by FFT on an n x n grid of a box of side L (include/vp.h)."""

    def __init__(self, alpha, n, side, stream=None):
        out = ctypes.c_void_p()
        _check(load_library().vp_periodic_create(float(alpha), int(n), float(side), _stream_ptr(stream),
                                                 ctypes.byref(out)), "vp_periodic_create")
        self.handle, self.n, self.alpha, self.side = out.value, n, alpha, side

    def __call__(self, F, u=None, gradu=None, stream=None):
        """F device float64 [2, n, n] -> u [2, n, n], gradu [2, 2, n, n]."""
        import torch
        n = self.n
        u = torch.empty(2, n, n, dtype=torch.float64, device=F.device) if u is None else u
        gradu = torch.empty(2, 2, n, n, dtype=torch.float64, device=F.device) if gradu is None else gradu
        _check(load_library().vp_periodic_eval(ctypes.c_void_p(self.handle), ctypes.c_void_p(F.data_ptr()),
                                               ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(gradu.data_ptr()),
                                               _stream_ptr(stream)), "vp_periodic_eval")
        return u, gradu

    def close(self):
        if getattr(self, "handle", None):
            load_library().vp_periodic_free(ctypes.c_void_p(self.handle))
            self.handle = None


class SISDC:
    """Navier-Stokes time stepping on a periodic n x n grid of a box of side L by semi-implicit spectral
    deferred correction of order 1..4, every substep a periodic modified Stokes solve (include/vp.h)."""

    def __init__(self, re, dt, order, n, side, stream=None):
        out = ctypes.c_void_p()
        _check(load_library().vp_sdc_create(float(re), float(dt), int(order), int(n), float(side),
                                            _stream_ptr(stream), ctypes.byref(out)), "vp_sdc_create")
        self.handle, self.n, self.re, self.dt, self.order, self.side = out.value, n, re, dt, order, side

    def set(self, u0, gradu0, lap0, stream=None):
        """u0 [2, n, n], gradu0 [2, 2, n, n], lap0 [2, n, n]: device float64, contiguous."""
        _check(load_library().vp_sdc_set(ctypes.c_void_p(self.handle), ctypes.c_void_p(u0.data_ptr()),
                                         ctypes.c_void_p(gradu0.data_ptr()), ctypes.c_void_p(lap0.data_ptr()),
                                         _stream_ptr(stream)), "vp_sdc_set")

    def step(self, n_steps=1, stream=None):
        _check(load_library().vp_sdc_step(ctypes.c_void_p(self.handle), int(n_steps), _stream_ptr(stream)),
               "vp_sdc_step")

    def get(self, u=None, gradu=None, stream=None):
        import torch
        n = self.n
        u = torch.empty(2, n, n, dtype=torch.float64, device="cuda") if u is None else u
        gradu = torch.empty(2, 2, n, n, dtype=torch.float64, device="cuda") if gradu is None else gradu
        _check(load_library().vp_sdc_get(ctypes.c_void_p(self.handle), ctypes.c_void_p(u.data_ptr()),
                                         ctypes.c_void_p(gradu.data_ptr()), _stream_ptr(stream)), "vp_sdc_get")
        return u, gradu

    def close(self):
        if getattr(self, "handle", None):
            load_library().vp_sdc_free(ctypes.c_void_p(self.handle))
            self.handle = None


def vp_layer_near_star(layer: int, R, A, k, phase, n_panels, dist=1.2, stream=None) -> int:
    """Near-boundary corrections for a layer whose points are the star's panel nodes; returns the pair count."""
    n = ctypes.c_int64()
    _check(load_library().vp_layer_near_star(ctypes.c_void_p(layer), float(R), float(A), int(k), float(phase),
                                             int(n_panels), float(dist), _stream_ptr(stream), ctypes.byref(n)),
           "vp_layer_near_star")
    return n.value


def vp_layer_free(layer: int):
    if layer:
        load_library().vp_layer_free(ctypes.c_void_p(layer))


def vp_eval_host(tree: int, f, u, gradu, stream=None):
    """f, u: host float64 [N]; gradu: host float64 [2, N] (numpy arrays or CPU tensors, contiguous)."""
    def ptr(a):
        return ctypes.c_void_p(a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data)
    _check(load_library().vp_eval_host(ctypes.c_void_p(tree), ptr(f), ptr(u), ptr(gradu), _stream_ptr(stream)),
           "vp_eval_host")


def vp_tree_free(tree: int):
    if tree:
        load_library().vp_tree_free(ctypes.c_void_p(tree))


def vp_tables_free(tables: int):
    if tables:
        load_library().vp_tables_free(ctypes.c_void_p(tables))


def vp_plan_pairs(level, ix, iy):
    """Host-only: (target leaf, source leaf, mechanism) triples covered by the interaction lists
    (mechanism 0 = near table, 1 = multipole-to-local, 2 = multipole-to-target, 3 = source-to-local)."""
    lib = load_library()
    lv, plv = _i32(level)
    xx, pix = _i32(ix)
    yy, piy = _i32(iy)
    n = ctypes.c_int64()
    _check(lib.vp_plan_pairs(int(lv.size), plv, pix, piy, ctypes.byref(n), None, None, None), "vp_plan_pairs")
    t = np.zeros(n.value, np.int32); s = np.zeros(n.value, np.int32); m = np.zeros(n.value, np.int32)
    _check(lib.vp_plan_pairs(int(lv.size), plv, pix, piy, ctypes.byref(n), _i32(t)[1], _i32(s)[1], _i32(m)[1]),
           "vp_plan_pairs")
    return t, s, m


def _ptr_array(values):
    arr = (ctypes.c_void_p * len(values))()
    for k, v in enumerate(values):
        arr[k] = v
    return arr


def vp_batch_create(trees, f, u, gradu, n_streams=16, stream=None) -> int:
    """One CUDA graph evaluating every tree (handles) from f[t] into u[t], gradu[t] (torch CUDA tensors)."""
    n = len(trees)
    out = ctypes.c_void_p()
    rc = load_library().vp_batch_create(n, _ptr_array(trees), _ptr_array([x.data_ptr() for x in f]),
                                        _ptr_array([x.data_ptr() for x in u]),
                                        _ptr_array([x.data_ptr() for x in gradu]), int(n_streams),
                                        _stream_ptr(stream), ctypes.byref(out))
    _check(rc, "vp_batch_create")
    return out.value


def vp_batch_run(batch: int, stream=None):
    _check(load_library().vp_batch_run(ctypes.c_void_p(batch), _stream_ptr(stream)), "vp_batch_run")


def vp_batch_stats(batch: int):
    a = ctypes.c_int64(); b = ctypes.c_int64()
    _check(load_library().vp_batch_stats(ctypes.c_void_p(batch), ctypes.byref(a), ctypes.byref(b)), "vp_batch_stats")
    return a.value, b.value


def vp_batch_free(batch: int):
    if batch:
        load_library().vp_batch_free(ctypes.c_void_p(batch))


def vp_eval_batched(trees, f, u, gradu, use_graph=1, stream=None):
    n = len(trees)
    rc = load_library().vp_eval_batched(n, _ptr_array(trees), _ptr_array([x.data_ptr() for x in f]),
                                        _ptr_array([x.data_ptr() for x in u]),
                                        _ptr_array([x.data_ptr() for x in gradu]), int(use_graph),
                                        _stream_ptr(stream))
    _check(rc, "vp_eval_batched")


class VolumePotential:
    """Tables + tree for one workload; evaluates u and grad u at every leaf node on the GPU."""

    def __init__(self, kernel, alpha, p, tree, order=40, precision=VP_PREC_FP64, levels=None, stream=None):
        import torch
        self.p = p
        self.levels = int(tree.max_level if levels is None else levels)
        self.tables = vp_tables_build(kernel, alpha, p, self.levels, tree.side, order, precision, stream)
        try:
            self.tree = vp_tree_upload(self.tables, tree.cx, tree.cy, tree.level, tree.ix, tree.iy, stream)
        except Exception:
            vp_tables_free(self.tables)
            raise
        self.n_leaves, self.N = vp_tree_size(self.tree)
        self.device = torch.device("cuda", torch.cuda.current_device())

    def nodes(self):
        import torch
        xy = torch.empty(2, self.N, dtype=torch.float64, device=self.device)
        vp_tree_nodes(self.tree, xy)
        return xy

    def interp(self, fields, xy):
        """Leaf interpolants of fields [F, N] at points xy [2, M] -> [F, M]."""
        import torch
        fields = fields.reshape(-1, self.N).contiguous()
        xy = xy.contiguous()
        out = torch.empty(fields.shape[0], xy.shape[1], dtype=torch.float64, device=fields.device)
        vp_tree_interp(self.tree, fields, xy, out)
        return out

    def __call__(self, f, u=None, gradu=None):
        import torch
        if u is None:
            u = torch.empty(self.N, dtype=torch.float64, device=f.device)
        if gradu is None:
            gradu = torch.empty(2, self.N, dtype=torch.float64, device=f.device)
        vp_eval(self.tree, f, u, gradu)
        return u, gradu

    def close(self):
        if getattr(self, "tree", None):
            vp_tree_free(self.tree)
            self.tree = None
        if getattr(self, "tables", None):
            vp_tables_free(self.tables)
            self.tables = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------- boundary integral equation

def _p(t):
    return ctypes.c_void_p(t.data_ptr())


class BIE:
    """Nystrom discretisation of 1/2 mu + D[mu] + W[mu] = g on a star boundary, solved by GMRES on the GPU."""

    def __init__(self, alpha, R=1.0, A=0.3, k=5, phase=0.0, n_panels=256, max_krylov=300, stream=None):
        import torch
        out = ctypes.c_void_p()
        _check(load_library().bie_create(float(alpha), float(R), float(A), int(k), float(phase), int(n_panels),
                                         int(max_krylov), _stream_ptr(stream), ctypes.byref(out)), "bie_create")
        self.handle = out.value
        n = ctypes.c_int(); L = ctypes.c_double()
        _check(load_library().bie_size(ctypes.c_void_p(self.handle), ctypes.byref(n), ctypes.byref(L)), "bie_size")
        self.N, self.length, self.alpha = n.value, L.value, alpha
        self.max_krylov = max_krylov
        nodes = torch.empty(7, self.N, dtype=torch.float64, device="cuda")
        _check(load_library().bie_nodes(ctypes.c_void_p(self.handle), _p(nodes), _stream_ptr(stream)), "bie_nodes")
        self.nodes = nodes   # x, y, nx, ny, w, kappa, t

    def apply(self, mu, out=None, stream=None):
        import torch
        out = torch.empty_like(mu) if out is None else out
        _check(load_library().bie_apply(ctypes.c_void_p(self.handle), _p(mu), _p(out), _stream_ptr(stream)), "bie_apply")
        return out

    def solve(self, g, mu0=None, tol=1e-11, max_iter=None, stream=None, aug=None):
        """Returns (mu, iterations, true relative residual); mu0 is the initial guess (zeros if None);
        aug an optional augmentation direction (bie_solve_aug)."""
        import torch
        mu = torch.zeros_like(g) if mu0 is None else mu0.clone()
        it = ctypes.c_int(); rr = ctypes.c_double()
        augc = aug.contiguous() if aug is not None else None
        d = ctypes.c_void_p(augc.data_ptr()) if augc is not None else ctypes.c_void_p(0)
        _check(load_library().bie_solve_aug(ctypes.c_void_p(self.handle), _p(g), _p(mu), d, float(tol),
                                            int(max_iter or self.max_krylov), ctypes.byref(it), ctypes.byref(rr),
                                            _stream_ptr(stream)), "bie_solve_aug")
        return mu, it.value, rr.value

    def eval(self, mu, txy, stream=None):
        import torch
        M = txy.shape[1]
        u = torch.empty(2, M, dtype=torch.float64, device="cuda")
        _check(load_library().bie_eval(ctypes.c_void_p(self.handle), _p(mu), int(M), _p(txy), _p(u),
                                       _stream_ptr(stream)), "bie_eval")
        return u

    def close(self):
        if getattr(self, "handle", None):
            load_library().bie_free(ctypes.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bie_stokeslets(alpha, src, f, xy, stream=None):
    """u [2][M] of stokeslets at src [K][2] with strengths f [K][2] (device float64 tensors) at xy [2][M]."""
    import torch
    M = xy.shape[1]
    u = torch.empty(2, M, dtype=torch.float64, device="cuda")
    _check(load_library().bie_stokeslets(float(alpha), int(src.shape[0]), _p(src), _p(f), int(M), _p(xy), _p(u),
                                         _stream_ptr(stream)), "bie_stokeslets")
    return u


def bie_kernel_scalars(z, stream=None):
    """T1, T2, T3, S1, S2 of the stresslet and stokeslet at z (device float64) -> [5][n]."""
    import torch
    out = torch.empty(5, z.numel(), dtype=torch.float64, device="cuda")
    _check(load_library().bie_kernel_scalars(int(z.numel()), _p(z), _p(out), _stream_ptr(stream)),
           "bie_kernel_scalars")
    return out


class WarmStartNet:
    """Circular 1D conv net over boundary nodes (FP32), hand-written CUDA forward/backward/Adam."""

    def __init__(self, in_ch=8, width=64, out_ch=2, n_layers=4, ksize=9, n=4096, max_batch=32, seed=5, stream=None):
        out = ctypes.c_void_p()
        _check(load_library().ws_create(in_ch, width, out_ch, n_layers, ksize, n, max_batch, ctypes.c_uint64(seed),
                                        _stream_ptr(stream), ctypes.byref(out)), "ws_create")
        self.handle = out.value
        cnt = ctypes.c_int64()
        _check(load_library().ws_num_params(ctypes.c_void_p(self.handle), ctypes.byref(cnt)), "ws_num_params")
        self.n_params = cnt.value
        self.in_ch, self.out_ch, self.n, self.max_batch = in_ch, out_ch, n, max_batch

    def params(self):
        import torch
        buf = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        _check(load_library().ws_params(ctypes.c_void_p(self.handle), _p(buf), 1, _stream_ptr(None)), "ws_params")
        return buf

    def set_params(self, buf):
        _check(load_library().ws_params(ctypes.c_void_p(self.handle), _p(buf), 0, _stream_ptr(None)), "ws_params")

    def forward(self, x):
        import torch
        y = torch.empty(x.shape[0], self.out_ch, self.n, dtype=torch.float32, device="cuda")
        _check(load_library().ws_forward(ctypes.c_void_p(self.handle), _p(x), int(x.shape[0]), _p(y),
                                         _stream_ptr(None)), "ws_forward")
        return y

    def grad(self, x, t):
        import torch
        g = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        loss = ctypes.c_float()
        _check(load_library().ws_grad(ctypes.c_void_p(self.handle), _p(x), _p(t), int(x.shape[0]), _p(g),
                                      ctypes.byref(loss), _stream_ptr(None)), "ws_grad")
        return g, loss.value

    def train_step(self, x, t, lr):
        loss = ctypes.c_float()
        _check(load_library().ws_train_step(ctypes.c_void_p(self.handle), _p(x), _p(t), int(x.shape[0]), float(lr),
                                            ctypes.byref(loss), _stream_ptr(None)), "ws_train_step")
        return loss.value

    def close(self):
        if getattr(self, "handle", None):
            load_library().ws_free(ctypes.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
