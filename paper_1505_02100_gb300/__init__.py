"""Python binding of libkde (include/kde.h): argument marshalling only.

Every step of the PLUGIN bandwidth selector (Algorithm 1 of Gramacki, Sawerwain
& Gramacki) runs in the CUDA library; this module passes pointers and sizes.
It raises ``RuntimeError`` when ``libkde.so`` has not been built -- there is no
CPU fallback.

Inputs may be numpy arrays (host memory) or torch tensors (host or CUDA); the
library detects device pointers itself.  ``stream`` is a ``torch.cuda.Stream``,
a raw ``cudaStream_t`` as int, or ``None`` for the legacy default stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkde.so")

KDE_OK, KDE_ERR_INVALID, KDE_ERR_DEGENERATE, KDE_ERR_DOMAIN = 0, 1, 2, 3
KDE_ERR_OOM, KDE_ERR_CUDA, KDE_ERR_TIMEOUT, KDE_ERR_BUSY = 4, 5, 6, 7
KDE_FP32, KDE_FP64, KDE_Q32 = 0, 1, 2
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "DEGENERATE", 3: "DOMAIN", 4: "OOM", 5: "CUDA",
                6: "TIMEOUT", 7: "BUSY"}
RESULT_FIELDS = ("mean", "sigma", "psi8", "g1", "psi6", "g2", "psi4", "h")
STATIC_MAX_N = 65536   # KDE_STATIC_MAX_N


class KdeResult(ctypes.Structure):
    _fields_ = [(f, ctypes.c_double) for f in RESULT_FIELDS] + [
        ("status", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        d = {f: getattr(self, f) for f in RESULT_FIELDS}
        d["status"] = self.status
        return d


class KdeStageResult(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_double), ("sigma", ctypes.c_double),
                ("psi", ctypes.c_double * 6), ("g", ctypes.c_double * 6), ("h", ctypes.c_double),
                ("stages", ctypes.c_int32), ("status", ctypes.c_int32)]

    def as_dict(self):
        return {"mean": self.mean, "sigma": self.sigma, "h": self.h, "stages": self.stages,
                "status": self.status,
                "psi": {2 * k + 4: self.psi[k] for k in range(6)},
                "g": {2 * k + 4: self.g[k] for k in range(6)}}


class KdeServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int32),
                ("device", ctypes.c_int32), ("tick_target_ms", ctypes.c_double)]


class KdeRequestTimes(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("precision", ctypes.c_int32), ("status", ctypes.c_int32),
                ("t_submit_ns", ctypes.c_int64), ("t_admit_ns", ctypes.c_int64),
                ("t_done_ns", ctypes.c_int64), ("skipped6", ctypes.c_uint64),
                ("skipped4", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


RESULT_BYTES = ctypes.sizeof(KdeResult)

# (name, restype, argtypes) of every exported function
_vp, _i64, _i32, _d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
SIGNATURES = {
    "kde_psi": (_i32, [_vp, _i64, ctypes.c_int, _d, ctypes.c_int, _vp, _vp]),
    "kde_plugin_h": (_i32, [_vp, _i64, ctypes.c_int, _vp, _vp]),
    "kde_plugin_h_f32": (_i32, [_vp, _i64, ctypes.c_int, _vp, _vp]),
    "kde_plugin_h_batch": (_i32, [_vp, _vp, _i64, ctypes.c_int, _vp, _vp]),
    "kde_plugin_h_stages": (_i32, [_vp, _i64, ctypes.c_int, ctypes.c_int, _vp, _vp]),
    "kde_psi_slots": (_i32, [_vp, _i64, ctypes.c_int, _d, ctypes.c_int, _vp, _i64, _vp]),
    "kde_psi_static": (_i32, [_vp, _i64, ctypes.c_int, _d, ctypes.c_int, _vp, _vp]),
    "kde_eval": (_i32, [_vp, _i64, _d, _vp, _i64, ctypes.c_int, _vp, _vp]),
    "kde_autotune": (_i32, [ctypes.c_int, _vp, ctypes.c_int]),
    "kde_autotune_clear": (_i32, [ctypes.c_int]),
    "kde_tile_config": (_i32, [ctypes.c_int, _i64, _vp]),
    "kde_server_create": (_i32, [_vp, _vp]),
    "kde_server_submit": (_i32, [_vp, _vp, _i64, ctypes.c_int, _vp]),
    "kde_server_poll": (_i32, [_vp, ctypes.c_uint64, _i32, _vp, _vp]),
    "kde_server_destroy": (None, [_vp]),
    "kde_last_error": (ctypes.c_char_p, []),
    "kde_version": (ctypes.c_char_p, []),
    "kde_shutdown": (None, []),
    "kde_profile_enable": (_i32, [ctypes.c_int]),
    "kde_profile_last": (_i32, [_vp, _vp, ctypes.c_int]),
    "kde_probe_pipe_rates": (_i32, [_vp, ctypes.c_int]),
}

_lib = None


class KdeError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load(path: str = LIB_PATH):
    """Load libkde.so; raise if it is missing (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libkde.so not built ({path}); run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _buf(x, dtype):
    """(pointer, count, keepalive) of a 1-D contiguous buffer of `dtype`."""
    if hasattr(x, "data_ptr"):  # torch tensor
        import torch
        want = torch.float64 if dtype == np.float64 else torch.float32
        if x.dtype != want:
            raise TypeError(f"expected {want}, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), x.numel(), x
    a = np.ascontiguousarray(np.asarray(x, dtype=dtype)).reshape(-1)
    return a.ctypes.data, a.size, a


def _check(st):
    if st != KDE_OK:
        raise KdeError(st, kde_last_error())


def kde_last_error() -> str:
    return load().kde_last_error().decode()


def kde_version() -> str:
    return load().kde_version().decode()


def kde_shutdown() -> None:
    load().kde_shutdown()


def kde_profile_enable(on: bool = True) -> None:
    _check(load().kde_profile_enable(1 if on else 0))


def kde_profile_last(stream=None):
    """Device ms of the last profiled run on `stream`: setup (init + sort +
    moments + prescale), pairs6, prescale4, pairs4; `launches`, the number of
    kernel launches of that run; `skipped6` / `skipped4`, the unique pairs the
    pair kernels skipped as far tile pairs."""
    ms = (ctypes.c_double * 7)()
    _check(load().kde_profile_last(_stream(stream), ctypes.addressof(ms), 7))
    out = dict(zip(("setup", "pairs6", "prescale4", "pairs4"), list(ms)[:4]))
    out["launches"] = int(ms[4])
    out["skipped6"], out["skipped4"] = int(ms[5]), int(ms[6])
    return out


def kde_probe_pipe_rates():
    """Per-SM throughputs (per second) measured by microbenchmark kernels."""
    out = (ctypes.c_double * 5)()
    _check(load().kde_probe_pipe_rates(ctypes.addressof(out), 5))
    return dict(zip(("fp32_fma_lanes_per_s_sm", "mufu_ex2_per_s_sm", "fp64_fma_lanes_per_s_sm",
                     "sms", "cycle_counter_hz"), list(out)))


def kde_psi(x, r: int, g: float, prec: int = KDE_FP32, out=None, stream=None):
    """psi_r(g) (Steps IV / VI, Eqs. 6-7).  With a CUDA tensor `out` (>= 1 float64)
    the call is asynchronous and returns None; else returns the float."""
    p, n, keep = _buf(x, np.float64)
    if out is not None:
        st = load().kde_psi(p, n, int(r), float(g), int(prec), out.data_ptr(), _stream(stream))
        _check(st)
        return None
    v = ctypes.c_double()
    st = load().kde_psi(p, n, int(r), float(g), int(prec), ctypes.addressof(v), _stream(stream))
    _check(st)
    return v.value


def kde_eval(x, h: float, points, prec: int = KDE_FP32, out=None, stream=None):
    """Eq. 1 with the Gaussian kernel (Eq. 2): fhat(t) = (1/(n h)) sum_i K((t - x_i)/h)
    at every point.  Returns a numpy array, or None with a CUDA tensor `out` of
    >= m float64 (asynchronous)."""
    px, n, keep_x = _buf(x, np.float64)
    pt, m, keep_t = _buf(points, np.float64)
    if out is not None:
        _check(load().kde_eval(px, n, float(h), pt, m, int(prec), out.data_ptr(), _stream(stream)))
        return None
    res = np.empty(m, dtype=np.float64)
    _check(load().kde_eval(px, n, float(h), pt, m, int(prec), res.ctypes.data, _stream(stream)))
    return res


def kde_autotune(prec: int = KDE_FP32):
    """Time every pair-kernel tile configuration on this device; the fastest per
    size class is used from now on.  Returns the chosen configuration per class
    (n = 2^10, 2^12, 2^14, 2^16, 2^18 and above)."""
    out = (ctypes.c_int32 * 5)()
    _check(load().kde_autotune(int(prec), ctypes.addressof(out), 5))
    return list(out)


def kde_autotune_clear(prec: int = KDE_FP32) -> None:
    _check(load().kde_autotune_clear(int(prec)))


def kde_tile_config(n: int, prec: int = KDE_FP32):
    """(configuration index, threads per block, rows per thread) a plan for n uses now."""
    out = (ctypes.c_int32 * 3)()
    _check(load().kde_tile_config(int(prec), int(n), ctypes.addressof(out)))
    return tuple(out)


def kde_psi_static(x, r: int, g: float, prec: int = KDE_FP32, out=None, stream=None):
    """psi_r(g) like kde_psi for n <= STATIC_MAX_N, in the library's fixed scratch
    area (no device allocation).  Calls must not overlap on the device."""
    p, n, keep = _buf(x, np.float64)
    if out is not None:
        _check(load().kde_psi_static(p, n, int(r), float(g), int(prec), out.data_ptr(), _stream(stream)))
        return None
    v = ctypes.c_double()
    _check(load().kde_psi_static(p, n, int(r), float(g), int(prec), ctypes.addressof(v), _stream(stream)))
    return v.value


def kde_plugin_h(x, prec: int = KDE_FP32, out=None, stream=None, check: bool = True):
    """Algorithm 1 for one sample.  Returns the result dict, or None with a CUDA
    `out` tensor of >= 72 bytes (asynchronous)."""
    f32 = (hasattr(x, "dtype") and str(x.dtype) in ("float32", "torch.float32"))
    p, n, keep = _buf(x, np.float32 if f32 else np.float64)
    fn = load().kde_plugin_h_f32 if f32 else load().kde_plugin_h
    if out is not None:
        _check(fn(p, n, int(prec), out.data_ptr(), _stream(stream)))
        return None
    res = KdeResult()
    st = fn(p, n, int(prec), ctypes.addressof(res), _stream(stream))
    if check and st not in (KDE_OK, KDE_ERR_DEGENERATE, KDE_ERR_DOMAIN):
        _check(st)
    return res.as_dict()


def kde_plugin_h_stages(x, stages: int, prec: int = KDE_FP32, out=None, stream=None, check: bool = True):
    """The l-stage direct plug-in (l = stages, 1..4; 2 is Algorithm 1).  Returns a dict
    with psi / g keyed by the order r, or None with a CUDA `out` tensor (asynchronous)."""
    p, n, keep = _buf(x, np.float64)
    if out is not None:
        _check(load().kde_plugin_h_stages(p, n, int(stages), int(prec), out.data_ptr(), _stream(stream)))
        return None
    res = KdeStageResult()
    st = load().kde_plugin_h_stages(p, n, int(stages), int(prec), ctypes.addressof(res), _stream(stream))
    if check and st not in (KDE_OK, KDE_ERR_DEGENERATE, KDE_ERR_DOMAIN):
        _check(st)
    return res.as_dict()


def kde_plugin_h_batch(x_packed, offsets, prec: int = KDE_FP32, out=None, stream=None):
    """Algorithm 1 for m samples packed back to back; offsets has m+1 entries."""
    p, n, keep = _buf(x_packed, np.float64)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    m = off.size - 1
    if out is not None:
        _check(load().kde_plugin_h_batch(p, off.ctypes.data, m, int(prec), out.data_ptr(),
                                         _stream(stream)))
        return None
    res = (KdeResult * m)()
    _check(load().kde_plugin_h_batch(p, off.ctypes.data, m, int(prec), ctypes.addressof(res),
                                     _stream(stream)))
    return [res[k].as_dict() for k in range(m)]


def kde_psi_slots(x, r: int, g: float, prec: int = KDE_FP32):
    """(slots, info) of the pair kernel for psi_r(g): per-chunk sums of He_r(u) exp(-u^2/2)."""
    p, n, keep = _buf(x, np.float64)
    info = (ctypes.c_int64 * 4)()
    _check(load().kde_psi_slots(p, n, int(r), float(g), int(prec), None, 0, ctypes.addressof(info)))
    slots = np.empty(info[3], dtype=np.float64)
    _check(load().kde_psi_slots(p, n, int(r), float(g), int(prec), slots.ctypes.data, slots.size,
                                ctypes.addressof(info)))
    return slots, {"tile": info[0], "chunk": info[1], "n_tile_pairs": info[2], "n_slots": info[3]}


class Server:
    """Continuous-batching bandwidth-selection server (kde_server_* entry points)."""

    def __init__(self, hbm_budget_bytes: int = 8 << 30, max_inflight: int = 256, device: int = 0,
                 tick_target_ms: float = 0.0):
        cfg = KdeServerConfig(hbm_budget_bytes, max_inflight, device, tick_target_ms)
        h = ctypes.c_void_p()
        _check(load().kde_server_create(ctypes.addressof(cfg), ctypes.addressof(h)))
        self._h = h

    def submit(self, x, prec: int = KDE_FP32) -> int:
        a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
        t = ctypes.c_uint64()
        _check(load().kde_server_submit(self._h, a.ctypes.data, a.size, int(prec), ctypes.addressof(t)))
        return t.value

    def poll(self, ticket: int, timeout_ms: int = -1):
        """(result dict, times dict), or None on timeout."""
        res, tm = KdeResult(), KdeRequestTimes()
        st = load().kde_server_poll(self._h, ctypes.c_uint64(ticket), int(timeout_ms),
                                    ctypes.addressof(res), ctypes.addressof(tm))
        if st == KDE_ERR_TIMEOUT:
            return None
        _check(st)
        return res.as_dict(), tm.as_dict()

    def close(self):
        if self._h:
            load().kde_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
