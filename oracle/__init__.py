"""CPU oracle of the PLUGIN bandwidth selector (Algorithm 1, Steps I-VII; Eqs. 6-7).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
(the CUDA path behind the C ABI) never imports, links or calls it, and the two
share no code: this package is plain C compiled with gcc plus a ctypes shim.

Precision: IEEE binary64 throughout, compensated (Neumaier) sums; a long double
brute force (``plugin_ld`` / ``psi_ld``) for tiny n.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kde_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_INVALID, ERR_DEGENERATE, ERR_DOMAIN = 0, 1, 2, 3
FORM_FULL, FORM_SYMMETRIC = 0, 1


class Result(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("mean", "sigma", "psi8", "g1", "psi6", "g2", "psi4", "h")] + [("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class StageResult(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_double), ("sigma", ctypes.c_double),
                ("psi", ctypes.c_double * 6), ("g", ctypes.c_double * 6), ("h", ctypes.c_double),
                ("stages", ctypes.c_int), ("status", ctypes.c_int)]

    def as_dict(self):
        return {"mean": self.mean, "sigma": self.sigma, "h": self.h, "stages": self.stages,
                "status": self.status,
                "psi": {2 * k + 4: self.psi[k] for k in range(6)},
                "g": {2 * k + 4: self.g[k] for k in range(6)}}


class ResultLD(ctypes.Structure):
    _fields_ = [(k, ctypes.c_longdouble) for k in
                ("mean", "sigma", "psi8", "g1", "psi6", "g2", "psi4", "h")] + [("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (no GPU, no CUDA)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                                  os.path.getmtime(os.path.join(_HERE, "kde_oracle.h")))):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-fno-fast-math",
                        "-ffp-contract=off", "-Wall", "-o", tmp, _SRC, "-lm", "-lpthread"],
                       check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        d, i64, ip = ctypes.c_double, ctypes.c_int64, ctypes.c_int
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_moments.argtypes = [dp, i64, dp, dp]
        lib.oracle_kernel_deriv.argtypes = [ip, d]
        lib.oracle_kernel_deriv.restype = d
        lib.oracle_psi.argtypes = [dp, i64, ip, d, ip, ip, dp]
        lib.oracle_psi_block.argtypes = [dp, i64, i64, i64, i64, i64, ip, d, dp, dp]
        lib.oracle_plugin.argtypes = [dp, i64, ip, ip, ctypes.POINTER(Result)]
        lib.oracle_plugin_ld.argtypes = [dp, i64, ctypes.POINTER(ResultLD)]
        lib.oracle_psi_ld.argtypes = [dp, i64, ip, ctypes.c_longdouble,
                                      ctypes.POINTER(ctypes.c_longdouble)]
        lib.oracle_long_double_mantissa_bits.restype = ip
        lib.oracle_kde_eval.argtypes = [dp, i64, d, dp, i64, ip, dp]
        lib.oracle_plugin_stages.argtypes = [dp, i64, ip, ip, ip, ctypes.POINTER(StageResult)]
        lib.oracle_q32_mul.argtypes = [i64, i64]
        lib.oracle_q32_mul.restype = i64
        lib.oracle_q32_exp_half.argtypes = [i64]
        lib.oracle_q32_exp_half.restype = i64
        lib.oracle_psi_q32.argtypes = [dp, i64, ip, d, d, d, ip, dp, dp]
        lib.oracle_plugin_q32.argtypes = [dp, i64, ip, ctypes.POINTER(Result)]
        _lib = lib
    return _lib


def default_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def _arr(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def moments(x):
    """Step I: (mean, unbiased variance)."""
    a = _arr(x)
    m, v = ctypes.c_double(), ctypes.c_double()
    st = _load().oracle_moments(_ptr(a), a.size, ctypes.byref(m), ctypes.byref(v))
    if st != OK:
        raise ValueError(f"oracle_moments status {st}")
    return m.value, v.value


def kernel_deriv(r: int, u: float) -> float:
    """K^(r)(u), r in {4, 6} (Algorithm 1, Steps IV and VI) and r in {8, 10}."""
    return _load().oracle_kernel_deriv(int(r), float(u))


def psi(x, r: int, g: float, form: int = FORM_SYMMETRIC, threads: int | None = None) -> float:
    """psi_r(g) = n^-2 g^-(r+1) sum_i sum_j K^(r)((X_i - X_j)/g)."""
    a = _arr(x)
    out = ctypes.c_double()
    st = _load().oracle_psi(_ptr(a), a.size, int(r), float(g), int(form),
                            int(threads or default_threads()), ctypes.byref(out))
    if st != OK:
        raise ValueError(f"oracle_psi status {st}")
    return out.value


def psi_block(x, i0: int, i1: int, j0: int, j1: int, r: int, g: float):
    """(sum, sum of |terms|) of K^(r)((X_i - X_j)/g) over i in [i0,i1), j in [j0,j1), i < j."""
    a = _arr(x)
    s, t = ctypes.c_double(), ctypes.c_double()
    st = _load().oracle_psi_block(_ptr(a), a.size, i0, i1, j0, j1, int(r), float(g),
                                  ctypes.byref(s), ctypes.byref(t))
    if st != OK:
        raise ValueError(f"oracle_psi_block status {st}")
    return s.value, t.value


def plugin(x, form: int = FORM_SYMMETRIC, threads: int | None = None) -> dict:
    """Algorithm 1, Steps I-VII; returns the dict of all intermediate scalars."""
    a = _arr(x)
    res = Result()
    _load().oracle_plugin(_ptr(a), a.size, int(form), int(threads or default_threads()),
                          ctypes.byref(res))
    return res.as_dict()


def plugin_ld(x) -> dict:
    """Algorithm 1 in long double by brute force (full double loop)."""
    a = _arr(x)
    res = ResultLD()
    _load().oracle_plugin_ld(_ptr(a), a.size, ctypes.byref(res))
    return res.as_dict()


def psi_ld(x, r: int, g: float) -> float:
    a = _arr(x)
    out = ctypes.c_longdouble()
    st = _load().oracle_psi_ld(_ptr(a), a.size, int(r), ctypes.c_longdouble(g), ctypes.byref(out))
    if st != OK:
        raise ValueError(f"oracle_psi_ld status {st}")
    return out.value


def long_double_bits() -> int:
    return _load().oracle_long_double_mantissa_bits()


def kde_eval(x, h: float, points, threads: int | None = None) -> np.ndarray:
    """Eq. (1) with the Gaussian kernel (Eq. 2): fhat(t) = (1/(n h)) sum_i K((t - X_i)/h)
    at every point t."""
    a, t = _arr(x), _arr(points).reshape(-1)
    out = np.empty(t.size, dtype=np.float64)
    st = _load().oracle_kde_eval(_ptr(a), a.size, float(h), _ptr(t), t.size,
                                 int(threads or default_threads()), _ptr(out))
    if st != OK:
        raise ValueError(f"oracle_kde_eval status {st}")
    return out


def plugin_stages(x, stages: int, form: int = FORM_SYMMETRIC, threads: int | None = None) -> dict:
    """The l-stage direct plug-in (l = stages, 1..4): psi_{2l+4} by the normal scale,
    then psi_{2l+2} .. psi_4 at pilot bandwidths, then h; l = 2 is Algorithm 1."""
    a = _arr(x)
    res = StageResult()
    _load().oracle_plugin_stages(_ptr(a), a.size, int(stages), int(form),
                                 int(threads or default_threads()), ctypes.byref(res))
    return res.as_dict()


def q32_mul(a: int, b: int) -> int:
    """Q32.32 product (truncation toward -inf) of two raw int64 values."""
    return _load().oracle_q32_mul(int(a), int(b))


def q32_exp_half(w: int) -> int:
    """floor(2^32 exp(-w/2)) for the Q32.32 raw value w >= 0."""
    return _load().oracle_q32_exp_half(int(w))


def psi_q32(x, r: int, g: float, mean: float, sigma: float, threads: int | None = None):
    """(psi_r(g), sum |He_r|) with the pair sum in Q32.32 on z-scored data."""
    a = _arr(x)
    out, tot = ctypes.c_double(), ctypes.c_double()
    st = _load().oracle_psi_q32(_ptr(a), a.size, int(r), float(g), float(mean), float(sigma),
                                int(threads or default_threads()), ctypes.byref(out), ctypes.byref(tot))
    if st != OK:
        raise ValueError(f"oracle_psi_q32 status {st}")
    return out.value, tot.value


def plugin_q32(x, threads: int | None = None) -> dict:
    """Algorithm 1 with the Steps IV / VI pair sums in Q32.32 on z-scored data (Eq. 3)."""
    a = _arr(x)
    res = Result()
    _load().oracle_plugin_q32(_ptr(a), a.size, int(threads or default_threads()), ctypes.byref(res))
    return res.as_dict()
