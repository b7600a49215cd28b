"""ctypes binding of the C ABI declared in include/map_smoother.h.

Argument marshalling only: every computation runs in the CUDA library.  The
library must have been built (``paper_2512_13319_gb300.build.build()``);
loading fails loudly otherwise, and there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

MAP_OK, MAP_ERR_INVALID_ARG, MAP_ERR_SHAPE, MAP_ERR_CUDA = 0, -1, -2, -3
MAP_ERR_SINGULAR, MAP_ERR_TIMEOUT, MAP_ERR_UNSUPPORTED = -4, -5, -6
MAP_MODEL_LINEAR, MAP_MODEL_COORD_TURN, MAP_MODEL_CUBIC = 0, 1, 2
MAP_FP64, MAP_FP32 = 0, 1
MAP_EULER, MAP_EXPM, MAP_AUTO, MAP_BLOCK_EULER, MAP_RICCATI_EXACT = 0, 1, 2, 3, 4
MAP_RTS, MAP_TWO_FILTER = 0, 1

_STATUS = {0: "MAP_OK", -1: "MAP_ERR_INVALID_ARG", -2: "MAP_ERR_SHAPE", -3: "MAP_ERR_CUDA",
           -4: "MAP_ERR_SINGULAR", -5: "MAP_ERR_TIMEOUT", -6: "MAP_ERR_UNSUPPORTED"}

_D = ctypes.POINTER(ctypes.c_double)


class map_problem_desc(ctypes.Structure):
    _fields_ = [
        ("model", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nw", ctypes.c_int),
        ("T", ctypes.c_int64), ("t0", ctypes.c_double), ("dt", ctypes.c_double),
        ("F", _D), ("c", _D), ("L", _D), ("W", _D), ("H", _D), ("r", _D), ("R", _D),
        ("m0", _D), ("P0", _D), ("gamma", ctypes.c_double),
        ("precision", ctypes.c_int), ("discretisation", ctypes.c_int), ("smoother", ctypes.c_int),
        ("gn_iters", ctypes.c_int), ("cond_max", ctypes.c_double), ("tile_threads", ctypes.c_int),
        ("substeps", ctypes.c_int), ("steps_per_thread", ctypes.c_int),
    ]


# every exported symbol of include/map_smoother.h with its ctypes signature
_VP, _I, _CH = ctypes.c_void_p, ctypes.c_int, ctypes.c_char_p
EXPORTS = {
    "map_smoother_create": (_I, [ctypes.POINTER(_VP), ctypes.POINTER(map_problem_desc)]),
    "map_smoother_solve": (_I, [_VP, _VP, _VP, _VP, _D, _VP]),
    "map_smoother_solve_sequential": (_I, [_VP, _VP, _VP, _VP]),
    "map_smoother_solve_host": (_I, [_VP, _VP, _VP, _VP]),
    "map_smoother_dense": (_I, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "map_smoother_solve_noalloc": (_I, [ctypes.POINTER(map_problem_desc), _VP, _VP, _VP]),
    "map_smoother_grad": (_I, [_VP, _VP, _VP, _VP, _I, _D, _VP]),
    "map_smoother_update": (_I, [_VP, _D, ctypes.c_double, ctypes.c_double]),
    "map_smoother_stats": (_I, [_VP, ctypes.POINTER(ctypes.c_ulonglong), _I, _VP]),
    "map_smoother_profile": (_I, [_VP, _I]),
    "map_smoother_phase_times": (_I, [_VP, ctypes.POINTER(ctypes.c_float), _I, ctypes.POINTER(_I)]),
    "map_smoother_geometry": (_I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "map_smoother_launches": (_I, [_VP, ctypes.POINTER(_I)]),
    "map_smoother_solve_path": (_I, [_VP, ctypes.POINTER(_I)]),
    "map_smoother_destroy": (None, [_VP]),
    "map_smoother_last_error": (_CH, [_VP]),
    "map_smoother_supported": (_I, [_I, _I, _I, _I]),
    "map_smoother_version": (_CH, []),
    "map_batch_create": (_I, [ctypes.POINTER(_VP), ctypes.POINTER(map_problem_desc), _I,
                              ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_I), _I]),
    "map_batch_rows": (_I, [_VP, _I, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "map_batch_solve": (_I, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _VP]),
    "map_batch_tuning": (_I, [_VP, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "map_batch_last_error": (_CH, [_VP]),
    "map_batch_destroy": (None, [_VP]),
    "map_batch_persistent": (_I, [_VP]),
    "map_fma_peak": (_I, [_I, _I, _D, ctypes.POINTER(ctypes.c_float), _VP]),
    "map_smoother_wait_selftest": (_I, [_VP, _I, _VP]),
    "map_smoother_log_normaliser": (_I, [_VP, _D]),
}

_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return _build.LIB


def load():
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = lib_path()
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library not built: {path} missing "
                                   "(run paper_2512_13319_gb300.build.build())")
            lib = ctypes.CDLL(path)
            for name, (res, args) in EXPORTS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
        return _lib


class MapError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


def _check(status, handle=None):
    if status != MAP_OK:
        msg = load().map_smoother_last_error(handle)
        raise MapError(status, msg.decode() if msg else "")


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_D)


def _f64(a, shape):
    if a is None:
        return None
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(shape))


def map_smoother_create(desc: map_problem_desc) -> int:
    h = ctypes.c_void_p()
    _check(load().map_smoother_create(ctypes.byref(h), ctypes.byref(desc)))
    return h.value


def map_smoother_solve(h, y_ptr, x_ptr, filt_ptr=None, want_cost=False, stream=None):
    cost = ctypes.c_double(0.0)
    _check(load().map_smoother_solve(h, y_ptr, x_ptr, filt_ptr,
                                     ctypes.pointer(cost) if want_cost else None, stream), h)
    return cost.value if want_cost else None


def map_smoother_solve_sequential(h, y_ptr, x_ptr, stream=None):
    _check(load().map_smoother_solve_sequential(h, y_ptr, x_ptr, stream), h)


def map_smoother_dense(h, y_ptr, x_ptr, filt_ptr, dense_ptr, stream=None):
    _check(load().map_smoother_dense(h, y_ptr, x_ptr, filt_ptr, dense_ptr, stream), h)


def map_smoother_solve_host(h, y_host_ptr, x_host_ptr, stream=None):
    _check(load().map_smoother_solve_host(h, y_host_ptr, x_host_ptr, stream), h)


MAP_GRAD_LOGDET = 1


def map_smoother_grad(h, y_ptr, x_ptr, dldx_ptr, n_theta, flags=0, stream=None):
    out = (ctypes.c_double * n_theta)()
    _check(load().map_smoother_grad(h, y_ptr, x_ptr, dldx_ptr, int(flags), out, stream), h)
    return np.array(out[:], dtype=np.float64)


def map_smoother_update(h, F=None, log_q=0.0, log_r=0.0):
    Fp = None if F is None else np.ascontiguousarray(np.asarray(F, dtype=np.float64))
    _check(load().map_smoother_update(h, _ptr(Fp), float(log_q), float(log_r)), h)


def map_smoother_stats(h, reset=False, stream=None):
    out = (ctypes.c_ulonglong * 3)()
    _check(load().map_smoother_stats(h, out, int(bool(reset)), stream), h)
    return int(out[0]), int(out[1]), int(out[2])


PHASES = ("filter_reduce", "filter_down", "rts_down")
PHASES_TWO_FILTER = ("forward_reduce", "forward_states", "backward_reduce", "backward_combine")


def map_smoother_profile(h, enable=True):
    _check(load().map_smoother_profile(h, int(bool(enable))), h)


def map_smoother_geometry(h):
    """(K steps per thread, B threads per tile, tiles) of the handle."""
    K, Bt, nt = _I(), _I(), _I()
    _check(load().map_smoother_geometry(h, ctypes.byref(K), ctypes.byref(Bt), ctypes.byref(nt)), h)
    return K.value, Bt.value, nt.value


def map_smoother_log_normaliser(h):
    out = ctypes.c_double(0.0)
    _check(load().map_smoother_log_normaliser(h, ctypes.byref(out)), h)
    return out.value


def map_smoother_wait_selftest(h, polls, stream=None):
    _check(load().map_smoother_wait_selftest(h, int(polls), stream), h)


FMA_FP32, FMA_FP32X2, FMA_FP64 = 0, 1, 2


def map_fma_peak(kind, iters, stream=None):
    """(flops executed, device ms) of the FMA-throughput kernel of `kind`."""
    flop, ms = ctypes.c_double(0.0), ctypes.c_float(0.0)
    st = load().map_fma_peak(kind, iters, ctypes.byref(flop), ctypes.byref(ms), stream)
    if st != MAP_OK:
        raise MapError(st, "map_fma_peak failed")
    return flop.value, ms.value


MAP_PATH_TABLES, MAP_PATH_SINGLE, MAP_PATH_PIPELINE = 1, 2, 3
PATH_NAMES = {0: "none", 1: "single launch, per-step tables", 2: "single launch, per-step combines",
              3: "multi-kernel pipeline"}


def map_smoother_solve_path(h):
    n = ctypes.c_int(0)
    _check(load().map_smoother_solve_path(h, ctypes.byref(n)), h)
    return n.value


def map_smoother_launches(h):
    """Kernels launched by the handle's last solve."""
    n = _I()
    _check(load().map_smoother_launches(h, ctypes.byref(n)), h)
    return n.value


def map_smoother_phase_times(h):
    buf = (ctypes.c_float * 8)()
    n = ctypes.c_int(0)
    _check(load().map_smoother_phase_times(h, buf, 8, ctypes.byref(n)), h)
    return [float(v) for v in buf[:n.value]]


def map_smoother_destroy(h):
    if h:
        load().map_smoother_destroy(h)


def map_smoother_supported(model, nx, ny, precision) -> bool:
    return bool(load().map_smoother_supported(model, nx, ny, precision))


def map_smoother_version() -> str:
    return load().map_smoother_version().decode()


_MODEL_KIND = {"linear": MAP_MODEL_LINEAR, "coord_turn": MAP_MODEL_COORD_TURN, "cubic": MAP_MODEL_CUBIC}


def make_desc(model, T, dt, precision=MAP_FP32, discretisation=MAP_EULER, smoother=MAP_RTS,
              gn_iters=1, cond_max=0.0, tile_threads=0, t0=0.0, substeps=0, steps_per_thread=0):
    """Build a map_problem_desc from a ``synth.Model``; returns (desc, keepalive)."""
    n, m = model.nx, model.ny
    nw = model.L.shape[1]
    arrs = {
        "F": _f64(model.F, (n, n)) if model.F is not None else None,
        "c": _f64(model.c, (n,)) if model.c is not None else None,
        "L": _f64(model.L, (n, nw)), "W": _f64(model.W, (nw, nw)),
        "H": _f64(model.H, (m, n)) if model.H is not None else None,
        "r": _f64(model.r, (m,)) if model.r is not None else None,
        "R": _f64(model.R, (m, m)), "m0": _f64(model.m0, (n,)), "P0": _f64(model.P0, (n, n)),
    }
    d = map_problem_desc()
    d.model = _MODEL_KIND[model.kind]
    d.nx, d.ny, d.nw, d.T, d.t0, d.dt = n, m, nw, int(T), float(t0), float(dt)
    for k, v in arrs.items():
        setattr(d, k, _ptr(v))
    d.gamma = float(model.params.get("gamma", 0.0))
    d.precision, d.discretisation, d.smoother = precision, discretisation, smoother
    d.gn_iters, d.cond_max, d.tile_threads = int(gn_iters), float(cond_max), int(tile_threads)
    d.substeps = int(substeps)
    d.steps_per_thread = int(steps_per_thread)
    return d, arrs
