"""FP64 CPU oracle for the parallel MAP smoother (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference legs may import this package.  It shares no code with the CUDA
library: the arithmetic lives in ``map_oracle.c`` (plain C, FP64) and in
``dense.py`` (NumPy, the brute-force definition), both written from the paper.

Parity status of each function (see the pins in ``tests/test_oracle_*.py``):
every exported function here is pinned by at least one test that does not
re-type its own formula; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "map_oracle.c")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

KIND_LINEAR, KIND_CT, KIND_CUBIC = 0, 1, 2
# model kind names carried by the model objects the tests pass in
_KIND_BY_NAME = {"linear": KIND_LINEAR, "coord_turn": KIND_CT, "cubic": KIND_CUBIC}


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            D = ctypes.POINTER(ctypes.c_double)
            i, d, l = ctypes.c_int, ctypes.c_double, ctypes.c_long
            _lib.orc_discretise.argtypes = [i, d, D, D, D, i, D, D, D]
            _lib.orc_forward_model.argtypes = [i, D, D, D, D, D, D]
            _lib.orc_kf_rts.argtypes = [i, i, D, l, D, l, D, l, D, l, D, l, D, D, D, D, D]
            _lib.orc_two_filter.argtypes = [i, i, D, l, D, l, D, l, D, l, D, l, D, D, D]
            _lib.orc_combine.argtypes = [i, D, D, D]
            _lib.orc_elements_lti.argtypes = [i, i, i, d, D, D, D, D, D, D, D, D]
            _lib.orc_filter_by_combine.argtypes = [i, i, D, D, D, D, D]
            _lib.orc_two_filter_paper.argtypes = [i, i, D, D, D, D]
            _lib.orc_smooth_lti.argtypes = [i, i, i, d, i, i, D, D, D, D, D, D, D, D, D, D, D, D]
            _lib.orc_cost.argtypes = [i, i, i, i, d, D, D, d, D, D, D, D, D, D, D, D, D]
            _lib.orc_gauss_newton.argtypes = [i, i, i, i, d, D, D, d, D, D, D, D, D, D, D, D, i, i, D]
            _lib.orc_grad_lti.argtypes = [i, i, i, d, D, D, D, d, D, D, D, d, D, D, D, D, i, D, D]
            _lib.orc_block_elements.argtypes = [i, i, i, i, d, D, D, D, D, D, D, D, D]
            _lib.orc_exact_elements.argtypes = [i, i, i, d, D, D, D, D, D, D, D, D]
            _lib.orc_smooth_elements.argtypes = [i, i, D, D, D, D, D, D]
            _lib.orc_dense_block.argtypes = [i, i, i, i, d, D, D, D, D, D, D, D, D, D, D, D]
        return _lib


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _check(rc):
    if rc != 0:
        raise np.linalg.LinAlgError(f"oracle returned status {rc}")


EULER, EXPM = 0, 1


def discretise(F, c, Q, dt, mode=EULER):
    """Interval element (A, b, C) of a linear drift over one step (Eq. 37)."""
    F = _f(F); n = F.shape[0]
    A = np.empty((n, n)); b = np.empty(n); C = np.empty((n, n))
    _check(_load().orc_discretise(n, dt, _p(F), _p(_f(c, (n,))), _p(_f(Q)), mode, _p(A), _p(b), _p(C)))
    return A, b, C


def forward_model(A, b, C):
    """Forward transition (Phi, beta, Sigma) equivalent to the element (A, b, C)."""
    A = _f(A); n = A.shape[0]
    Phi = np.empty((n, n)); beta = np.empty(n); Sig = np.empty((n, n))
    _check(_load().orc_forward_model(n, _p(A), _p(_f(b)), _p(_f(C)), _p(Phi), _p(beta), _p(Sig)))
    return Phi, beta, Sig


def _per_step(a, T, shape):
    a = _f(a)
    size = int(np.prod(shape))
    if a.size == size:
        return a.reshape(shape), 0
    assert a.shape[0] == T and a[0].size == size, (a.shape, T, shape)
    return a, size


def kf_rts(Phi, beta, Sig, J, eta, m0, P0, T, return_filter=False):
    """Sequential Kalman filter + RTS smoother with information terms on x_{k+1}."""
    m0 = _f(m0); n = m0.shape[0]
    Phi, sP = _per_step(Phi, T, (n, n)); beta, sb = _per_step(beta, T, (n,))
    Sig, sS = _per_step(Sig, T, (n, n)); J, sJ = _per_step(J, T, (n, n))
    eta, se = _per_step(eta, T, (n,))
    x = np.empty((T + 1, n))
    mf = np.empty((T + 1, n)) if return_filter else None
    Pf = np.empty((T + 1, n, n)) if return_filter else None
    _check(_load().orc_kf_rts(n, T, _p(Phi), sP, _p(beta), sb, _p(Sig), sS, _p(J), sJ,
                              _p(eta), se, _p(m0), _p(_f(P0)), _p(x), _p(mf), _p(Pf)))
    return (x, mf, Pf) if return_filter else x


def two_filter(Phi, beta, Sig, J, eta, m0, P0, T):
    """Two-filter smoother (forward filter + backward information filter)."""
    m0 = _f(m0); n = m0.shape[0]
    Phi, sP = _per_step(Phi, T, (n, n)); beta, sb = _per_step(beta, T, (n,))
    Sig, sS = _per_step(Sig, T, (n, n)); J, sJ = _per_step(J, T, (n, n))
    eta, se = _per_step(eta, T, (n,))
    x = np.empty((T + 1, n))
    _check(_load().orc_two_filter(n, T, _p(Phi), sP, _p(beta), sb, _p(Sig), sS, _p(J), sJ,
                                  _p(eta), se, _p(m0), _p(_f(P0)), _p(x)))
    return x


def elem_size(n):
    return 3 * n * n + 2 * n


def pack_element(A, b, C, eta, J):
    return np.concatenate([_f(A).ravel(), _f(b).ravel(), _f(C).ravel(), _f(eta).ravel(), _f(J).ravel()])


def unpack_element(e, n):
    e = _f(e)
    o = 0
    A = e[o:o + n * n].reshape(n, n); o += n * n
    b = e[o:o + n]; o += n
    C = e[o:o + n * n].reshape(n, n); o += n * n
    eta = e[o:o + n]; o += n
    J = e[o:o + n * n].reshape(n, n)
    return A, b, C, eta, J


def combine(ei, ej, n):
    """The paper's combine e_i (x) e_j (Eq. 36)."""
    out = np.empty(elem_size(n))
    _check(_load().orc_combine(n, _p(_f(ei)), _p(_f(ej)), _p(out)))
    return out


def elements_lti(model, y, dt, mode=EULER):
    """Original-time-ordered interval elements (T, 3n^2+2n) of a linear model."""
    y = _f(y); T = y.shape[0]; n, m = model.nx, model.ny
    A, b, C = discretise(model.F, model.c, model.Q, dt, mode)
    out = np.empty((T, elem_size(n)))
    _check(_load().orc_elements_lti(n, m, T, dt, _p(A), _p(b), _p(C), _p(_f(model.H)),
                                    _p(_f(model.r)), _p(_f(model.R)), _p(y), _p(out)))
    return out


def filter_by_combine(elems, m0, P0):
    """S_k, v_k by sequentially folding the combine with the prior element."""
    elems = _f(elems); T = elems.shape[0]; m0 = _f(m0); n = m0.shape[0]
    S = np.empty((T + 1, n, n)); v = np.empty((T + 1, n))
    _check(_load().orc_filter_by_combine(n, T, _p(elems), _p(m0), _p(_f(P0)), _p(S), _p(v)))
    return S, v


def two_filter_paper(elems, m0, P0):
    """The paper's two-filter smoother with abar_0 (needs invertible J_0)."""
    elems = _f(elems); T = elems.shape[0]; m0 = _f(m0); n = m0.shape[0]
    x = np.empty((T + 1, n))
    _check(_load().orc_two_filter_paper(n, T, _p(elems), _p(m0), _p(_f(P0)), _p(x)))
    return x


RTS, TWO_FILTER = 0, 1


def smooth_lti(model, y, dt, mode=EULER, smoother=RTS, return_filter=False):
    """MAP trajectory (T+1, nx) of a linear model by the sequential smoother."""
    y = _f(y); T = y.shape[0]; n, m = model.nx, model.ny
    x = np.empty((T + 1, n))
    mf = np.empty((T + 1, n)) if return_filter else None
    Pf = np.empty((T + 1, n, n)) if return_filter else None
    _check(_load().orc_smooth_lti(n, m, T, dt, mode, smoother, _p(_f(model.F)), _p(_f(model.c)),
                                  _p(_f(model.Q)), _p(_f(model.H)), _p(_f(model.r)),
                                  _p(_f(model.R)), _p(_f(model.m0)), _p(_f(model.P0)), _p(y),
                                  _p(x), _p(mf), _p(Pf)))
    return (x, mf, Pf) if return_filter else x


def _kind_of(model):
    return _KIND_BY_NAME[model.kind]


def _model_arrays(model):
    n, m = model.nx, model.ny
    F = _f(model.F) if model.F is not None else np.zeros((n, n))
    c = _f(model.c) if model.c is not None else np.zeros(n)
    H = _f(model.H) if model.H is not None else np.zeros((m, n))
    r = _f(model.r) if model.r is not None else np.zeros(m)
    return F, c, H, r


def cost(model, y, x, dt):
    """Discrete Onsager-Machlup cost M(x) (Euler intervals; Q must be invertible)."""
    y = _f(y); x = _f(x); T = y.shape[0]; n, m = model.nx, model.ny
    F, c, H, r = _model_arrays(model)
    out = ctypes.c_double()
    _check(_load().orc_cost(_kind_of(model), n, m, T, dt, _p(F), _p(c),
                            float(model.params.get("gamma", 0.0)), _p(_f(model.Q)), _p(H), _p(r),
                            _p(_f(model.R)), _p(_f(model.m0)), _p(_f(model.P0)), _p(y), _p(x),
                            ctypes.byref(out)))
    return out.value


def gauss_newton(model, y, dt, x_init, iters, mode=EULER):
    """Iterated linearisation (Gauss-Newton) MAP trajectory of a nonlinear model
    (Section 4.4); mode EXPM discretises each step's local linear drift exactly."""
    y = _f(y); T = y.shape[0]; n, m = model.nx, model.ny
    F, c, H, r = _model_arrays(model)
    x = np.empty((T + 1, n))
    _check(_load().orc_gauss_newton(_kind_of(model), n, m, T, dt, _p(F), _p(c),
                                    float(model.params.get("gamma", 0.0)), _p(_f(model.Q)),
                                    _p(H), _p(r), _p(_f(model.R)), _p(_f(model.m0)),
                                    _p(_f(model.P0)), _p(y), _p(_f(x_init)), iters, int(mode), _p(x)))
    return x


def grad_lti(model, y, dt, logq=0.0, logr=0.0, dLdx=None, logdet=False):
    """dL/d(F, log q, log r) with Q = e^logq Q_model, R = e^logr R_model.

    Returns (grad (n*n+2,), x*).  ``dLdx=None`` differentiates the MAP cost.
    """
    y = _f(y); T = y.shape[0]; n, m = model.nx, model.ny
    F, c, H, r = _model_arrays(model)
    g = np.empty(n * n + 2)
    x = np.empty((T + 1, n))
    _check(_load().orc_grad_lti(n, m, T, dt, _p(F), _p(c), _p(_f(model.Q)), float(logq), _p(H),
                                _p(r), _p(_f(model.R)), float(logr), _p(_f(model.m0)),
                                _p(_f(model.P0)), _p(y), _p(None if dLdx is None else _f(dLdx)),
                                int(bool(logdet)), _p(g), _p(x)))
    return g, x


# ---------------------------------------------------------------- block and exact elements

def block_elements(model, y, dt, nsub):
    """Block elements (T, 3n^2+2n): nsub explicit Euler substeps of Eq. 37 per
    interval (Section 5.1) with the interval's sample held, combined by Eq. 36."""
    y = _f(y); T = y.shape[0]; n, m = model.nx, model.ny
    out = np.empty((T, elem_size(n)))
    _check(_load().orc_block_elements(n, m, T, int(nsub), dt, _p(_f(model.F)), _p(_f(model.c, (n,))),
                                      _p(_f(model.Q)), _p(_f(model.H)), _p(_f(model.r, (m,))),
                                      _p(_f(model.R)), _p(y), _p(out)))
    return out


def exact_elements(model, y, dt):
    """Exact elements (T, 3n^2+2n): Eq. 37 solved over each interval with constant
    coefficients and the interval's sample held (Hamiltonian matrix exponential)."""
    y = _f(y); T = y.shape[0]; n, m = model.nx, model.ny
    out = np.empty((T, elem_size(n)))
    _check(_load().orc_exact_elements(n, m, T, dt, _p(_f(model.F)), _p(_f(model.c, (n,))), _p(_f(model.Q)),
                                      _p(_f(model.H)), _p(_f(model.r, (m,))), _p(_f(model.R)), _p(y), _p(out)))
    return out


def smooth_elements(elems, m0, P0, return_filter=False):
    """MAP trajectory (T+1, n) for per-step elements by the sequential KF + RTS."""
    elems = _f(elems); T = elems.shape[0]; m0 = _f(m0); n = m0.shape[0]
    x = np.empty((T + 1, n))
    mf = np.empty((T + 1, n)) if return_filter else None
    Pf = np.empty((T + 1, n, n)) if return_filter else None
    _check(_load().orc_smooth_elements(n, T, _p(elems), _p(m0), _p(_f(P0)), _p(x), _p(mf), _p(Pf)))
    return (x, mf, Pf) if return_filter else x


def smooth_block(model, y, dt, nsub, return_filter=False):
    """MAP trajectory of the block-element discretisation (Section 5.1)."""
    return smooth_elements(block_elements(model, y, dt, nsub), model.m0, model.P0, return_filter)


def smooth_exact(model, y, dt, return_filter=False):
    """MAP trajectory of the exact-element discretisation (Eq. 37 solved exactly)."""
    return smooth_elements(exact_elements(model, y, dt), model.m0, model.P0, return_filter)


def dense_block(model, y, dt, nsub):
    """States at every substep (nsub T + 1, n) of a block solve (Section 4.3
    recovery between grid points) from its grid states and filter moments."""
    y = _f(y); T = y.shape[0]; n, m = model.nx, model.ny
    x, mf, Pf = smooth_block(model, y, dt, nsub, return_filter=True)
    xd = np.empty((nsub * T + 1, n))
    _check(_load().orc_dense_block(n, m, T, int(nsub), dt, _p(_f(model.F)), _p(_f(model.c, (n,))),
                                   _p(_f(model.Q)), _p(_f(model.H)), _p(_f(model.r, (m,))), _p(_f(model.R)),
                                   _p(y), _p(x), _p(mf), _p(_f(Pf)), _p(xd)))
    return xd
