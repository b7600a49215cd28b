"""Seeded synthetic workloads: model definitions and simulated observations.

This module only *describes* models and *simulates* data from them.  It holds
none of the estimation method's arithmetic (no discretisation of the smoothing
problem, no filtering, no combine): both the CUDA path and the FP64 oracle
consume its output, and neither is used to produce it.

Models (all FP64 numpy):

* Wiener velocity in ``d`` dimensions (Section 5.1, linear experiment): state
  (positions, velocities), ``F = [[0, I], [0, 0]]``, ``L = [0; I]``, position
  measurements ``H = [I 0]``.
* Ornstein-Uhlenbeck with random stable drift: ``F = U diag(lam) U^T`` with
  ``U`` Haar-orthogonal and ``lam ~ U[-5, -0.1]``, ``L = I``, ``H = [I_m 0]``.
* Coordinated turn (Section 5.2, nonlinear experiment): state
  ``(xi, zeta, dxi, dzeta, omega)``, drift ``(dxi, dzeta, -omega dzeta,
  omega dxi, 0)``, range-bearing measurement.

Observations follow the continuous-time measurement model of Eq. (1) sampled
on the grid: ``y_k = h(x_k) + N(0, R/dt)`` for ``k = 1..T`` (row ``k-1`` of the
returned array); ``x_0`` is observed only through the prior.  The truth is
simulated by Euler-Maruyama with ``substeps`` sub-steps per grid interval.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# model kinds, mirrored by the C-ABI enum in include/map_smoother.h
LINEAR = "linear"
COORD_TURN = "coord_turn"
CUBIC = "cubic"


@dataclass
class Model:
    """A state-space model of Eq. (1) with Gaussian prior p(x(t0)) = N(m0, P0).

    Linear models carry ``F, c, H, r`` (Eq. 14); nonlinear ones carry a
    ``kind`` that names a built-in drift/measurement pair.  ``L`` and ``W``
    give ``Q = L W L^T``; ``R`` is the measurement spectral density.
    """

    kind: str
    nx: int
    ny: int
    L: np.ndarray
    W: np.ndarray
    R: np.ndarray
    m0: np.ndarray
    P0: np.ndarray
    F: np.ndarray | None = None
    c: np.ndarray | None = None
    H: np.ndarray | None = None
    r: np.ndarray | None = None
    params: dict = field(default_factory=dict)

    @property
    def Q(self) -> np.ndarray:
        return self.L @ self.W @ self.L.T


def wiener_velocity(d: int = 2, q: float = 1.0, r: float = 0.1,
                    m0=None, P0=None) -> Model:
    """Wiener-velocity model in ``d`` dimensions (Eq. 44 with ``n_x = 2d``)."""
    n = 2 * d
    F = np.zeros((n, n))
    F[:d, d:] = np.eye(d)
    L = np.zeros((n, d))
    L[d:, :] = np.eye(d)
    H = np.zeros((d, n))
    H[:, :d] = np.eye(d)
    return Model(kind=LINEAR, nx=n, ny=d, F=F, c=np.zeros(n), L=L,
                 W=q * np.eye(d), H=H, r=np.zeros(d), R=r * np.eye(d),
                 m0=np.zeros(n) if m0 is None else np.asarray(m0, float),
                 P0=np.eye(n) if P0 is None else np.asarray(P0, float))


def wiener_velocity_paper_preset() -> Model:
    """Section 5.1 parameters: W = 4 I, R = 1e-2 I, m0 = (5,5,0,0), P0 = 1e-2 I."""
    return wiener_velocity(2, q=4.0, r=1e-2, m0=[5.0, 5.0, 0.0, 0.0],
                           P0=1e-2 * np.eye(4))


def haar_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal matrix (QR of a Gaussian with sign fix)."""
    z = rng.standard_normal((n, n))
    qm, rm = np.linalg.qr(z)
    return qm * np.sign(np.diag(rm))


def ou_model(n: int = 8, m: int = 4, seed: int = 1001, q: float = 1.0,
             r: float = 0.1, lam_range=(-5.0, -0.1)) -> Model:
    """OU model with random stable drift ``F = U diag(lam) U^T``."""
    rng = np.random.default_rng(seed)
    U = haar_orthogonal(n, rng)
    lam = rng.uniform(lam_range[0], lam_range[1], size=n)
    F = U @ np.diag(lam) @ U.T
    H = np.zeros((m, n))
    H[:, :m] = np.eye(m)
    return Model(kind=LINEAR, nx=n, ny=m, F=F, c=np.zeros(n), L=np.eye(n),
                 W=q * np.eye(n), H=H, r=np.zeros(m), R=r * np.eye(m),
                 m0=np.zeros(n), P0=np.eye(n),
                 params={"lam": lam, "U": U})


def coordinated_turn(sigma_v: float = 5e-4, sigma_w: float = 0.02,
                     R=(0.05 ** 2, 0.01 ** 2), m0=(5.0, 5.0, 0.0, 0.3, 0.0),
                     P0=(0.01, 0.01, 0.01, 0.01, 0.04)) -> Model:
    """Coordinated-turn model of Section 5.2 (Eq. 46) with range-bearing h.

    ``L`` is 5x3 with ``sigma_v`` on the two velocity rows and ``sigma_w`` on
    the turn-rate row; ``W = I_3``.
    """
    L = np.zeros((5, 3))
    L[2, 0] = sigma_v
    L[3, 1] = sigma_v
    L[4, 2] = sigma_w
    return Model(kind=COORD_TURN, nx=5, ny=2, L=L, W=np.eye(3),
                 R=np.diag(np.asarray(R, float)), m0=np.asarray(m0, float),
                 P0=np.diag(np.asarray(P0, float)))


def coordinated_turn_paper_preset() -> Model:
    """Section 5.2 values verbatim: R = diag(5e-3, 1e-3)."""
    return coordinated_turn(R=(5e-3, 1e-3))


def cubic_model(n: int = 2, gamma: float = 1.0, q: float = 0.5,
                r: float = 0.05) -> Model:
    """Test model with state-dependent divergence: ``f(x) = F x - gamma x**3``.

    ``F = -0.5 I`` and full-state measurements.  Its divergence
    ``-0.5 n - 3 gamma sum x_i^2`` is not constant, so the Onsager-Machlup
    divergence term of Eq. (2) changes the MAP.
    """
    return Model(kind=CUBIC, nx=n, ny=n, F=-0.5 * np.eye(n), c=np.zeros(n),
                 L=np.eye(n), W=q * np.eye(n), H=np.eye(n), r=np.zeros(n),
                 R=r * np.eye(n), m0=np.zeros(n), P0=np.eye(n),
                 params={"gamma": gamma})


# --------------------------------------------------------------------------
# simulation
# --------------------------------------------------------------------------

def _drift(model: Model, x: np.ndarray) -> np.ndarray:
    if model.kind == LINEAR:
        return x @ model.F.T + model.c
    if model.kind == COORD_TURN:
        out = np.zeros_like(x)
        out[..., 0] = x[..., 2]
        out[..., 1] = x[..., 3]
        out[..., 2] = -x[..., 4] * x[..., 3]
        out[..., 3] = x[..., 4] * x[..., 2]
        return out
    if model.kind == CUBIC:
        return x @ model.F.T + model.c - model.params["gamma"] * x ** 3
    raise ValueError(model.kind)


def measure(model: Model, x: np.ndarray) -> np.ndarray:
    """Noise-free measurement function h(x) of the model."""
    if model.kind in (LINEAR, CUBIC):
        return x @ model.H.T + model.r
    if model.kind == COORD_TURN:
        return np.stack([np.hypot(x[..., 0], x[..., 1]),
                         np.arctan2(x[..., 1], x[..., 0])], axis=-1)
    raise ValueError(model.kind)


def _chol_psd(S: np.ndarray) -> np.ndarray:
    w, V = np.linalg.eigh(0.5 * (S + S.T))
    return V * np.sqrt(np.clip(w, 0.0, None))


def simulate_truth(model: Model, T: int, dt: float, rng: np.random.Generator,
                   substeps: int = 10) -> np.ndarray:
    """Euler-Maruyama truth on the grid ``t_k = k dt``, ``k = 0..T``."""
    n = model.nx
    x0 = model.m0 + _chol_psd(model.P0) @ rng.standard_normal(n)
    h = dt / substeps
    Lw = model.L @ _chol_psd(model.W)
    nw = Lw.shape[1]
    if model.kind == LINEAR and _is_wiener_velocity(model):
        return _simulate_wv(model, T, dt, rng, substeps, x0)
    if model.kind == LINEAR and "U" in model.params:
        return _simulate_ou(model, T, dt, rng, substeps, x0)
    # generic sequential Euler-Maruyama (small T or nonlinear models)
    if model.kind == COORD_TURN:
        return _simulate_ct(model, T, dt, rng, substeps, x0)
    xs = np.empty((T + 1, n))
    x = x0.copy()
    xs[0] = x
    for k in range(T):
        for _ in range(substeps):
            x = x + h * _drift(model, x) + math.sqrt(h) * (Lw @ rng.standard_normal(nw))
        xs[k + 1] = x
    return xs


def _is_wiener_velocity(model: Model) -> bool:
    n = model.nx
    if n % 2:
        return False
    d = n // 2
    ref = np.zeros((n, n))
    ref[:d, d:] = np.eye(d)
    return model.F is not None and np.array_equal(model.F, ref) and not np.any(model.c)


def _simulate_wv(model, T, dt, rng, substeps, x0):
    # velocity is a Brownian motion, position its Euler integral
    n = model.nx
    d = n // 2
    h = dt / substeps
    N = T * substeps
    sq = np.linalg.cholesky(model.W) * math.sqrt(h)
    dv = rng.standard_normal((N, d)) @ sq.T
    v = np.empty((N + 1, d))
    v[0] = x0[d:]
    np.cumsum(dv, axis=0, out=v[1:])
    v[1:] += x0[d:]
    p = np.empty((N + 1, d))
    p[0] = x0[:d]
    np.cumsum(h * v[:-1], axis=0, out=p[1:])
    p[1:] += x0[:d]
    xs = np.concatenate([p, v], axis=1)
    return np.ascontiguousarray(xs[::substeps])


def _simulate_ou(model, T, dt, rng, substeps, x0):
    # Euler-Maruyama in the eigenbasis of the symmetric drift: n AR(1) chains
    from scipy.signal import lfilter
    U = model.params["U"]
    lam = model.params["lam"]
    h = dt / substeps
    N = T * substeps
    Lw = model.L @ _chol_psd(model.W)
    noise = rng.standard_normal((N, Lw.shape[1])) @ (math.sqrt(h) * (U.T @ Lw)).T
    z0 = U.T @ x0
    z = np.empty((N + 1, model.nx))
    z[0] = z0
    for i in range(model.nx):
        a = 1.0 + h * lam[i]
        zi, _ = lfilter([1.0], [1.0, -a], noise[:, i], zi=[a * z0[i]])
        z[1:, i] = zi
    xs = z @ U.T
    return np.ascontiguousarray(xs[::substeps])


def _simulate_ct(model, T, dt, rng, substeps, x0):
    # turn rate: random walk; velocity (as a complex number) rotates by omega
    h = dt / substeps
    N = T * substeps
    sv = model.L[2, 0] * math.sqrt(model.W[0, 0])
    sw = model.L[4, 2] * math.sqrt(model.W[2, 2])
    nz = rng.standard_normal((N, 3)) * math.sqrt(h)
    om = np.empty(N + 1)
    om[0] = x0[4]
    np.cumsum(sw * nz[:, 2], out=om[1:])
    om[1:] += x0[4]
    g = 1.0 + 1j * h * om[:-1]              # u_{j+1} = g_j u_j + e_j
    logP = np.concatenate([[0.0], np.cumsum(np.log(g))])
    e = sv * (nz[:, 0] + 1j * nz[:, 1])
    u0 = x0[2] + 1j * x0[3]
    acc = np.cumsum(e * np.exp(-logP[1:]))
    u = np.empty(N + 1, complex)
    u[0] = u0
    u[1:] = np.exp(logP[1:]) * (u0 + acc)
    pos = np.empty(N + 1, complex)
    pos[0] = x0[0] + 1j * x0[1]
    np.cumsum(h * u[:-1], out=pos[1:])
    pos[1:] += pos[0]
    xs = np.stack([pos.real, pos.imag, u.real, u.imag, om], axis=1)
    return np.ascontiguousarray(xs[::substeps])


def simulate(model: Model, T: int, dt: float, seed: int, substeps: int = 10,
             min_range: float | None = 0.5, max_tries: int = 50):
    """Simulate truth ``x (T+1, nx)`` and observations ``y (T, ny)``.

    ``y[k-1] = h(x_k) + N(0, R/dt)`` for ``k = 1..T``.  For the coordinated
    turn the draw is repeated with the next seed while the trajectory comes
    closer than ``min_range`` to the origin (the bearing is singular there).
    """
    for attempt in range(max_tries):
        rng = np.random.default_rng(seed + 7919 * attempt)
        x = simulate_truth(model, T, dt, rng, substeps)
        if model.kind == COORD_TURN and min_range is not None:
            if np.min(np.hypot(x[:, 0], x[:, 1])) < min_range:
                continue
        Rc = _chol_psd(model.R / dt)
        y = measure(model, x[1:]) + rng.standard_normal((T, model.ny)) @ Rc.T
        return x, np.ascontiguousarray(y)
    raise RuntimeError("no admissible trajectory found")


# --------------------------------------------------------------------------
# workload presets (sizes and seeds of the benchmark configurations)
# --------------------------------------------------------------------------

def seed_for(config_index: int) -> int:
    return 1000 + config_index


def batched_lengths_and_dims(num: int = 4096, lo: int = 256, hi: int = 65536,
                             dims=(2, 4, 6), seed: int = 1003):
    """Ragged batch recipe: log-uniform lengths in [lo, hi], nx uniform in dims."""
    rng = np.random.default_rng(seed)
    lengths = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=num))).astype(np.int64)
    nxs = rng.choice(np.asarray(dims), size=num)
    return lengths, nxs


def batched_workload(num: int = 4096, lo: int = 256, hi: int = 65536, seed: int = 1003,
                     dt: float = 0.01, q: float = 1.0, r: float = 0.1, lengths=None, dims=None):
    """Ragged batch of Wiener-velocity trajectories in 1, 2 and 3 dimensions.

    Returns (models [d=1, 2, 3], lengths, model_of, ys) with ys[j] of shape
    (lengths[j], d_j).  Lengths are log-uniform in [lo, hi] unless given.
    """
    if lengths is None:
        lengths, nxs = batched_lengths_and_dims(num, lo, hi, (2, 4, 6), seed)
    else:
        lengths = np.asarray(lengths, dtype=np.int64)
        nxs = np.asarray(dims) * 2
    models = [wiener_velocity(d, q=q, r=r) for d in (1, 2, 3)]
    model_of = (nxs // 2 - 1).astype(np.int32)
    ys = []
    for j, (T, mi) in enumerate(zip(lengths, model_of)):
        _, y = simulate(models[mi], int(T), dt, seed=seed * 100003 + j, substeps=1)
        ys.append(y)
    return models, lengths, model_of, ys
