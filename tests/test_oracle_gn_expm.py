"""Pins of the oracle's Gauss-Newton with per-step exact discretisation of the
local linear drift (Section 4.4 iterated linearisation; Eq. 37 A, b, C rows
solved exactly with the coefficients of the linearisation at x_{k+1}).

- For a linear model the linearisation is exact: one iteration from any start
  is the linear EXPM solve, and the Euler mode is the linear Euler solve.
- On the coordinated turn (tiny T, brute force) the fixed point x* is the
  argmin of the linear problem whose elements are built at x* from
  finite-difference Jacobians of the model's own drift and measurement
  functions, with the interval integrals done by numerical quadrature of
  scipy's matrix exponential, minimised by the dense least-squares definition.
"""
import numpy as np
import pytest
from scipy.integrate import quad_vec
from scipy.linalg import expm

import oracle
from oracle import dense
from paper_2512_13319_gb300 import synth


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("mode", [oracle.EULER, oracle.EXPM])
def test_linear_model_one_iteration_is_the_linear_solve(mode):
    m = synth.ou_model(4, 2, seed=3)
    m.c = np.array([0.3, -0.2, 0.1, 0.05])
    m.r = np.array([0.1, -0.1])
    T, dt = 300, 0.05
    _, y = synth.simulate(m, T, dt, seed=4)
    x0 = np.random.default_rng(5).standard_normal((T + 1, 4))
    x = oracle.gauss_newton(m, y, dt, x0, 1, mode=mode)
    assert rel(x, oracle.smooth_lti(m, y, dt, mode=mode)) < 1e-11


def test_modes_differ_on_a_nonlinear_model():
    """The two discretisations are different problems (first order in dt)."""
    m = synth.coordinated_turn()
    T, dt = 200, 0.01
    _, y = synth.simulate(m, T, dt, seed=8)
    x0 = np.tile(m.m0, (T + 1, 1))
    xe = oracle.gauss_newton(m, y, dt, x0, 10, mode=oracle.EULER)
    xx = oracle.gauss_newton(m, y, dt, x0, 10, mode=oracle.EXPM)
    d = rel(xx, xe)
    assert 1e-9 < d < 1e-2


def _fd_jac(fun, x, h=1e-6):
    n = x.shape[0]
    f0 = fun(x)
    J = np.empty((f0.shape[0], n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = h
        J[:, j] = (fun(x + e) - fun(x - e)) / (2 * h)
    return J


def test_coordinated_turn_fixed_point_is_the_argmin_of_its_linearisation():
    m = synth.coordinated_turn()
    T, dt = 5, 0.05
    _, y = synth.simulate(m, T, dt, seed=11)
    x0 = np.tile(m.m0, (T + 1, 1))
    xs = oracle.gauss_newton(m, y, dt, x0, 60, mode=oracle.EXPM)
    assert np.abs(oracle.gauss_newton(m, y, dt, xs, 1, mode=oracle.EXPM) - xs).max() < 1e-10
    n, p = m.nx, m.ny
    Q = m.Q
    A = np.empty((T, n, n)); b = np.empty((T, n)); C = np.empty((T, n, n))
    G = np.empty((T, p, n)); g = np.empty((T, p))
    w, V = np.linalg.eigh(m.R / dt)
    Rm = V @ np.diag(w ** -0.5) @ V.T
    for k in range(T):
        xb = xs[k + 1]
        Fk = _fd_jac(lambda z: synth._drift(m, z), xb)
        ck = synth._drift(m, xb) - Fk @ xb
        A[k] = expm(-Fk * dt)
        C[k] = quad_vec(lambda u: expm(-Fk * u) @ Q @ expm(-Fk * u).T, 0.0, dt, epsabs=1e-15, epsrel=1e-13)[0]
        b[k] = -quad_vec(lambda u: expm(-Fk * u) @ ck, 0.0, dt, epsabs=1e-15, epsrel=1e-13)[0]
        Hk = _fd_jac(lambda z: synth.measure(m, z), xb)
        res = y[k] - synth.measure(m, xb)
        res[1] = (res[1] + np.pi) % (2 * np.pi) - np.pi
        G[k] = Rm @ Hk
        g[k] = Rm @ (res + Hk @ xb)
    xd = dense.dense_map(A, b, C, G, g, m.m0, m.P0)
    assert np.abs(xd - xs).max() <= 1e-7 * max(1.0, np.abs(xs).max())
