"""Pins of the oracle's block elements, exact (Riccati) elements and dense
output against things other than themselves (Section 5.1, Eq. 36-37, 40-43).

Block elements: n explicit Euler substeps of Eq. 37 per interval with the
interval's sample held.  Composing the substeps (Eq. 36) minimises out the
intermediate states, so the block problem on T intervals of dt is the
per-step Euler problem on n T intervals of dt / n whose observations repeat
each sample n times: its MAP at the grid points, and the dense output at
every substep, must equal that fine problem's MAP (a separately pinned code
path).  Exact elements: the closed form of Eq. 37 with constant
coefficients; pinned by the measurement-free case (the Van Loan exponential),
by the semigroup property, by the scalar Riccati closed form and by the
first-order convergence of the block elements as n grows.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2512_13319_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore")


def model_with_offsets(seed=5):
    m = synth.ou_model(4, 2, seed=seed)
    m.c = np.array([0.2, -0.1, 0.3, 0.0])
    m.r = np.array([0.1, -0.2])
    m.m0 = np.array([0.5, -0.3, 0.2, 0.1])
    return m


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_block_with_one_substep_is_the_euler_element():
    m = model_with_offsets()
    _, y = synth.simulate(m, 200, 0.02, seed=1)
    assert np.array_equal(oracle.block_elements(m, y, 0.02, 1), oracle.elements_lti(m, y, 0.02))
    assert rel(oracle.smooth_block(m, y, 0.02, 1), oracle.smooth_lti(m, y, 0.02)) < 1e-13


@pytest.mark.parametrize("nsub", [2, 10])
def test_block_solve_is_the_fine_euler_problem_at_the_grid(nsub):
    m = model_with_offsets(7)
    T, dt = 300, 0.02
    _, y = synth.simulate(m, T, dt, seed=2)
    xf = oracle.smooth_lti(m, np.repeat(y, nsub, axis=0), dt / nsub)
    assert rel(oracle.smooth_block(m, y, dt, nsub), xf[::nsub]) < 1e-11


def test_dense_output_is_the_fine_euler_problem_at_every_substep():
    m = model_with_offsets(9)
    T, dt, nsub = 250, 0.02, 10
    _, y = synth.simulate(m, T, dt, seed=3)
    xf = oracle.smooth_lti(m, np.repeat(y, nsub, axis=0), dt / nsub)
    xd = oracle.dense_block(m, y, dt, nsub)
    assert xd.shape == xf.shape
    assert rel(xd, xf) < 1e-11
    assert np.abs(xd - xf).max() / np.abs(xf).max() < 1e-10


def test_block_on_wiener_velocity_matches_fine_problem():
    m = synth.wiener_velocity(2, q=1.0, r=0.1)
    T, dt, nsub = 400, 0.01, 10
    _, y = synth.simulate(m, T, dt, seed=4)
    xf = oracle.smooth_lti(m, np.repeat(y, nsub, axis=0), dt / nsub)
    assert rel(oracle.dense_block(m, y, dt, nsub), xf) < 1e-11


def test_exact_element_without_measurement_is_the_van_loan_element():
    m = model_with_offsets(11)
    m.H = np.zeros_like(m.H)
    dt = 0.05
    e = oracle.exact_elements(m, np.zeros((1, 2)), dt)[0]
    A, b, C, eta, J = oracle.unpack_element(e, 4)
    Ax, bx, Cx = oracle.discretise(m.F, m.c, m.Q, dt, oracle.EXPM)
    assert np.abs(A - Ax).max() < 1e-13
    assert np.abs(b - bx).max() < 1e-13
    assert np.abs(C - Cx).max() < 1e-13
    assert np.abs(J).max() == 0.0 and np.abs(eta).max() == 0.0


def test_exact_elements_form_a_semigroup():
    """The element over 2 dt is the combination (Eq. 36) of two elements over
    dt with the same held sample."""
    m = model_with_offsets(13)
    y = np.array([[0.4, -0.7]])
    for dt in (0.01, 0.1):
        e1 = oracle.exact_elements(m, y, dt)[0]
        e2 = oracle.exact_elements(m, y, 2 * dt)[0]
        assert np.abs(oracle.combine(e1, e1, 4) - e2).max() < 1e-12 * max(1.0, np.abs(e2).max())


def test_scalar_exact_element_closed_form():
    """n = 1: the Riccati row of Eq. 37 with constant coefficients,
    J' = w + 2 a J - q J^2 from J(0) = 0 (a = -f the reversed drift,
    w = h^2 / R), has J(t) = w sinh(k t) / (k cosh(k t) - a sinh(k t)),
    k = sqrt(a^2 + q w); then A(t) = k / (k cosh - a sinh) and
    C(t) = q sinh(k t) / (k cosh(k t) - a sinh(k t))."""
    f, q, h, R = -0.7, 2.0, 1.5, 0.3
    m = synth.Model(kind=synth.LINEAR, nx=1, ny=1, F=np.array([[f]]), c=np.zeros(1), L=np.eye(1),
                    W=np.array([[q]]), H=np.array([[h]]), r=np.zeros(1), R=np.array([[R]]),
                    m0=np.zeros(1), P0=np.eye(1))
    a, w = -f, h * h / R
    k = math.sqrt(a * a + q * w)
    for t in (0.01, 0.3, 2.0):
        e = oracle.exact_elements(m, np.zeros((1, 1)), t)[0]
        A, b, C, eta, J = oracle.unpack_element(e, 1)
        den = k * math.cosh(k * t) - a * math.sinh(k * t)
        assert abs(J[0, 0] - w * math.sinh(k * t) / den) < 1e-12 * max(1.0, abs(J[0, 0]))
        assert abs(A[0, 0] - k / den) < 1e-12
        assert abs(C[0, 0] - q * math.sinh(k * t) / den) < 1e-12 * max(1.0, abs(C[0, 0]))


def test_block_elements_converge_to_the_exact_element_at_first_order():
    m = model_with_offsets(15)
    y = np.array([[0.3, 0.8]])
    dt = 0.05
    ex = oracle.exact_elements(m, y, dt)[0]
    err = {n: np.abs(oracle.block_elements(m, y, dt, n)[0] - ex).max() for n in (128, 256, 512)}
    assert 1.8 < err[128] / err[256] < 2.2 and 1.8 < err[256] / err[512] < 2.2
    # Richardson extrapolation removes the first-order term
    b256, b512 = oracle.block_elements(m, y, dt, 256)[0], oracle.block_elements(m, y, dt, 512)[0]
    assert np.abs(2 * b512 - b256 - ex).max() < 1e-3 * err[512]


def test_exact_solve_matches_fine_block_solve():
    """The exact-element MAP is the limit of the block-element MAP."""
    m = model_with_offsets(17)
    T, dt = 120, 0.05
    _, y = synth.simulate(m, T, dt, seed=5)
    xe = oracle.smooth_exact(m, y, dt)
    x1, x2 = oracle.smooth_block(m, y, dt, 200), oracle.smooth_block(m, y, dt, 400)
    e1, e2 = rel(x1, xe), rel(x2, xe)
    assert e2 < e1 and 1.7 < e1 / e2 < 2.3
    assert rel(2 * x2 - x1, xe) < 0.05 * e2
