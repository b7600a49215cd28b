"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks the oracle against the mathematics the paper fixes: the
brute-force dense solve of the MAP stationarity system, closed forms, a
library Riccati solver, the continuous-time Kalman-Bucy steady state, the
definition of the combine as a minimisation, and invariants the paper states
(two-filter = RTS, P = S^-1 and m = S^-1 v, associativity, identity element).
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from oracle import dense
from paper_2512_13319_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def random_lti(n, m, seed, full_rank_q=False):
    rng = np.random.default_rng(seed)
    F = rng.standard_normal((n, n)) * 0.5 - 0.8 * np.eye(n)
    k = n if full_rank_q else max(1, n // 2)
    L = rng.standard_normal((n, k))
    H = rng.standard_normal((m, n))
    return synth.Model(kind=synth.LINEAR, nx=n, ny=m, F=F, c=rng.standard_normal(n) * 0.3,
                       L=L, W=np.diag(rng.uniform(0.5, 2.0, k)), H=H,
                       r=rng.standard_normal(m) * 0.1, R=np.diag(rng.uniform(0.05, 0.3, m)),
                       m0=rng.standard_normal(n), P0=np.diag(rng.uniform(0.5, 2.0, n)))


MODELS = {
    "wv2": lambda: synth.wiener_velocity(2, q=1.0, r=0.1),
    "wv_paper": synth.wiener_velocity_paper_preset,
    "ou4": lambda: synth.ou_model(4, 2, seed=3),
    "rand5": lambda: random_lti(5, 3, seed=11),
    "rand3_fullq": lambda: random_lti(3, 1, seed=12, full_rank_q=True),
}


# ---------------------------------------------------------------- dense pin

@pytest.mark.parametrize("name", sorted(MODELS))
@pytest.mark.parametrize("mode,dt", [(oracle.EULER, 0.01), (oracle.EULER, 0.1), (oracle.EXPM, 0.1)])
def test_kf_rts_equals_dense_solve(name, mode, dt):
    model = MODELS[name]()
    T = 37
    _, y = synth.simulate(model, T, dt, seed=5)
    A, b, C = oracle.discretise(model.F, model.c, model.Q, dt, mode)
    x_orc = oracle.smooth_lti(model, y, dt, mode=mode)
    x_dense = dense.dense_map_lti(model, y, dt, A, b, C)
    assert rel(x_orc, x_dense) < 1e-10


def test_tiny_horizons_against_dense():
    model = MODELS["rand5"]()
    dt = 0.05
    A, b, C = oracle.discretise(model.F, model.c, model.Q, dt)
    for T in (1, 2, 3):
        _, y = synth.simulate(model, T, dt, seed=T)
        assert rel(oracle.smooth_lti(model, y, dt), dense.dense_map_lti(model, y, dt, A, b, C)) < 1e-11


# ---------------------------------------------------------- discretisation

@pytest.mark.parametrize("dt", [1e-3, 0.01, 0.3])
def test_wiener_velocity_exact_discretisation_closed_form(dt):
    """e^{F dt} = [[I, dt I], [0, I]], Sigma = q [[dt^3/3, dt^2/2], [dt^2/2, dt]] (x) I."""
    q, d = 1.7, 2
    model = synth.wiener_velocity(d, q=q)
    c = np.array([0.3, -0.1, 0.7, 0.2])
    A, b, C = oracle.discretise(model.F, c, model.Q, dt, oracle.EXPM)
    I = np.eye(d)
    Phi_ref = np.block([[I, dt * I], [0 * I, I]])
    Sig_ref = q * np.kron(np.array([[dt ** 3 / 3, dt ** 2 / 2], [dt ** 2 / 2, dt]]), I)
    C_ref = q * np.kron(np.array([[dt ** 3 / 3, -dt ** 2 / 2], [-dt ** 2 / 2, dt]]), I)
    b_ref = -np.block([[dt * I, -dt ** 2 / 2 * I], [0 * I, dt * I]]) @ c
    Phi, beta, Sig = oracle.forward_model(A, b, C)
    assert np.allclose(Phi, Phi_ref, rtol=0, atol=1e-14)
    assert np.allclose(Sig, Sig_ref, rtol=1e-12, atol=1e-18)
    assert np.allclose(C, C_ref, rtol=1e-12, atol=1e-18)
    assert np.allclose(b, b_ref, rtol=1e-12, atol=1e-16)


def test_exact_discretisation_matches_library_expm_and_quadrature():
    from scipy.integrate import quad_vec
    model = synth.ou_model(5, 2, seed=9)
    c = np.linspace(-1, 1, 5)
    dt = 0.37
    A, b, C = oracle.discretise(model.F, c, model.Q, dt, oracle.EXPM)
    assert np.allclose(A, sla.expm(-model.F * dt), rtol=1e-13, atol=1e-14)
    C_ref, _ = quad_vec(lambda u: sla.expm(-model.F * u) @ model.Q @ sla.expm(-model.F.T * u), 0, dt,
                        epsabs=1e-14, epsrel=1e-13)
    b_ref, _ = quad_vec(lambda u: -sla.expm(-model.F * u) @ c, 0, dt, epsabs=1e-14, epsrel=1e-13)
    assert np.allclose(C, C_ref, rtol=1e-10, atol=1e-14)
    assert np.allclose(b, b_ref, rtol=1e-10, atol=1e-14)


def test_euler_discretisation_is_one_euler_step():
    """A = I - dt F, b = -dt c, C = dt Q: one Euler step of Eq. (37) from A=I, b=C=0."""
    model = random_lti(4, 2, seed=4)
    dt = 0.02
    A, b, C = oracle.discretise(model.F, model.c, model.Q, dt, oracle.EULER)
    # the Eq. (37) right-hand sides at the boundary values, integrated backwards one step
    Ft, ct = -model.F, -model.c
    dA = -np.eye(4) @ Ft            # -A Q J^T - A F~ with J = 0
    db = -np.eye(4) @ ct            # -A Q eta - A c~ with eta = 0
    dC = -model.Q                   # -A Q A^T
    assert np.allclose(A, np.eye(4) - dt * dA)
    assert np.allclose(b, -dt * db)
    assert np.allclose(C, -dt * dC)


# ------------------------------------------------------------- Riccati pins

def test_filter_covariance_reaches_discrete_riccati_fixed_point():
    model = synth.ou_model(4, 2, seed=21)
    dt = 0.05
    T = 2000
    _, y = synth.simulate(model, T, dt, seed=2)
    A, b, C = oracle.discretise(model.F, model.c, model.Q, dt, oracle.EXPM)
    Phi, beta, Sig = oracle.forward_model(A, b, C)
    _, mf, Pf = oracle.smooth_lti(model, y, dt, mode=oracle.EXPM, return_filter=True)
    P_pred = Phi @ Pf[-1] @ Phi.T + Sig
    X = sla.solve_discrete_are(Phi.T, model.H.T, Sig, model.R / dt)
    assert rel(P_pred, X) < 1e-10


def test_filter_covariance_tends_to_kalman_bucy_steady_state():
    """1-D Wiener velocity: P11 = sqrt2 q^1/4 r^3/4, P12 = sqrt(q r), P22 = sqrt2 q^3/4 r^1/4."""
    q, r = 2.0, 0.3
    model = synth.wiener_velocity(1, q=q, r=r)
    P_ref = np.array([[math.sqrt(2) * q ** 0.25 * r ** 0.75, math.sqrt(q * r)],
                      [math.sqrt(q * r), math.sqrt(2) * q ** 0.75 * r ** 0.25]])
    errs = []
    for dt in (1e-2, 1e-3):
        T = int(round(40.0 / dt))
        y = np.zeros((T, 1))
        _, _, Pf = oracle.smooth_lti(model, y, dt, mode=oracle.EXPM, return_filter=True)
        errs.append(rel(Pf[-1], P_ref))
    assert errs[1] < 2e-3
    assert 5.0 < errs[0] / errs[1] < 20.0          # first order in dt


# ---------------------------------------------------------- smoother pins

@pytest.mark.parametrize("name", sorted(MODELS))
def test_two_filter_equals_rts(name):
    model = MODELS[name]()
    dt = 0.02
    _, y = synth.simulate(model, 300, dt, seed=8)
    for mode in (oracle.EULER, oracle.EXPM):
        x_rts = oracle.smooth_lti(model, y, dt, mode=mode)
        x_tf = oracle.smooth_lti(model, y, dt, mode=mode, smoother=oracle.TWO_FILTER)
        assert rel(x_tf, x_rts) < 1e-11


def test_paper_two_filter_with_full_state_measurement():
    """The literal abar_0 form (needs J_0 invertible) with b_0 included; c != 0."""
    model = synth.wiener_velocity(2, q=1.0, r=0.1)
    model.H = np.eye(4); model.ny = 4; model.r = np.zeros(4); model.R = 0.1 * np.eye(4)
    model.c = np.array([0.3, -0.2, 0.1, 0.5])
    dt = 0.01
    _, y = synth.simulate(model, 120, dt, seed=3)
    el = oracle.elements_lti(model, y, dt)
    x_paper = oracle.two_filter_paper(el, model.m0, model.P0)
    assert rel(x_paper, oracle.smooth_lti(model, y, dt)) < 1e-12


def test_terminal_state_is_filter_mean():
    model = MODELS["rand5"]()
    dt = 0.03
    _, y = synth.simulate(model, 50, dt, seed=4)
    x, mf, _ = oracle.smooth_lti(model, y, dt, return_filter=True)
    assert np.allclose(x[-1], mf[-1], rtol=0, atol=0)


# ---------------------------------------------------------- combine pins

def random_element(n, rng, pd_c=True, scale=1.0):
    A = np.eye(n) + 0.3 * rng.standard_normal((n, n))
    B = rng.standard_normal((n, n if pd_c else max(1, n // 2)))
    C = scale * (B @ B.T + (1e-1 * np.eye(n) if pd_c else 0))
    Bj = rng.standard_normal((n, max(1, n // 2)))
    J = Bj @ Bj.T
    return oracle.pack_element(A, rng.standard_normal(n), C, rng.standard_normal(n), J)


def value(e, n, x, z):
    A, b, C, eta, J = oracle.unpack_element(e, n)
    d = z - A @ x - b
    return 0.5 * x @ J @ x - x @ eta + 0.5 * d @ np.linalg.solve(C, d)


@pytest.mark.parametrize("n", [2, 4, 5])
def test_combine_is_the_min_plus_composition(n):
    """V_ij(x, y) = min_z V_i(x, z) + V_j(z, y) + const (Eq. 35 definition)."""
    rng = np.random.default_rng(100 + n)
    ei, ej = random_element(n, rng), random_element(n, rng)
    eij = oracle.combine(ei, ej, n)
    Ai, bi, Ci, _, _ = oracle.unpack_element(ei, n)
    Aj, bj, Cj, etaj, Jj = oracle.unpack_element(ej, n)
    diffs = []
    for _ in range(6):
        x, yv = rng.standard_normal(n), rng.standard_normal(n)
        # stationarity in z of the sum of the two quadratics
        Ci_inv, Cj_inv = np.linalg.inv(Ci), np.linalg.inv(Cj)
        Hz = Ci_inv + Jj + Aj.T @ Cj_inv @ Aj
        gz = Ci_inv @ (Ai @ x + bi) + etaj + Aj.T @ Cj_inv @ (yv - bj)
        z = np.linalg.solve(Hz, gz)
        diffs.append(value(eij, n, x, yv) - (value(ei, n, x, z) + value(ej, n, z, yv)))
    assert np.ptp(diffs) < 1e-10 * max(1.0, np.max(np.abs(diffs)))


def test_identity_element_is_two_sided():
    n = 4
    rng = np.random.default_rng(1)
    e = random_element(n, rng, pd_c=False)
    ident = oracle.pack_element(np.eye(n), np.zeros(n), np.zeros((n, n)), np.zeros(n), np.zeros((n, n)))
    assert np.allclose(oracle.combine(e, ident, n), e, rtol=0, atol=1e-15)
    assert np.allclose(oracle.combine(ident, e, n), e, rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", range(4))
def test_combine_is_associative(seed):
    n = 4
    rng = np.random.default_rng(seed)
    a, b, c = (random_element(n, rng, pd_c=bool(seed % 2)) for _ in range(3))
    left = oracle.combine(oracle.combine(a, b, n), c, n)
    right = oracle.combine(a, oracle.combine(b, c, n), n)
    assert rel(left, right) < 1e-12


@pytest.mark.parametrize("name", ["wv2", "rand5", "ou4"])
def test_value_function_fold_is_the_information_filter(name):
    """P = S^-1 and m = S^-1 v (Section 2.5) for the fold a_i (x) ... (x) a_T."""
    model = MODELS[name]()
    dt = 0.02
    _, y = synth.simulate(model, 200, dt, seed=6)
    el = oracle.elements_lti(model, y, dt)
    S, v = oracle.filter_by_combine(el, model.m0, model.P0)
    _, mf, Pf = oracle.smooth_lti(model, y, dt, return_filter=True)
    P = np.linalg.inv(S)
    assert rel(P, Pf) < 1e-12
    assert rel(np.einsum("kij,kj->ki", P, v), mf) < 1e-12


# ------------------------------------------------------- Gauss-Newton pins

def test_linear_model_converges_in_one_gauss_newton_iteration():
    model = MODELS["rand5"]()
    dt = 0.02
    T = 80
    _, y = synth.simulate(model, T, dt, seed=1)
    x0 = np.random.default_rng(0).standard_normal((T + 1, model.nx)) * 3
    x_gn = oracle.gauss_newton(model, y, dt, x0, 1)
    assert rel(x_gn, oracle.smooth_lti(model, y, dt)) < 1e-12


def fd_gradient(fun, x, h=1e-6):
    g = np.zeros_like(x)
    it = np.nditer(x, flags=["multi_index"])
    for _ in it:
        idx = it.multi_index
        xp = x.copy(); xp[idx] += h
        xm = x.copy(); xm[idx] -= h
        g[idx] = (fun(xp) - fun(xm)) / (2 * h)
    return g


def test_gauss_newton_fixed_point_is_stationary_cubic_drift():
    """Divergence term included: the fixed point satisfies grad M = 0 (FD of the cost)."""
    model = synth.cubic_model(2, gamma=1.5, q=0.5, r=0.05)
    model.m0 = np.array([1.0, -0.5])
    dt = 0.02
    T = 30
    _, y = synth.simulate(model, T, dt, seed=3)
    x0 = np.tile(model.m0, (T + 1, 1))
    x = oracle.gauss_newton(model, y, dt, x0, 30)
    g = fd_gradient(lambda z: oracle.cost(model, y, z, dt), x)
    scale = np.abs(fd_gradient(lambda z: oracle.cost(model, y, z, dt), x0)).max()
    assert np.abs(g).max() < 1e-7 * scale
    # the divergence gradient 1/2 dt grad(div f) = -3 gamma dt x is far above that
    # bound, so a fixed point that ignored it would fail the check above
    assert 3 * 1.5 * dt * np.abs(x).max() > 1e3 * 1e-7 * scale


def ct_full_rank(R=(0.05 ** 2, 0.01 ** 2)):
    m = synth.coordinated_turn(R=R)
    m.L = np.diag([0.05, 0.05, 0.2, 0.2, 0.05])
    m.W = np.eye(5)
    return m


def test_gauss_newton_fixed_point_is_stationary_coordinated_turn():
    """Pins the turn model's drift, range-bearing h, their Jacobians and the wrap."""
    model = ct_full_rank()
    model.m0 = np.array([-3.0, -0.2, 0.5, 0.8, 0.4])   # crosses the bearing branch cut
    dt = 0.05
    T = 40
    _, y = synth.simulate(model, T, dt, seed=4, min_range=0.5)
    xbar = np.tile(model.m0, (T + 1, 1))
    x = oracle.gauss_newton(model, y, dt, xbar, 25)
    g = fd_gradient(lambda z: oracle.cost(model, y, z, dt), x)
    scale = np.abs(fd_gradient(lambda z: oracle.cost(model, y, z, dt), xbar)).max()
    assert np.abs(g).max() < 1e-7 * scale


# ------------------------------------------------------------ gradient pins

def _ou_theta_model(model, F):
    m = synth.Model(**{**model.__dict__})
    m.F = F
    return m


def _with_noise(model, logq, logr):
    m = synth.Model(**{**model.__dict__})
    m.W = model.W * math.exp(logq)
    m.R = model.R * math.exp(logr)
    return m


@pytest.mark.parametrize("loss", ["map_cost", "trajectory"])
def test_gradient_matches_central_differences(loss):
    model = synth.ou_model(4, 2, seed=31)
    dt = 0.01
    T = 60
    x_true, y = synth.simulate(model, T, dt, seed=2)
    logq, logr = 0.2, -0.3

    def L(F, lq, lr):
        m = _with_noise(_ou_theta_model(model, F), lq, lr)
        x = oracle.smooth_lti(m, y, dt)
        if loss == "map_cost":
            return oracle.cost(m, y, x, dt)
        return 0.5 * np.sum((x - x_true) ** 2)

    m_theta = _with_noise(model, 0.0, 0.0)
    if loss == "map_cost":
        g, x = oracle.grad_lti(m_theta, y, dt, logq, logr)
    else:
        x = oracle.smooth_lti(_with_noise(model, logq, logr), y, dt)
        g, _ = oracle.grad_lti(m_theta, y, dt, logq, logr, dLdx=x - x_true)
    h = 1e-6
    fd = np.zeros_like(g)
    for a in range(4):
        for b in range(4):
            Fp = model.F.copy(); Fp[a, b] += h
            Fm = model.F.copy(); Fm[a, b] -= h
            fd[a * 4 + b] = (L(Fp, logq, logr) - L(Fm, logq, logr)) / (2 * h)
    fd[16] = (L(model.F, logq + h, logr) - L(model.F, logq - h, logr)) / (2 * h)
    fd[17] = (L(model.F, logq, logr + h) - L(model.F, logq, logr - h)) / (2 * h)
    assert rel(g, fd) < 1e-6


def test_gradient_log_normaliser_terms():
    model = synth.ou_model(4, 2, seed=32)
    dt = 0.02
    T = 25
    _, y = synth.simulate(model, T, dt, seed=3)

    def normaliser(lq, lr):
        C = dt * model.Q * math.exp(lq)
        R = model.R * math.exp(lr) / dt
        return 0.5 * T * (np.linalg.slogdet(2 * math.pi * C)[1] + np.linalg.slogdet(2 * math.pi * R)[1])

    g0, _ = oracle.grad_lti(model, y, dt, 0.0, 0.0, logdet=False)
    g1, _ = oracle.grad_lti(model, y, dt, 0.0, 0.0, logdet=True)
    h = 1e-5
    assert abs((g1 - g0)[16] - (normaliser(h, 0) - normaliser(-h, 0)) / (2 * h)) < 1e-6
    assert abs((g1 - g0)[17] - (normaliser(0, h) - normaliser(0, -h)) / (2 * h)) < 1e-6


# --------------------------------------------------------- golden fixtures

def test_paper_model_presets_match_printed_parameters():
    gold = json.load(open(os.path.join(GOLDEN, "paper_models.json")))
    wv = synth.wiener_velocity_paper_preset()
    g = gold["wiener_velocity"]
    assert np.array_equal(wv.F, np.array(g["F"], float))
    assert np.array_equal(wv.H, np.array(g["H"], float))
    assert np.array_equal(wv.L, np.array(g["L"], float))
    assert np.array_equal(wv.W, np.array(g["W"], float))
    assert np.array_equal(wv.R, np.array(g["R"], float))
    assert np.array_equal(wv.m0, np.array(g["m0"], float))
    assert np.array_equal(np.diag(wv.P0), np.array(g["P0_diag"], float))
    ct = synth.coordinated_turn_paper_preset()
    g = gold["coordinated_turn"]
    assert ct.L[2, 0] == g["sigma_v"] and ct.L[3, 1] == g["sigma_v"] and ct.L[4, 2] == g["sigma_omega"]
    assert np.array_equal(ct.W, np.array(g["W"], float))
    assert np.array_equal(np.diag(ct.R), np.array(g["R_diag"], float))
    assert np.array_equal(ct.m0, np.array(g["m0"], float))
    assert np.array_equal(np.diag(ct.P0), np.array(g["P0_diag"], float))
