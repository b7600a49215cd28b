"""Gradient of the MAP solve (hand-written adjoint in the CUDA library) against
the FP64 oracle's implicit-function gradient and central finite differences."""
import math

import numpy as np
import pytest

import oracle
from paper_2512_13319_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {"fp64": torch.float64, "fp32": torch.float32}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_13319_gb300 import build
    build.build()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


# Per-block tolerances.  The gradient's blocks differ in scale by orders of
# magnitude (the log r entry grows with T while the F block stays O(1)), so a
# norm over the whole vector would hide an error in the F block.  Each block
# -- dL/dF (n*n entries), dL/dlog q, dL/dlog r -- is compared on its own, and
# every F entry against the block's largest entry.  FP64: 1e-8.  FP32: the
# per-step terms are exact functions of the FP32 trajectories x (and lambda),
# so their error is that of the trajectories, about 5e-6 of |x|, and it is
# not smooth: the scan composes its maps in a different order at every
# thread and tile boundary.  The residuals x_k - A x_{k+1} - b that the F
# block is built from are of order dt |w| ~ 1e-3 |x| at the MAP trajectory,
# so at a boundary step a residual is off by ~5e-3 of itself; one step in K
# (K ~ 18) carries such an error, which gives ~1e-4 on the F block (measured:
# 5e-5 .. 2e-4 at T = 2e4 .. 2^18).  1e-3 per block leaves a margin of 5-10.
BTOL = {"fp64": 1e-8, "fp32": 1e-3}


def assert_grad(g, ref, tol):
    g, ref = np.asarray(g, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    nn = len(ref) - 2
    gF, rF = g[:nn], ref[:nn]
    eF = rel(gF, rF)
    assert eF <= tol, f"dL/dF block relative error {eF:.3e} > {tol:.0e}"
    scale = np.abs(rF).max()
    worst = np.abs(gF - rF).max() / scale
    assert worst <= 10 * tol, f"largest dL/dF entry error {worst:.3e} of the block scale > {10 * tol:.0e}"
    for i, name in ((nn, "log q"), (nn + 1, "log r")):
        e = abs(g[i] - ref[i]) / abs(ref[i])
        assert e <= tol, f"dL/d{name} relative error {e:.3e} > {tol:.0e} ({g[i]!r} vs {ref[i]!r})"


def problem(T, dt=1e-3, seed=51):
    model = synth.ou_model(4, 2, seed=seed)
    x_true, y = synth.simulate(model, T, dt, seed=seed + 1, substeps=1)
    return model, x_true, y


def scaled(model, logq, logr):
    m = synth.Model(**{**model.__dict__})
    m.W = model.W * math.exp(logq)
    m.R = model.R * math.exp(logr)
    return m


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("loss", ["map_cost", "trajectory"])
def test_gradient_matches_oracle(prec, loss):
    from paper_2512_13319_gb300 import MapSmoother
    T, dt = 20_000, 1e-3
    model, x_true, y = problem(T, dt)
    logq, logr = 0.3, -0.2
    sm = MapSmoother(model, T, dt, precision=prec)
    sm.update(model.F, logq, logr)
    yt = torch.tensor(y, dtype=DT[prec], device="cuda")
    x = sm.solve(yt)
    if loss == "map_cost":
        g = sm.grad(yt, x)
        ref, _ = oracle.grad_lti(model, y, dt, logq, logr)
    else:
        xt = torch.tensor(x_true, dtype=DT[prec], device="cuda")
        g = sm.grad(yt, x, x - xt)
        x_ref = oracle.smooth_lti(scaled(model, logq, logr), y, dt)
        ref, _ = oracle.grad_lti(model, y, dt, logq, logr, dLdx=x_ref - x_true)
    sm.close()
    assert_grad(g, ref, BTOL[prec])


def test_log_normaliser_flag_matches_oracle():
    from paper_2512_13319_gb300 import MapSmoother
    T, dt = 3000, 1e-3
    model, _, y = problem(T, dt, seed=61)
    sm = MapSmoother(model, T, dt, precision="fp64")
    yt = torch.tensor(y, device="cuda")
    x = sm.solve(yt)
    g = sm.grad(yt, x, logdet=True)
    ref, _ = oracle.grad_lti(model, y, dt, 0.0, 0.0, logdet=True)
    assert_grad(g, ref, 1e-8)


def test_log_normaliser_value():
    """The C ABI's log-normaliser is -T (log N(0; 0, dt Q) + log N(0; 0, R/dt))
    (scipy's Gaussian log density at its mean), and an update of (log q, log r)
    moves it by T/2 (nx d log q + ny d log r)."""
    from scipy.stats import multivariate_normal
    from paper_2512_13319_gb300 import MapSmoother
    T, dt = 1000, 1e-2
    model, _, _ = problem(T, dt, seed=63)
    sm = MapSmoother(model, T, dt, precision="fp64")
    C = dt * model.L @ model.W @ model.L.T
    Rd = model.R / dt
    ref = -T * (multivariate_normal(np.zeros(model.nx), C).logpdf(np.zeros(model.nx))
                + multivariate_normal(np.zeros(model.ny), Rd).logpdf(np.zeros(model.ny)))
    v0 = sm.log_normaliser()
    assert abs(v0 - ref) <= 1e-10 * abs(ref)
    sm.update(model.F, 0.3, -0.2)
    v1 = sm.log_normaliser()
    assert abs((v1 - v0) - 0.5 * T * (model.nx * 0.3 - model.ny * 0.2)) <= 1e-9 * abs(ref)
    sm.close()


def test_gradient_against_central_differences_on_the_gpu():
    """FP64 GPU solves at theta +- h (h = 1e-6) against the adjoint gradient."""
    from paper_2512_13319_gb300 import MapSmoother
    T, dt = 2000, 1e-3
    model, x_true, y = problem(T, dt, seed=71)
    sm = MapSmoother(model, T, dt, precision="fp64")
    yt = torch.tensor(y, device="cuda")
    xt = torch.tensor(x_true, device="cuda")
    F0, lq, lr = model.F.copy(), 0.1, -0.1

    def L(F, q, r):
        sm.update(F, q, r)
        x = sm.solve(yt)
        return 0.5 * float(((x - xt) ** 2).sum())

    sm.update(F0, lq, lr)
    x = sm.solve(yt)
    g = sm.grad(yt, x, x - xt)
    h = 1e-6
    fd = np.zeros(18)
    for a, b in [(0, 0), (1, 2), (3, 1), (2, 3)]:
        Fp = F0.copy(); Fp[a, b] += h
        Fm = F0.copy(); Fm[a, b] -= h
        fd[a * 4 + b] = (L(Fp, lq, lr) - L(Fm, lq, lr)) / (2 * h)
    fd[16] = (L(F0, lq + h, lr) - L(F0, lq - h, lr)) / (2 * h)
    fd[17] = (L(F0, lq, lr + h) - L(F0, lq, lr - h)) / (2 * h)
    idx = [0, 6, 13, 11, 16, 17]
    for i in idx:   # each entry: relative 1e-6 plus the FD rounding floor
        assert abs(g[i] - fd[i]) <= 1e-6 * abs(fd[i]) + 5e-8, (i, g[i], fd[i])
    sm.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_gradient_workload_T_2_18(prec):
    """OU nx=4 MAP-cost gradient at T = 2^18 against the FP64 oracle."""
    from paper_2512_13319_gb300 import MapSmoother
    T, dt = 2 ** 18, 1e-3
    model, _, y = problem(T, dt, seed=1004)
    sm = MapSmoother(model, T, dt, precision=prec)
    yt = torch.tensor(y, dtype=DT[prec], device="cuda")
    x = sm.solve(yt)
    g = sm.grad(yt, x)
    ref, _ = oracle.grad_lti(model, y, dt, 0.0, 0.0)
    sm.close()
    assert_grad(g, ref, BTOL[prec])


def test_autograd_function_matches_c_abi_gradient():
    from paper_2512_13319_gb300 import MapSmoother
    from paper_2512_13319_gb300.autograd import map_cost, map_solve
    T, dt = 4000, 1e-3
    model, x_true, y = problem(T, dt, seed=81)
    sm = MapSmoother(model, T, dt, precision="fp64")
    yt = torch.tensor(y, device="cuda")
    xt = torch.tensor(x_true, device="cuda")
    F = torch.tensor(model.F, requires_grad=True)
    lq = torch.tensor(0.2, dtype=torch.float64, requires_grad=True)
    lr = torch.tensor(-0.3, dtype=torch.float64, requires_grad=True)
    x = map_solve(sm, yt, F, lq, lr)
    loss = 0.5 * ((x - xt) ** 2).sum()
    loss.backward()
    ref, _ = oracle.grad_lti(model, y, dt, 0.2, -0.3, dLdx=x.detach().cpu().numpy() - x_true)
    got = np.concatenate([F.grad.numpy().ravel(), [lq.grad.item(), lr.grad.item()]])
    assert_grad(got, ref, 1e-8)
    F.grad = None
    c = map_cost(sm, yt, F, lq, lr)
    c.backward()
    ref_c, _ = oracle.grad_lti(model, y, dt, 0.2, -0.3)
    got_c = np.concatenate([F.grad.numpy().ravel(), [lq.grad.item() - got[16], lr.grad.item() - got[17]]])
    assert_grad(got_c, ref_c, 1e-8)
    sm.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_update_equals_fresh_handle(prec):
    """After update(F, log q, log r) the plan-time constants (set-up, folds,
    tile tables, products) are recomputed: the solve equals, bit for bit, the
    solve of a handle created with the updated model, and both match the
    oracle."""
    from paper_2512_13319_gb300 import MapSmoother
    T, dt = 300_000, 1e-3
    model, _, y = problem(T, dt, seed=81)
    rng = np.random.default_rng(82)
    F2 = model.F + 0.05 * rng.standard_normal(model.F.shape)
    lq, lr = 0.2, -0.3
    yt = torch.tensor(y, dtype=DT[prec], device="cuda")
    sm = MapSmoother(model, T, dt, precision=prec)
    sm.solve(yt)
    sm.update(F2, lq, lr)
    x1 = sm.solve(yt)
    m2 = scaled(model, lq, lr)
    m2.F = F2
    sm2 = MapSmoother(m2, T, dt, precision=prec)
    x2 = sm2.solve(yt)
    torch.cuda.synchronize()
    assert sm.geometry() == sm2.geometry()
    assert torch.equal(x1, x2)
    sm.close()
    sm2.close()
    tol = {"fp64": 1e-9, "fp32": 1e-4}[prec]
    xr = oracle.smooth_lti(m2, y, dt)
    xg = x1.cpu().numpy()
    assert rel(xg, xr) <= tol
    assert np.abs(xg - xr).max() / np.abs(xr).max() <= 10 * tol
