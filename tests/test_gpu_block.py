"""Parity of the block-element and exact-element solves and of the dense output
(Section 5.1, Eq. 36-37, Section 4.3) on the GPU with the FP64 oracle.

Same tolerances as the per-step solves (relative trajectory error 1e-9 FP64,
1e-4 FP32, and no entry off by more than 10x that of the trajectory scale):
the block and exact elements are built once per handle in FP64 and the solve
is the per-step RTS scan with offsets that depend on the held sample.
"""
import numpy as np
import pytest

import oracle
from paper_2512_13319_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32": 1e-4}
DT = {"fp64": torch.float64, "fp32": torch.float32}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_13319_gb300 import build
    build.build()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def assert_traj(x, ref, tol):
    assert x.shape == ref.shape
    assert np.isfinite(x).all()
    e = rel(x, ref)
    m = float(np.abs(x - ref).max() / np.abs(ref).max())
    assert e <= tol, f"relative trajectory error {e:.3e} > {tol:.0e}"
    assert m <= 10 * tol, f"largest entry error {m:.3e} > {10 * tol:.0e} of the trajectory scale"


def model_with_offsets(n=4, m=2, seed=5):
    mod = synth.ou_model(n, m, seed=seed)
    rng = np.random.default_rng(seed)
    mod.c = rng.uniform(-0.3, 0.3, n)
    mod.r = rng.uniform(-0.2, 0.2, m)
    mod.m0 = rng.uniform(-0.5, 0.5, n)
    return mod


def smoother(model, T, dt, prec, disc, **kw):
    from paper_2512_13319_gb300 import MapSmoother
    return MapSmoother(model, T, dt, precision=prec, discretisation=disc, **kw)


def solve(model, y, dt, prec, disc, filt=False, sequential=False, **kw):
    sm = smoother(model, y.shape[0], dt, prec, disc, **kw)
    yt = torch.tensor(y, dtype=DT[prec], device="cuda")
    if sequential:
        x = sm.solve_sequential(yt)
        f = None
    else:
        x, f, _ = sm.solve(yt, filt=True)
    st = sm.stats()
    out = (sm, yt, x, f) if filt else x.cpu().numpy()
    if not filt:
        sm.close()
    assert st[1] == 0
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("T", [1, 2, 7, 511, 2049, 20_000])
def test_block_elements_ragged(prec, T):
    m = model_with_offsets(seed=T % 97)
    dt = 0.02
    _, y = synth.simulate(m, T, dt, seed=T)
    x = solve(m, y, dt, prec, "block", substeps=10)
    assert_traj(x, oracle.smooth_block(m, y, dt, 10), TOL[prec])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("nsub", [1, 2, 7, 64])
def test_block_substep_counts(prec, nsub):
    m = model_with_offsets(seed=21)
    T, dt = 3000, 0.05
    _, y = synth.simulate(m, T, dt, seed=22)
    x = solve(m, y, dt, prec, "block", substeps=nsub)
    assert_traj(x, oracle.smooth_block(m, y, dt, nsub), TOL[prec])


def test_one_substep_block_is_the_euler_solve():
    m = model_with_offsets(seed=23)
    T, dt = 4000, 0.02
    _, y = synth.simulate(m, T, dt, seed=24)
    xb = solve(m, y, dt, "fp64", "block", substeps=1)
    xe = solve(m, y, dt, "fp64", "euler")
    assert rel(xb, xe) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", [(2, 1), (3, 1), (5, 2), (6, 3)])
def test_block_and_exact_state_dimensions(prec, shape):
    n, mm = shape
    m = model_with_offsets(n, mm, seed=31 + n)
    T, dt = 5000, 0.03
    _, y = synth.simulate(m, T, dt, seed=32 + n)
    assert_traj(solve(m, y, dt, prec, "block", substeps=5), oracle.smooth_block(m, y, dt, 5), TOL[prec])
    assert_traj(solve(m, y, dt, prec, "exact"), oracle.smooth_exact(m, y, dt), TOL[prec])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("T", [1, 3, 1000, 30_001])
def test_exact_elements(prec, T):
    m = model_with_offsets(seed=41)
    dt = 0.1
    _, y = synth.simulate(m, T, dt, seed=42)
    assert_traj(solve(m, y, dt, prec, "exact"), oracle.smooth_exact(m, y, dt), TOL[prec])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_exact_on_wiener_velocity(prec):
    m = synth.wiener_velocity(2, q=1.0, r=0.1)
    T, dt = 10_000, 0.01
    _, y = synth.simulate(m, T, dt, seed=43)
    assert_traj(solve(m, y, dt, prec, "exact"), oracle.smooth_exact(m, y, dt), TOL[prec])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("T,nsub", [(1, 10), (5, 3), (2000, 10), (4099, 64)])
def test_dense_output(prec, T, nsub):
    m = model_with_offsets(seed=51)
    dt = 0.02
    _, y = synth.simulate(m, T, dt, seed=52)
    sm, yt, x, f = solve(m, y, dt, prec, "block", filt=True, substeps=nsub)
    xd = sm.dense(yt, x, f).cpu().numpy()
    sm.close()
    ref = oracle.dense_block(m, y, dt, nsub)
    assert_traj(xd, ref, TOL[prec])
    # the grid rows are the trajectory itself
    assert np.array_equal(xd[::nsub], x.cpu().numpy())


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("disc", ["block", "exact"])
def test_tiled_scan_and_general_path(prec, disc):
    """A, C and J of block and exact elements are the same for every interval:
    the solve takes the tiled scan with per-step tables and the sample's share
    of the offset (path 1); with per-phase events it takes the general
    combine path.  Both against the oracle, and the filter output of the
    tiled scan against the oracle's filter means."""
    m = model_with_offsets(seed=91)
    T, dt = 30_000, 0.01
    _, y = synth.simulate(m, T, dt, seed=92)
    ref, mf, _ = (oracle.smooth_block(m, y, dt, 10, return_filter=True) if disc == "block"
                  else oracle.smooth_exact(m, y, dt, return_filter=True))
    sm = smoother(m, T, dt, prec, disc, substeps=10)
    yt = torch.tensor(y, dtype=DT[prec], device="cuda")
    x, f, _ = sm.solve(yt, filt=True)
    assert sm.path() == 1
    sm.profile(True)
    xg = sm.solve(yt).cpu().numpy()
    assert sm.path() == 3
    st = sm.stats()
    assert st[1] == 0 and st[2] == 0
    sm.close()
    assert_traj(x.cpu().numpy(), ref, TOL[prec])
    assert_traj(xg, ref, TOL[prec] if prec == "fp64" else 5e-4)
    f = f.cpu().numpy().astype(np.float64)
    n = 4
    iu = np.triu_indices(n)
    for k in (0, 1, T // 3, T):
        S = np.zeros((n, n))
        S[iu] = f[k, n:]
        S = S + S.T - np.diag(np.diag(S))
        mk = np.linalg.solve(S, f[k, :n])
        assert np.abs(mk - mf[k]).max() <= 100 * TOL[prec] * max(1.0, np.abs(mf[k]).max())


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sequential_block_baseline(prec):
    m = model_with_offsets(seed=61)
    T, dt = 3000, 0.02
    _, y = synth.simulate(m, T, dt, seed=62)
    tol = TOL[prec] if prec == "fp64" else 5e-4
    assert_traj(solve(m, y, dt, prec, "block", sequential=True, substeps=10),
                oracle.smooth_block(m, y, dt, 10), tol)
    assert_traj(solve(m, y, dt, prec, "exact", sequential=True), oracle.smooth_exact(m, y, dt), tol)


def test_block_full_size_T_2_20_fp32():
    """The bench workload's length: T = 2^20 intervals of 10 substeps, and the
    dense output at all 10 T + 1 substep times, against the oracle."""
    m = synth.ou_model(4, 2, seed=71)
    T, dt, nsub = 1 << 20, 0.01, 10
    _, y = synth.simulate(m, T, dt, seed=72)
    sm, yt, x, f = solve(m, y, dt, "fp32", "block", filt=True, substeps=nsub)
    xd = sm.dense(yt, x, f).cpu().numpy()
    assert sm.path() == 1
    sm.close()
    assert_traj(x.cpu().numpy(), oracle.smooth_block(m, y, dt, nsub), TOL["fp32"])
    assert_traj(xd, oracle.dense_block(m, y, dt, nsub), TOL["fp32"])


def test_block_and_exact_argument_checks():
    from paper_2512_13319_gb300 import MapSmoother
    from paper_2512_13319_gb300._binding import MapError
    m = model_with_offsets(seed=81)
    with pytest.raises(MapError):
        MapSmoother(m, 100, 0.01, discretisation="block", substeps=65)
    with pytest.raises(MapError):
        MapSmoother(m, 100, 0.01, discretisation="block", smoother="two_filter")
    with pytest.raises(MapError):
        MapSmoother(synth.ou_model(8, 4, seed=1), 100, 0.01, discretisation="exact")
    ct = synth.coordinated_turn()
    with pytest.raises(MapError):
        MapSmoother(ct, 100, 0.01, discretisation="block")
    # dense output needs block elements
    sm = MapSmoother(m, 100, 0.01, discretisation="euler")
    _, y = synth.simulate(m, 100, 0.01, seed=82)
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    x, f, _ = sm.solve(yt, filt=True)
    with pytest.raises(MapError):
        sm.dense(yt, x, f, out=torch.empty((101, 4), device="cuda"))
    sm.close()
