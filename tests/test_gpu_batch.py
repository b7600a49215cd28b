"""Batched solve (one launch of the persistent kernel for every model and
trajectory, in a CUDA graph) against the FP64 oracle, trajectory by
trajectory."""
import numpy as np
import pytest

import oracle
from paper_2512_13319_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_13319_gb300 import build
    build.build()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def assert_traj(x, ref, tol, what=""):
    """Relative trajectory error within tol and no entry off by more than
    10 tol of the trajectory's largest entry."""
    assert x.shape == ref.shape and np.isfinite(x).all(), what
    e, m = rel(x, ref), float(np.abs(x - ref).max() / np.abs(ref).max())
    assert e <= tol and m <= 10 * tol, (what, e, m)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mixed_batch_matches_oracle_per_trajectory(prec):
    from paper_2512_13319_gb300.batch import MapBatch
    rng = np.random.default_rng(5)
    lengths = np.concatenate([[1, 2, 3, 15, 16, 17, 2047, 2048, 2049],
                              rng.integers(1, 3000, size=21)])
    dims = rng.choice([1, 2, 3], size=len(lengths))
    dt = 0.01
    models, lengths, model_of, ys = synth.batched_workload(lengths=lengths, dims=dims, dt=dt, seed=7)
    mb = MapBatch(models, lengths, model_of, [dt] * 3, precision=prec)
    ydev = mb.pack_observations(ys)
    xdev = mb.empty_outputs()
    mb.solve(ydev, xdev)
    torch.cuda.synchronize()
    xs = mb.unpack_states(xdev)
    for j in range(len(lengths)):
        ref = oracle.smooth_lti(models[model_of[j]], ys[j], dt)
        assert_traj(xs[j], ref, TOL[prec], (j, lengths[j], dims[j]))
    # the persistent kernel over every model's step tables, with an autotuned
    # (steps per thread, threads per CTA) shared by all models
    assert mb.persistent()
    tun = {mb.tuning(m) for m in range(3)}
    assert len(tun) == 1
    K, B = tun.pop()
    assert K in (8, 12, 16) and B in (64, 128)
    # graph replay and re-capture on new arrays give the same states
    first = [x.clone() for x in xdev]
    mb.solve(ydev, xdev)
    xdev2 = mb.empty_outputs()
    mb.solve(ydev, xdev2)
    torch.cuda.synchronize()
    for a, b, c in zip(first, xdev, xdev2):
        assert torch.equal(a, b) and torch.equal(a, c)
    mb.close()


def test_single_model_single_trajectory_batch_equals_plain_solve():
    from paper_2512_13319_gb300 import MapSmoother
    from paper_2512_13319_gb300.batch import MapBatch
    model = synth.wiener_velocity(2)
    dt, T = 0.01, 5000
    _, y = synth.simulate(model, T, dt, seed=3)
    mb = MapBatch([model], [T], [0], [dt], precision="fp64")
    ydev = mb.pack_observations([y])
    xdev = mb.empty_outputs()
    mb.solve(ydev, xdev)
    sm = MapSmoother(model, T, dt, precision="fp64")
    x = sm.solve(torch.tensor(y, device="cuda"))
    assert_traj(xdev[0].cpu().numpy(), x.cpu().numpy(), 1e-12)
    assert_traj(xdev[0].cpu().numpy(), oracle.smooth_lti(model, y, dt), 1e-9)
    mb.close()
    sm.close()


def test_full_batch_4096_trajectories_sampled():
    """The benchmark batch: 4096 trajectories, lengths log-uniform in [256, 65536],
    nx in {2, 4, 6}; a sample of 40 trajectories compared with the oracle."""
    from paper_2512_13319_gb300.batch import MapBatch
    dt = 0.01
    models, lengths, model_of, ys = synth.batched_workload()
    mb = MapBatch(models, lengths, model_of, [dt] * 3, precision="fp32")
    ydev = mb.pack_observations(ys)
    xdev = mb.empty_outputs()
    mb.solve(ydev, xdev)
    torch.cuda.synchronize()
    xs = mb.unpack_states(xdev)
    rng = np.random.default_rng(0)
    sample = np.concatenate([[0, len(lengths) - 1, int(np.argmax(lengths)), int(np.argmin(lengths))],
                             rng.choice(len(lengths), size=36, replace=False)])
    for j in sample:
        ref = oracle.smooth_lti(models[model_of[j]], ys[j], dt)
        assert_traj(xs[j], ref, TOL["fp32"], (j, lengths[j]))
    mb.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_every_state_shape_matches_oracle(prec):
    """One batch over every (nx, ny) the batch kernel is built for: OU models
    with (3, 1) and (5, 2) beside Wiener velocity (2, 1), (4, 2) and (6, 3),
    ragged lengths across several blocks of the kernel and a block boundary
    +- 1, each trajectory against the oracle."""
    from paper_2512_13319_gb300.batch import MapBatch
    dt = 0.01
    models = [synth.wiener_velocity(1), synth.ou_model(3, 1, seed=11), synth.wiener_velocity(2),
              synth.ou_model(5, 2, seed=12), synth.wiener_velocity(3)]
    rng = np.random.default_rng(21)
    lengths = np.concatenate([[1, 5, 1535, 1536, 1537, 3072, 4097, 9000],
                              rng.integers(1, 6000, size=12)]).astype(np.int64)
    model_of = np.arange(len(lengths)) % len(models)
    ys = []
    for j, L in enumerate(lengths):
        _, y = synth.simulate(models[model_of[j]], int(L), dt, seed=300 + j, substeps=1)
        ys.append(y)
    mb = MapBatch(models, lengths, model_of, [dt] * len(models), precision=prec)
    ydev = mb.pack_observations(ys)
    xdev = mb.empty_outputs()
    mb.solve(ydev, xdev)
    torch.cuda.synchronize()
    xs = mb.unpack_states(xdev)
    for j in range(len(lengths)):
        ref = oracle.smooth_lti(models[model_of[j]], ys[j], dt)
        assert_traj(xs[j], ref, TOL[prec], (j, int(lengths[j]), models[model_of[j]].nx))
    mb.close()
