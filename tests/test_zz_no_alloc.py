"""The allocation-free entry point (map_smoother_solve_noalloc) agrees with the
allocating one (map_smoother_create + map_smoother_solve) and with the oracle.

It serves callers that cannot call cudaMalloc (fixed device-memory budgets:
real-time loops, embedded services, plug-ins whose host owns the allocator);
its workspace is a __device__ array of the library.  Called through the C ABI
twice in a row, since every call shares that array, and the second call must
leave the device's free memory unchanged.  This file is collected last so
that a run that stops at the first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2512_13319_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-4, "fp64": 1e-9}
# largest horizon of the 64 MiB scratch at nx = 4, ny = 2 (see the header)
MAX_T = {"fp32": 632_832, "fp64": 329_728}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_13319_gb300 import _binding, build
    build.build()
    return _binding.load()


def check(x, ref, tol):
    assert np.isfinite(x).all()
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= tol
    assert np.abs(x - ref).max() / np.abs(ref).max() <= 10 * tol


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_noalloc_matches_allocating_solve_on_two_calls(lib, prec):
    from paper_2512_13319_gb300 import MapSmoother
    from paper_2512_13319_gb300 import _binding as B
    dtype = torch.float32 if prec == "fp32" else torch.float64
    model = synth.wiener_velocity(2, q=1.0, r=0.1)
    T, dt = 100_003, 1e-3
    _, y = synth.simulate(model, T, dt, seed=77, substeps=1)
    x_or = oracle.smooth_lti(model, y, dt)
    yt = torch.tensor(y, dtype=dtype, device="cuda")
    sm = MapSmoother(model, T, dt, precision=prec)
    x_ref = sm.solve(yt).cpu().numpy()
    sm.close()
    desc, keep = B.make_desc(model, T, dt, B.MAP_FP32 if prec == "fp32" else B.MAP_FP64)
    stream = torch.cuda.current_stream().cuda_stream
    outs = [torch.full((T + 1, 4), float("nan"), dtype=dtype, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    free = []
    for x in outs:
        free.append(torch.cuda.mem_get_info()[0])
        status = lib.map_smoother_solve_noalloc(ctypes.byref(desc), yt.data_ptr(), x.data_ptr(), stream)
        assert status == B.MAP_OK, lib.map_smoother_last_error(None)
        torch.cuda.synchronize()
        xn = x.cpu().numpy()
        check(xn, x_ref, TOL[prec])
        check(xn, x_or, TOL[prec])
    free.append(torch.cuda.mem_get_info()[0])
    # the second call (module and kernels already loaded by the first) allocates nothing
    assert free[2] == free[1], free
    assert torch.equal(outs[0], outs[1])


def test_noalloc_horizon_limit(lib):
    """The largest horizon the scratch holds solves; one interval more is
    rejected with MAP_ERR_SHAPE and a message naming the bytes needed."""
    from paper_2512_13319_gb300 import _binding as B
    model = synth.wiener_velocity(2)
    dt = 1e-3
    T = MAX_T["fp32"]
    _, y = synth.simulate(model, T, dt, seed=78, substeps=1)
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    x = torch.empty((T + 1, 4), dtype=torch.float32, device="cuda")
    desc, keep = B.make_desc(model, T, dt, B.MAP_FP32)
    status = lib.map_smoother_solve_noalloc(ctypes.byref(desc), yt.data_ptr(), x.data_ptr(), None)
    assert status == B.MAP_OK, lib.map_smoother_last_error(None)
    torch.cuda.synchronize()
    check(x.cpu().numpy(), oracle.smooth_lti(model, y, dt), TOL["fp32"])
    for prec, flag in (("fp32", B.MAP_FP32), ("fp64", B.MAP_FP64)):
        desc, keep = B.make_desc(model, MAX_T[prec] + 1, dt, flag)
        status = lib.map_smoother_solve_noalloc(ctypes.byref(desc), yt.data_ptr(), x.data_ptr(), None)
        assert status == B.MAP_ERR_SHAPE
        assert b"too large" in lib.map_smoother_last_error(None)
