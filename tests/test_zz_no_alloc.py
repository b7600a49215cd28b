"""The allocation-free entry point (map_smoother_solve_noalloc) agrees with the
allocating one (map_smoother_create + map_smoother_solve).

It serves callers that cannot call cudaMalloc (fixed device-memory budgets:
real-time loops, embedded services, plug-ins whose host owns the allocator);
its workspace is a __device__ array of the library.  Called through the C ABI
twice in a row, since every call shares that array.  This file is collected
last so that a run that stops at the first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest

from paper_2512_13319_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-4, "fp64": 1e-9}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_13319_gb300 import _binding, build
    build.build()
    return _binding.load()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_noalloc_matches_allocating_solve_on_two_calls(lib, prec):
    from paper_2512_13319_gb300 import MapSmoother
    from paper_2512_13319_gb300 import _binding as B
    dtype = torch.float32 if prec == "fp32" else torch.float64
    model = synth.wiener_velocity(2, q=1.0, r=0.1)
    T, dt = 100_003, 1e-3
    _, y = synth.simulate(model, T, dt, seed=77, substeps=1)
    yt = torch.tensor(y, dtype=dtype, device="cuda")
    sm = MapSmoother(model, T, dt, precision=prec)
    x_ref = sm.solve(yt).cpu().numpy()
    sm.close()
    desc, keep = B.make_desc(model, T, dt, B.MAP_FP32 if prec == "fp32" else B.MAP_FP64)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        x = torch.full((T + 1, 4), float("nan"), dtype=dtype, device="cuda")
        status = lib.map_smoother_solve_noalloc(ctypes.byref(desc), yt.data_ptr(), x.data_ptr(), stream)
        assert status == B.MAP_OK, lib.map_smoother_last_error(None)
        torch.cuda.synchronize()
        xn = x.cpu().numpy()
        assert np.linalg.norm(xn - x_ref) / np.linalg.norm(x_ref) <= TOL[prec]


def test_noalloc_rejects_horizons_beyond_its_scratch(lib):
    from paper_2512_13319_gb300 import _binding as B
    model = synth.wiener_velocity(2)
    T = 4_000_000
    desc, keep = B.make_desc(model, T, 1e-3, B.MAP_FP32)
    y = torch.zeros((8, 2), device="cuda")
    x = torch.zeros((8, 4), device="cuda")
    status = lib.map_smoother_solve_noalloc(ctypes.byref(desc), y.data_ptr(), x.data_ptr(), None)
    assert status == B.MAP_ERR_SHAPE
    assert b"too large" in lib.map_smoother_last_error(None)
