"""Timing helper for the sequential GPU baseline (map_smoother_solve_sequential)."""
from __future__ import annotations

import statistics


def time_sequential(model, y, dt, dtype, dev, flush, stream, runs=3):
    """Median device time of the one-thread sequential solve on the same workload."""
    import torch

    from .smoother import MapSmoother
    prec = "fp32" if dtype == torch.float32 else "fp64"
    T = y.shape[0]
    sm = MapSmoother(model, T, dt, precision=prec)
    x = torch.empty((T + 1, model.nx), dtype=dtype, device=dev)
    sm.solve_sequential(y, x_out=x)
    times = []
    for _ in range(runs):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sm.solve_sequential(y, x_out=x)
        b.record(stream)
        torch.cuda.synchronize(dev)
        times.append(a.elapsed_time(b))
    sm.close()
    ms = statistics.median(times)
    return {"value": T / (ms * 1e-3), "unit": "time-steps/s", "ms_per_step": ms,
            "kind": "one GPU thread, same elements, no scan", "precision": prec}
