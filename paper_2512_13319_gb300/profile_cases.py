"""Small self-contained workloads for profiling one kernel of the library.

    python -m paper_2512_13319_gb300.profile_cases scan    # k_lti_scan: Wiener velocity nx=4, T=2^20, FP32
    python -m paper_2512_13319_gb300.profile_cases batch   # k_batch_*: the 4096-trajectory batch, FP32
    python -m paper_2512_13319_gb300.profile_cases gn      # general path: coordinated-turn GN, T=2^16, FP32
    python -m paper_2512_13319_gb300.profile_cases plan    # plan kernels: OU nx=4, T=2^18, update + solve

Each case builds its inputs, runs a few solves and synchronises, so that a
profiler capture filtered to one kernel (ncu -k ... -s ... -c ...) sees only a
few launches before the captured one and holds at most a few GB on the device.
"""
from __future__ import annotations

import sys

import numpy as np
import torch

from . import MapSmoother, synth


def scan(reps=4):
    T, dt = 2 ** 20, 1e-3
    model = synth.wiener_velocity(2, q=1.0, r=0.1)
    _, y = synth.simulate(model, T, dt, seed=1001, substeps=1)
    sm = MapSmoother(model, T, dt, precision="fp32")
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    x = torch.empty((T + 1, 4), dtype=torch.float32, device="cuda")
    for _ in range(reps):
        sm.solve(yt, x_out=x)
    torch.cuda.synchronize()
    print("scan: path", sm.path(), "geometry", sm.geometry())
    sm.close()


def batch(reps=3):
    from .batch import MapBatch
    models, lengths, model_of, ys = synth.batched_workload()
    mb = MapBatch(models, lengths, model_of, [0.01] * len(models), precision="fp32")
    yd = mb.pack_observations(ys)
    xd = mb.empty_outputs()
    for _ in range(reps):
        mb.solve(yd, xd)
    torch.cuda.synchronize()
    print("batch: tuning", [mb.tuning(i) for i in range(len(models))])
    mb.close()


def gn(reps=2):
    model = synth.coordinated_turn()
    T, iters, dt = 2 ** 16, 10, 1e-3
    _, y = synth.simulate(model, T, dt, seed=1002)
    x0 = np.tile(model.m0, (T + 1, 1))
    sm = MapSmoother(model, T, dt, precision="fp32", gn_iters=iters)
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    xi = torch.tensor(x0, dtype=torch.float32, device="cuda")
    x = torch.empty_like(xi)
    for _ in range(reps):
        sm.solve(yt, x_out=x, x_init=xi)
    torch.cuda.synchronize()
    print("gn: geometry", sm.geometry(), "launches", sm.launches())
    sm.close()


def plan(reps=2):
    T, dt = 2 ** 18, 1e-3
    model = synth.ou_model(4, 2, seed=51)
    _, y = synth.simulate(model, T, dt, seed=1004, substeps=1)
    sm = MapSmoother(model, T, dt, precision="fp32")
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    x = sm.solve(yt)
    for _ in range(reps):
        sm.update(F=model.F, log_q=0.0, log_r=0.0)
        sm.solve(yt, x_out=x)
    torch.cuda.synchronize()
    print("plan: path", sm.path())
    sm.close()


CASES = {"scan": scan, "batch": batch, "gn": gn, "plan": plan}

if __name__ == "__main__":
    if len(sys.argv) != 2 or sys.argv[1] not in CASES:
        sys.exit("usage: python -m paper_2512_13319_gb300.profile_cases " + "|".join(CASES))
    CASES[sys.argv[1]]()
