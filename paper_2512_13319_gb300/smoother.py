"""PyTorch-facing wrapper of the C ABI: device memory and streams come from torch.

Argument marshalling only; the solve runs in the CUDA library.
"""
from __future__ import annotations

import torch

from . import _binding as B

_PREC = {"fp32": B.MAP_FP32, "fp64": B.MAP_FP64}
_DISC = {"euler": B.MAP_EULER, "expm": B.MAP_EXPM, "auto": B.MAP_AUTO, "block": B.MAP_BLOCK_EULER,
         "exact": B.MAP_RICCATI_EXACT}
_SMOOTHER = {"rts": B.MAP_RTS, "two_filter": B.MAP_TWO_FILTER}


class MapSmoother:
    """One problem (model, T, dt, precision) with its device workspace.

    ``solve(y)`` takes observations ``y`` (T, ny) on the current CUDA device and
    returns the MAP trajectory (T+1, nx) in the handle's precision.
    """

    def __init__(self, model, T, dt, precision="fp32", discretisation="euler", smoother="rts",
                 gn_iters=1, cond_max=0.0, tile_threads=0, substeps=0, steps_per_thread=0):
        self.model, self.T, self.dt, self.smoother = model, int(T), float(dt), smoother
        self.dtype = torch.float32 if precision == "fp32" else torch.float64
        self.nx, self.ny = model.nx, model.ny
        desc, keep = B.make_desc(model, T, dt, _PREC[precision], _DISC[discretisation],
                                 _SMOOTHER[smoother], gn_iters, cond_max, tile_threads, substeps=substeps,
                                 steps_per_thread=steps_per_thread)
        self.substeps = (substeps or 10) if discretisation == "block" else 1
        self._h = B.map_smoother_create(desc)
        del keep

    def _stream(self, stream):
        s = stream if stream is not None else torch.cuda.current_stream()
        return ctypes_stream(s)

    def _check_dev(self, t, shape, name):
        if not (t.is_cuda and t.dtype == self.dtype and t.is_contiguous() and tuple(t.shape) == shape):
            raise ValueError(f"{name} must be a contiguous {self.dtype} CUDA tensor of shape {shape}")

    def solve(self, y, x_out=None, x_init=None, filt=False, cost=False, stream=None):
        """MAP trajectory for device observations ``y``.

        For nonlinear models ``x_init`` (T+1, nx) is the first linearisation
        trajectory.  Returns ``x`` or a tuple ``(x, filt, cost)`` when extras are asked.
        """
        self._check_dev(y, (self.T, self.ny), "y")
        if x_out is None:
            x_out = torch.empty((self.T + 1, self.nx), dtype=self.dtype, device=y.device)
        self._check_dev(x_out, (self.T + 1, self.nx), "x_out")
        if x_init is not None:
            x_out.copy_(x_init)
        f = None
        if filt:
            f = torch.empty((self.T + 1, self.nx + self.nx * (self.nx + 1) // 2), dtype=self.dtype,
                            device=y.device)
        c = B.map_smoother_solve(self._h, y.data_ptr(), x_out.data_ptr(),
                                 f.data_ptr() if f is not None else None, cost, self._stream(stream))
        if filt or cost:
            return x_out, f, c
        return x_out

    def dense(self, y, x, filt, out=None, stream=None):
        """States at every substep ((T substeps + 1, nx)) of a block-element solve
        from its observations, trajectory and filter output."""
        self._check_dev(y, (self.T, self.ny), "y")
        self._check_dev(x, (self.T + 1, self.nx), "x")
        self._check_dev(filt, (self.T + 1, self.nx + self.nx * (self.nx + 1) // 2), "filt")
        if out is None:
            out = torch.empty((self.T * self.substeps + 1, self.nx), dtype=self.dtype, device=y.device)
        self._check_dev(out, (self.T * self.substeps + 1, self.nx), "out")
        B.map_smoother_dense(self._h, y.data_ptr(), x.data_ptr(), filt.data_ptr(), out.data_ptr(),
                             self._stream(stream))
        return out

    def solve_sequential(self, y, x_out=None, x_init=None, stream=None):
        """Single-thread sequential baseline on the GPU (same elements, no scan)."""
        self._check_dev(y, (self.T, self.ny), "y")
        if x_out is None:
            x_out = torch.empty((self.T + 1, self.nx), dtype=self.dtype, device=y.device)
        if x_init is not None:
            x_out.copy_(x_init)
        B.map_smoother_solve_sequential(self._h, y.data_ptr(), x_out.data_ptr(), self._stream(stream))
        return x_out

    def solve_host(self, y_host, x_host=None, stream=None):
        """End-to-end solve from host memory (pinned CPU tensors) into host memory."""
        if x_host is None:
            x_host = torch.empty((self.T + 1, self.nx), dtype=self.dtype).pin_memory()
        B.map_smoother_solve_host(self._h, y_host.data_ptr(), x_host.data_ptr(), self._stream(stream))
        return x_host

    def grad(self, y, x, dLdx=None, logdet=False, stream=None):
        """dL/d(F, log q, log r) (numpy, nx*nx + 2) at the handle's parameters.

        ``dLdx=None`` differentiates the MAP cost itself; otherwise the loss
        whose gradient with respect to the trajectory ``x`` is ``dLdx``.
        """
        self._check_dev(y, (self.T, self.ny), "y")
        self._check_dev(x, (self.T + 1, self.nx), "x")
        if dLdx is not None:
            self._check_dev(dLdx, (self.T + 1, self.nx), "dLdx")
        return B.map_smoother_grad(self._h, y.data_ptr(), x.data_ptr(),
                                   dLdx.data_ptr() if dLdx is not None else None,
                                   self.nx * self.nx + 2, B.MAP_GRAD_LOGDET if logdet else 0,
                                   self._stream(stream))

    def log_normaliser(self):
        """T/2 log det(2 pi C) + T/2 log det(2 pi R/dt) at the current parameters
        (the constants the MAP cost of ``solve(cost=True)`` omits)."""
        return B.map_smoother_log_normaliser(self._h)

    def update(self, F=None, log_q=0.0, log_r=0.0):
        """Set theta = (F, log q, log r) (Q = e^log_q L W L^T, R = e^log_r R)."""
        B.map_smoother_update(self._h, F, log_q, log_r)

    def geometry(self):
        """(K steps per thread, B threads per tile, number of tiles)."""
        return B.map_smoother_geometry(self._h)

    def launches(self):
        """Kernels launched by the last solve (1: the single cooperative launch)."""
        return B.map_smoother_launches(self._h)

    def path(self):
        """How the last solve's scan ran: 1 single launch with per-step tables,
        2 single launch with per-step combines, 3 multi-kernel pipeline."""
        return B.map_smoother_solve_path(self._h)

    def profile(self, enable=True):
        """Record per-phase CUDA events in every solve (see phase_times)."""
        B.map_smoother_profile(self._h, enable)

    def phase_times(self):
        """{phase name: ms} of the last profiled solve."""
        names = B.PHASES_TWO_FILTER if self.smoother == "two_filter" else B.PHASES
        return dict(zip(names, B.map_smoother_phase_times(self._h)))

    def stats(self, reset=False, stream=None):
        """(combines recomputed in FP64, singular pivots, bulk copies whose bounded
        wait gave up) since create or the last reset."""
        return B.map_smoother_stats(self._h, reset, self._stream(stream))

    def wait_selftest(self, polls=1000, stream=None):
        """Run the bounded-wait self-test kernel: the handle's next checking
        call raises MapError(MAP_ERR_TIMEOUT)."""
        B.map_smoother_wait_selftest(self._h, polls, self._stream(stream))

    def close(self):
        if getattr(self, "_h", None):
            B.map_smoother_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ctypes_stream(s):
    return s.cuda_stream if hasattr(s, "cuda_stream") else s
