"""PyTorch-facing wrapper of the batch C ABI (map_batch_*): marshalling only."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _binding as B


class MapBatch:
    """Independent trajectories of a few linear models: one launch of the
    persistent batch kernel for all of them, or per model one scan with reset
    elements (see include/map_smoother.h, map_batch_create)."""

    def __init__(self, models, lengths, model_of, dts, precision="fp32"):
        self.models = list(models)
        self.lengths = np.asarray(lengths, dtype=np.int64)
        self.model_of = np.asarray(model_of, dtype=np.int32)
        self.dtype = torch.float32 if precision == "fp32" else torch.float64
        prec = B.MAP_FP32 if precision == "fp32" else B.MAP_FP64
        descs = (B.map_problem_desc * len(self.models))()
        self._keep = []
        for i, (m, dt) in enumerate(zip(self.models, dts)):
            d, keep = B.make_desc(m, 1, dt, prec)
            descs[i] = d
            self._keep.append(keep)
        h = ctypes.c_void_p()
        lib = B.load()
        st = lib.map_batch_create(ctypes.byref(h), descs, len(self.models),
                                  self.lengths.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                  self.model_of.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                  len(self.lengths))
        if st != B.MAP_OK:
            raise B.MapError(st, lib.map_batch_last_error(None).decode())
        self._h = h.value
        self.rows = []
        for i in range(len(self.models)):
            yr, xr = ctypes.c_int64(), ctypes.c_int64()
            lib.map_batch_rows(self._h, i, ctypes.byref(yr), ctypes.byref(xr))
            self.rows.append((yr.value, xr.value))

    def pack_observations(self, ys):
        """Host list of per-trajectory y (T_j, ny) -> per-model device arrays with
        one unused row between consecutive trajectories."""
        out = []
        for i, m in enumerate(self.models):
            idx = np.nonzero(self.model_of == i)[0]
            if len(idx) == 0:
                out.append(None)
                continue
            parts = []
            for c, j in enumerate(idx):
                if c > 0:
                    parts.append(np.zeros((1, m.ny)))
                parts.append(np.asarray(ys[j]))
            arr = np.concatenate(parts, axis=0)
            assert arr.shape[0] == self.rows[i][0]
            out.append(torch.tensor(arr, dtype=self.dtype, device="cuda"))
        return out

    def unpack_states(self, xs):
        """Per-model device outputs -> host list of per-trajectory x (T_j + 1, nx)."""
        res = [None] * len(self.lengths)
        for i in range(len(self.models)):
            if xs[i] is None:
                continue
            arr = xs[i].cpu().numpy()
            o = 0
            for j in np.nonzero(self.model_of == i)[0]:
                n = int(self.lengths[j]) + 1
                res[j] = arr[o:o + n]
                o += n
        return res

    def empty_outputs(self):
        return [None if self.rows[i][1] == 0 else
                torch.empty((self.rows[i][1], m.nx), dtype=self.dtype, device="cuda")
                for i, m in enumerate(self.models)]

    def solve(self, ys, xs, stream=None):
        n = len(self.models)
        yp = (ctypes.c_void_p * n)(*[0 if t is None else t.data_ptr() for t in ys])
        xp = (ctypes.c_void_p * n)(*[0 if t is None else t.data_ptr() for t in xs])
        s = stream if stream is not None else torch.cuda.current_stream()
        lib = B.load()
        st = lib.map_batch_solve(self._h, yp, xp, s.cuda_stream)
        if st != B.MAP_OK:
            raise B.MapError(st, lib.map_batch_last_error(self._h).decode())
        return xs

    def tuning(self, model):
        K, Bt = ctypes.c_int(), ctypes.c_int()
        B.load().map_batch_tuning(self._h, model, ctypes.byref(K), ctypes.byref(Bt))
        return K.value, Bt.value

    def persistent(self):
        """True when the batch runs as one launch of the persistent kernel."""
        return bool(B.load().map_batch_persistent(self._h))

    def close(self):
        if getattr(self, "_h", None):
            B.load().map_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
