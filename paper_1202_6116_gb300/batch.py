"""Many films advanced together through the batch entry points of the C ABI.

Every batch step is one CUDA graph launch that holds each film's whole time
step as an independent branch, with the electrode voltage ramps applied
before and the polarization-voltage loops recorded after (``pf_batch_*``).
PyTorch supplies the device memory; all computation runs in the CUDA library.
"""
from __future__ import annotations

import numpy as np
import torch

from . import pf
from .film import Film


class Batch:
    """A batch over existing films (which must share one CUDA stream)."""

    def __init__(self, films: list[Film], max_records: int, record_every: int = 1):
        if not films:
            raise ValueError("need at least one film")
        self.films = list(films)
        self.nfilms = len(films)
        self.max_records = int(max_records)
        nbytes = pf.pf_batch_workspace_bytes(self.nfilms, self.max_records)
        if nbytes == 0:
            raise ValueError("invalid batch size")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=films[0].P.device)
        self.handle = pf.pf_batch_create([f.ctx for f in films], self.workspace, nbytes, self.max_records,
                                         record_every)

    def set_ramp(self, film: int, face: int, amplitude: float, period: float):
        pf.pf_batch_set_ramp(self.handle, film, face, amplitude, period)

    def step(self, nsteps: int = 1, ok=(pf.PF_OK,)):
        st, info = pf.pf_batch_step(self.handle, nsteps, ok)
        return st, info.as_dict()

    def film_info(self, film: int) -> dict:
        return pf.pf_batch_film_info(self.handle, film).as_dict()

    def loops(self) -> np.ndarray:
        """Loop records as an array (records, films, 4): ramp voltage, mean
        P_x, P_y, P_z after the recorded step."""
        out = np.zeros(max(1, self.max_records) * self.nfilms * 4)
        n = pf.pf_batch_read_loops(self.handle, out, self.max_records)
        n = min(n, self.max_records)
        return out[: n * self.nfilms * 4].reshape(n, self.nfilms, 4)

    def close(self):
        if getattr(self, "handle", None):
            pf.pf_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
