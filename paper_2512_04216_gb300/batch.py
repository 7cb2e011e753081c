"""Batch: many independent circuits in one persistent, graph-captured launch
(sv_batch_* in include/sv.h).  Every call is one library call."""
from __future__ import annotations

import numpy as np

from . import capi


class Batch:
    def __init__(self, circuits, n_qubits, shots, seeds, k_max=0, tile_qubits=0, keep_states=False,
                 stream=None, zmasks=None, irs=None):
        self.args = capi.BatchArgs(circuits, n_qubits, shots, seeds, zmasks, irs)
        self.opts = capi.make_opts(k_max, tile_qubits)
        self.h = capi.sv_batch_create(self.args, self.opts, keep_states, stream)

    def launch(self):
        capi.sv_batch_launch(self.h)

    def synchronize(self):
        capi.sv_batch_synchronize(self.h)

    def samples(self, i: int) -> np.ndarray:
        out = np.empty(int(self.args.shots[i]), dtype=np.uint64)
        capi.sv_batch_samples(self.h, i, out, False)
        return out

    def expectation(self, i: int):
        """(<Z_zmask>, norm) of circuit i."""
        return capi.sv_batch_expectation(self.h, i)

    def amplitudes(self, i: int) -> np.ndarray:
        out = np.empty(1 << int(self.args.n_qubits[i]), dtype=np.complex64)
        capi.sv_batch_amplitudes(self.h, i, out)
        return out

    def stats(self) -> dict:
        return capi.sv_batch_stats(self.h)

    def close(self):
        if getattr(self, "h", None) is not None:
            capi.sv_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
