"""StateVector: a resident 2^n complex64 state in a torch CUDA tensor, driven
through the C-ABI (every operation is one library call)."""
from __future__ import annotations

import numpy as np
import torch

from . import capi


class StateVector:
    """Owns a torch complex64 tensor of 2^n amplitudes wrapped by sv_wrap.

    ``stream``: a torch.cuda.Stream (default: the current stream at creation).
    """

    def __init__(self, n: int, stream: torch.cuda.Stream | None = None, device=None,
                 basis_index: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("StateVector needs a CUDA device")
        self.n = int(n)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        with torch.cuda.device(self.device):
            self.amps = torch.empty(1 << self.n, dtype=torch.complex64, device=self.device)
            self.h = capi.sv_wrap(self.amps, self.n, capi.SV_C64, self.stream)
            capi.sv_reset(self.h, basis_index)

    # -- lifetime -------------------------------------------------------------
    def close(self):
        if getattr(self, "h", None) is not None:
            capi.sv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- operations -------------------------------------------------------------
    def reset(self, basis_index: int = 0):
        capi.sv_reset(self.h, basis_index)

    def apply(self, circuit, k_max=0, tile_qubits=0, low_qubits=0, precision=0, kernel_variant=0):
        ir, keep = capi.to_ir(circuit)
        opts = capi.make_opts(k_max, tile_qubits, low_qubits, precision, kernel_variant)
        capi.sv_apply_circuit(self.h, ir, len(circuit), opts)
        del keep

    def synchronize(self):
        capi.sv_synchronize(self.h)

    def norm2(self) -> float:
        return capi.sv_norm(self.h)

    def expect_z(self, zmask: int) -> float:
        return capi.sv_expect_pauli(self.h, 0, zmask)

    def sample(self, shots: int, seed: int, on_device: bool = False):
        if on_device:
            out = torch.empty(shots, dtype=torch.int64, device=self.device)
        else:
            out = np.empty(shots, dtype=np.uint64)
        capi.sv_sample(self.h, shots, seed, out, on_device)
        return out

    def sample_uniforms(self, uniforms, on_device: bool = False):
        if on_device:
            u = uniforms if torch.is_tensor(uniforms) else torch.as_tensor(uniforms, device=self.device)
            out = torch.empty(u.shape[0], dtype=torch.int64, device=self.device)
        else:
            u = np.ascontiguousarray(uniforms, dtype=np.float64)
            out = np.empty(u.shape[0], dtype=np.uint64)
        nb = capi.sv_sample_uniforms(self.h, u, u.shape[0], out, on_device)
        return out, nb

    def sample_expect_z(self, uniforms, z_mask: int):
        """Draws for the uniforms, <Z_mask> and ||psi||^2 from one read of the state:
        (bitstrings, n_boundary, expectation, norm2)."""
        u = np.ascontiguousarray(uniforms, dtype=np.float64)
        out = np.empty(u.shape[0], dtype=np.uint64)
        nb, e, n2 = capi.sv_sample_expect_z(self.h, u, u.shape[0], out, False, z_mask)
        return out, nb, e, n2

    def alias_build(self):
        """Snapshot the outcome distribution into a Walker alias table (synchronises)."""
        capi.sv_alias_build(self.h)

    def sample_alias(self, shots: int, seed: int, on_device: bool = False):
        """Draws from the last alias table, uniforms from seed (SplitMix64, as sample())."""
        if on_device:
            out = torch.empty(shots, dtype=torch.int64, device=self.device)
        else:
            out = np.empty(shots, dtype=np.uint64)
        capi.sv_alias_sample(self.h, shots, seed, out, on_device)
        return out

    def sample_alias_uniforms(self, uniforms, on_device: bool = False):
        if on_device:
            u = uniforms if torch.is_tensor(uniforms) else torch.as_tensor(uniforms, device=self.device)
            out = torch.empty(u.shape[0], dtype=torch.int64, device=self.device)
        else:
            u = np.ascontiguousarray(uniforms, dtype=np.float64)
            out = np.empty(u.shape[0], dtype=np.uint64)
        capi.sv_alias_sample_uniforms(self.h, u, u.shape[0], out, on_device)
        return out

    def alias_table(self, offset: int = 0, count: int | None = None):
        """(own uint32[count], alias uint32[count]) of the last alias table."""
        count = (1 << self.n) - offset if count is None else count
        raw = np.empty(count, dtype=np.uint64)
        capi.sv_alias_table(self.h, raw, offset, count, False)
        return (raw >> np.uint64(32)).astype(np.uint32), (raw & np.uint64(0xFFFFFFFF)).astype(np.uint32)

    def alias_release(self):
        capi.sv_alias_release(self.h)

    def probabilities(self, offset: int = 0, count: int | None = None, on_device: bool = False):
        count = (1 << self.n) - offset if count is None else count
        if on_device:
            out = torch.empty(count, dtype=torch.float64, device=self.device)
        else:
            out = np.empty(count, dtype=np.float64)
        capi.sv_probabilities(self.h, out, offset, count, on_device)
        return out

    def amplitudes(self, offset: int = 0, count: int | None = None) -> np.ndarray:
        count = (1 << self.n) - offset if count is None else count
        out = np.empty(count, dtype=np.complex64)
        capi.sv_get_amplitudes(self.h, out, offset, count, False)
        return out

    def set_amplitudes(self, values, offset: int = 0):
        v = np.ascontiguousarray(values, dtype=np.complex64)
        capi.sv_set_amplitudes(self.h, v, offset, v.shape[0], False)

    def measure(self, qubit: int, u: float):
        """Mid-circuit measurement of one qubit with uniform u: (outcome, probability)."""
        return capi.sv_measure_qubit(self.h, qubit, u)

    def reset_qubit(self, qubit: int, u: float) -> int:
        return capi.sv_reset_qubit(self.h, qubit, u)

    def clone(self, stream=None) -> "ClonedState":
        """A library-owned copy of this state (on `stream`, default this state's stream)."""
        st = stream if stream is not None else self.stream
        return ClonedState(capi.sv_clone(self.h, st), self.n, st, self.device)

    def merge(self, other: "StateVector", stream=None) -> "ClonedState":
        """p-block merge: self (x) other, self on the low qubits."""
        st = stream if stream is not None else self.stream
        return ClonedState(capi.sv_merge(self.h, other.h, st), self.n + other.n, st, self.device)

    def take_qubit(self, qubit: int, tol: float = 1e-6):
        """Removes a qubit that is in a basis state: (new (n-1)-qubit state, its value)."""
        h, v = capi.sv_take_qubit(self.h, qubit, tol)
        return ClonedState(h, self.n - 1, self.stream, self.device), v

    def profile(self, on: bool = True):
        capi.sv_profile_enable(self.h, on)

    def profile_read(self) -> dict:
        return capi.sv_profile_read(self.h)


class ClonedState(StateVector):
    """A state created by sv_clone: the library owns its buffer."""

    def __init__(self, handle, n: int, stream, device):
        self.n = int(n)
        self.device = device
        self.stream = stream
        self.amps = None
        self.h = handle
