"""ctypes binding of libsvgb.so (include/sv.h): same names, argument marshalling only.

Every function here calls straight into the C-ABI; no step of the hot path runs
in Python.  A non-zero status raises ``SvError`` carrying the library's
``sv_last_error()`` message.  If the library has not been built this module
raises ImportError -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsvgb.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python -m paper_2512_04216_gb300.build, or __graft_entry__.build())")

_L = ctypes.CDLL(LIB_PATH)

SV_OK, SV_ERR_ARG, SV_ERR_OOM, SV_ERR_CUDA, SV_ERR_UNSUPPORTED, SV_ERR_TIMEOUT, SV_ERR_STATE = (
    0, -1, -2, -3, -4, -5, -6)
SV_C64, SV_C128 = 1, 2

GATE_KIND = {
    "u3": 1, "h": 2, "x": 3, "y": 4, "z": 5, "s": 6, "sdg": 7, "t": 8, "tdg": 9, "rx": 10,
    "ry": 11, "rz": 12, "p": 13, "cx": 14, "cz": 15, "cp": 16, "swap": 17, "unitary": 18,
}

GATE_DTYPE = np.dtype([("kind", "u1"), ("nq", "u1"), ("reserved", "<u2"), ("q", "<i4", (5,)),
                       ("p", "<f8", (3,)), ("mat", "<u8")], align=True)
assert GATE_DTYPE.itemsize == 56


class SvError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class sv_opts(ctypes.Structure):
    _fields_ = [("k_max", ctypes.c_int32), ("tile_qubits", ctypes.c_int32),
                ("low_qubits", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("kernel_variant", ctypes.c_int32)]


class sv_plan_info(ctypes.Structure):
    _fields_ = [("n_gates", ctypes.c_uint64), ("n_blocks", ctypes.c_uint64),
                ("n_phase", ctypes.c_uint64), ("n_passes", ctypes.c_uint64),
                ("hist_k", ctypes.c_uint64 * 6), ("flops", ctypes.c_uint64),
                ("bytes", ctypes.c_uint64), ("upload_bytes", ctypes.c_uint64),
                ("n_stages", ctypes.c_uint64), ("tc_stages", ctypes.c_uint64),
                ("passes_by_kind", ctypes.c_uint64 * 3)]

    def as_dict(self):
        return {"n_gates": self.n_gates, "n_blocks": self.n_blocks, "n_phase": self.n_phase,
                "n_passes": self.n_passes, "hist_k": list(self.hist_k), "flops": self.flops,
                "bytes": self.bytes, "upload_bytes": self.upload_bytes,
                "n_stages": self.n_stages, "tc_stages": self.tc_stages,
                "passes_by_kind": list(self.passes_by_kind)}


class sv_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_uint64),
                ("ms", ctypes.c_double), ("bytes", ctypes.c_double)]


_P = ctypes.c_void_p
_u64 = ctypes.c_uint64
_i = ctypes.c_int
_SIGS = {
    "sv_create": ([_i, _i, _P, ctypes.POINTER(_P)], _i),
    "sv_wrap": ([_P, _i, _i, _P, ctypes.POINTER(_P)], _i),
    "sv_destroy": ([_P], _i),
    "sv_set_stream": ([_P, _P], _i),
    "sv_synchronize": ([_P], _i),
    "sv_reset": ([_P, _u64], _i),
    "sv_num_qubits": ([_P], _i),
    "sv_device_ptr": ([_P], _P),
    "sv_apply_circuit": ([_P, _P, ctypes.c_size_t, _P], _i),
    "sv_plan_stats": ([_i, _P, ctypes.c_size_t, _P, _P], _i),
    "sv_norm": ([_P, _P], _i),
    "sv_probabilities": ([_P, _P, _u64, _u64, _i], _i),
    "sv_get_amplitudes": ([_P, _P, _u64, _u64, _i], _i),
    "sv_set_amplitudes": ([_P, _P, _u64, _u64, _i], _i),
    "sv_sample": ([_P, _u64, _u64, _P, _i], _i),
    "sv_sample_uniforms": ([_P, _P, _u64, _P, _P, _i], _i),
    "sv_expect_pauli": ([_P, _u64, _u64, _P], _i),
    "sv_alias_build": ([_P], _i),
    "sv_alias_sample": ([_P, _u64, _u64, _P, _i], _i),
    "sv_alias_sample_uniforms": ([_P, _P, _u64, _P, _i], _i),
    "sv_alias_table": ([_P, _P, _u64, _u64, _i], _i),
    "sv_alias_release": ([_P], _i),
    "sv_profile_enable": ([_P, _i], _i),
    "sv_profile_read": ([_P, _P, _i, _P], _i),
    "sv_last_error": ([], ctypes.c_char_p),
    "sv_version": ([], ctypes.c_char_p),
    "sv_launch_count": ([], ctypes.c_uint64),
    "sv_tc_selftest": ([_P, _P, _P], _i),
    "sv_tc_selftest_r": ([_i, _P, _P, _P], _i),
    "sv_measure_qubit": ([_P, _i, ctypes.c_double, ctypes.POINTER(_i), ctypes.POINTER(ctypes.c_double)], _i),
    "sv_reset_qubit": ([_P, _i, ctypes.c_double, ctypes.POINTER(_i)], _i),
    "sv_clone": ([_P, _P, ctypes.POINTER(_P)], _i),
    "sv_merge": ([_P, _P, _P, ctypes.POINTER(_P)], _i),
    "sv_take_qubit": ([_P, _i, ctypes.c_double, ctypes.POINTER(_i), ctypes.POINTER(_P)], _i),
    "sv_diag_bounded_wait": ([_i], _i),
    "sv_expect_z_static": ([_P, _i, _u64, _P, _P], _i),
    "sv_sample_expect_z": ([_P, _P, _u64, _P, _P, _i, _u64, _P, _P], _i),
    "sv_batch_create": ([ctypes.c_size_t, _P, _P, _P, _P, _P, _P, _P, _i, _P, ctypes.POINTER(_P)], _i),
    "sv_batch_expectation": ([_P, ctypes.c_size_t, _P], _i),
    "sv_batch_launch": ([_P], _i),
    "sv_batch_synchronize": ([_P], _i),
    "sv_batch_samples": ([_P, ctypes.c_size_t, _P, _i], _i),
    "sv_batch_amplitudes": ([_P, ctypes.c_size_t, _P], _i),
    "sv_batch_stats": ([_P, _P, _P], _i),
    "sv_batch_destroy": ([_P], _i),
    "sv_batch_run": ([_P, _P, _P, ctypes.c_size_t, _P, _P, _P, _P], _i),
    "sv_batch_autotune": ([ctypes.c_size_t, _P, _P, _P, _P, _P, _i, _P, _P], _i),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_L, _name)
    _f.argtypes = _args
    _f.restype = _res

EXPORTED = tuple(_SIGS)


def _check(rc: int):
    if rc != SV_OK:
        raise SvError(rc, _L.sv_last_error().decode())


def _ptr(x) -> int:
    """Address of a numpy array or torch tensor (device or host)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return int(x.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# ---------------------------------------------------------------------------
# IR marshalling
# ---------------------------------------------------------------------------

def to_ir(circuit):
    """(name, qubits, params) tuples -> (sv_gate array, keep-alive list)."""
    ir = np.zeros(max(len(circuit), 1), dtype=GATE_DTYPE)
    keep = []
    for a, (name, qs, ps) in enumerate(circuit):
        ir["kind"][a] = GATE_KIND[name]
        ir["nq"][a] = len(qs)
        ir["q"][a, : len(qs)] = qs
        if name == "unitary":
            m = np.ascontiguousarray(np.asarray(ps[0], dtype=np.complex128))
            keep.append(m)
            ir["mat"][a] = m.ctypes.data
        else:
            ir["p"][a, : len(ps)] = ps
    return ir, keep


def make_opts(k_max=0, tile_qubits=0, low_qubits=0, precision=0, kernel_variant=0):
    return sv_opts(int(k_max), int(tile_qubits), int(low_qubits), int(precision),
                   int(kernel_variant))


# ---------------------------------------------------------------------------
# the C-ABI, one wrapper per entry point
# ---------------------------------------------------------------------------

def sv_version() -> str:
    return _L.sv_version().decode()


def sv_launch_count() -> int:
    return int(_L.sv_launch_count())


def sv_last_error() -> str:
    return _L.sv_last_error().decode()


def sv_create(n_qubits: int, dtype: int = SV_C64, stream=None):
    h = _P()
    _check(_L.sv_create(n_qubits, dtype, _stream_ptr(stream), ctypes.byref(h)))
    return h


def sv_wrap(dev_tensor, n_qubits: int, dtype: int = SV_C64, stream=None):
    h = _P()
    _check(_L.sv_wrap(_ptr(dev_tensor), n_qubits, dtype, _stream_ptr(stream), ctypes.byref(h)))
    return h


def sv_destroy(h):
    _check(_L.sv_destroy(h))


def sv_set_stream(h, stream):
    _check(_L.sv_set_stream(h, _stream_ptr(stream)))


def sv_synchronize(h):
    _check(_L.sv_synchronize(h))


def sv_reset(h, basis_index: int = 0):
    _check(_L.sv_reset(h, int(basis_index)))


def sv_num_qubits(h) -> int:
    return int(_L.sv_num_qubits(h))


def sv_device_ptr(h) -> int:
    return int(_L.sv_device_ptr(h) or 0)


def sv_apply_circuit(h, ir, n_gates=None, opts=None):
    """ir: an sv_gate ndarray (see to_ir) with n_gates rows, or a circuit list."""
    keep = None
    if not isinstance(ir, np.ndarray):
        n_gates = len(ir)
        ir, keep = to_ir(ir)
    elif n_gates is None:
        n_gates = ir.shape[0]
    _check(_L.sv_apply_circuit(h, ir.ctypes.data, int(n_gates),
                               ctypes.byref(opts) if opts is not None else None))
    return keep


def sv_plan_stats(n_qubits, circuit, opts=None) -> dict:
    ir, keep = to_ir(circuit)
    info = sv_plan_info()
    _check(_L.sv_plan_stats(n_qubits, ir.ctypes.data, len(circuit),
                            ctypes.byref(opts) if opts is not None else None, ctypes.byref(info)))
    return info.as_dict()


def sv_plan_stats_ir(n_qubits, ir, n_gates, opts=None) -> dict:
    """sv_plan_stats on an already marshalled IR."""
    info = sv_plan_info()
    _check(_L.sv_plan_stats(n_qubits, ir.ctypes.data, int(n_gates),
                            ctypes.byref(opts) if opts is not None else None, ctypes.byref(info)))
    return info.as_dict()


def sv_norm(h) -> float:
    out = ctypes.c_double()
    _check(_L.sv_norm(h, ctypes.byref(out)))
    return out.value


def sv_probabilities(h, out, offset: int, count: int, out_on_device: bool):
    _check(_L.sv_probabilities(h, _ptr(out), int(offset), int(count), int(bool(out_on_device))))


def sv_get_amplitudes(h, out, offset: int, count: int, out_on_device: bool):
    _check(_L.sv_get_amplitudes(h, _ptr(out), int(offset), int(count), int(bool(out_on_device))))


def sv_set_amplitudes(h, src, offset: int, count: int, in_on_device: bool):
    _check(_L.sv_set_amplitudes(h, _ptr(src), int(offset), int(count), int(bool(in_on_device))))


def sv_sample(h, shots: int, seed: int, out, on_device: bool):
    _check(_L.sv_sample(h, int(shots), int(seed) & (2**64 - 1), _ptr(out), int(bool(on_device))))


def sv_sample_uniforms(h, uniforms, shots: int, out, on_device: bool) -> int:
    nb = ctypes.c_uint64()
    _check(_L.sv_sample_uniforms(h, _ptr(uniforms), int(shots), _ptr(out), ctypes.byref(nb),
                                 int(bool(on_device))))
    return int(nb.value)


def sv_sample_expect_z(h, uniforms, shots: int, out, on_device: bool, z_mask: int):
    """Draws (as sv_sample_uniforms), <Z_mask> and ||psi||^2 from one read of the
    state; returns (n_boundary, expectation, norm2)."""
    nb = ctypes.c_uint64(0)
    e = ctypes.c_double(0.0)
    n2 = ctypes.c_double(0.0)
    _check(_L.sv_sample_expect_z(h, _ptr(uniforms), int(shots), _ptr(out), ctypes.byref(nb),
                                 int(bool(on_device)), int(z_mask), ctypes.byref(e), ctypes.byref(n2)))
    return int(nb.value), float(e.value), float(n2.value)


def sv_alias_build(h):
    _check(_L.sv_alias_build(h))


def sv_alias_sample(h, shots: int, seed: int, out, on_device: bool):
    _check(_L.sv_alias_sample(h, int(shots), int(seed) & (2**64 - 1), _ptr(out), int(bool(on_device))))


def sv_alias_sample_uniforms(h, uniforms, shots: int, out, on_device: bool):
    _check(_L.sv_alias_sample_uniforms(h, _ptr(uniforms), int(shots), _ptr(out), int(bool(on_device))))


def sv_alias_table(h, out, offset: int, count: int, on_device: bool):
    _check(_L.sv_alias_table(h, _ptr(out), int(offset), int(count), int(bool(on_device))))


def sv_alias_release(h):
    _check(_L.sv_alias_release(h))


def sv_expect_pauli(h, x_mask: int, z_mask: int) -> float:
    out = ctypes.c_double()
    _check(_L.sv_expect_pauli(h, int(x_mask), int(z_mask), ctypes.byref(out)))
    return out.value


def sv_tc_selftest(a, b):
    """Tensor-core product check (include/sv_diag.h): a 128x32 float32, b 32x32 float64."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float64)
    assert a.shape == (128, 32) and b.shape == (32, 32)
    d = np.empty((128, 32), dtype=np.float32)
    _check(_L.sv_tc_selftest(a.ctypes.data, b.ctypes.data, d.ctypes.data))
    return d


def sv_tc_selftest_r(r, a, b):
    """Tensor-core product check of an r-qubit stage (include/sv_diag.h):
    a 128 x 2^(r+1) float32, b 2^(r+1) x 2^(r+1) float64."""
    k = 2 << r
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float64)
    assert a.shape == (128, k) and b.shape == (k, k)
    d = np.empty((128, k), dtype=np.float32)
    _check(_L.sv_tc_selftest_r(int(r), a.ctypes.data, b.ctypes.data, d.ctypes.data))
    return d


def sv_measure_qubit(h, qubit: int, u: float):
    """Mid-circuit measurement: returns (outcome, probability of that outcome)."""
    out = _i()
    prob = ctypes.c_double()
    _check(_L.sv_measure_qubit(h, int(qubit), float(u), ctypes.byref(out), ctypes.byref(prob)))
    return int(out.value), float(prob.value)


def sv_reset_qubit(h, qubit: int, u: float) -> int:
    """Reset of one qubit to |0> by measurement; returns the measured bit."""
    out = _i()
    _check(_L.sv_reset_qubit(h, int(qubit), float(u), ctypes.byref(out)))
    return int(out.value)


def sv_clone(h, stream=None):
    out = _P()
    _check(_L.sv_clone(h, _stream_ptr(stream), ctypes.byref(out)))
    return out


def sv_merge(a, b, stream=None):
    out = _P()
    _check(_L.sv_merge(a, b, _stream_ptr(stream), ctypes.byref(out)))
    return out


def sv_take_qubit(h, qubit: int, tol: float = 1e-6):
    """Removes a basis-state qubit: returns (new handle, its value)."""
    out = _P()
    v = _i()
    _check(_L.sv_take_qubit(h, int(qubit), float(tol), ctypes.byref(v), ctypes.byref(out)))
    return out, int(v.value)


def sv_diag_bounded_wait(limit_ms: int) -> int:
    """Status of a bounded wait on nothing (include/sv_diag.h); SV_ERR_TIMEOUT expected."""
    return int(_L.sv_diag_bounded_wait(int(limit_ms)))


def sv_expect_z_static(dev_amplitudes, n_qubits: int, z_mask: int, dev_out, stream=None):
    """Allocation-free <Z_mask> into dev_out[0] (and the norm into dev_out[1]);
    both pointers are device memory; queued on `stream` (see include/sv.h)."""
    _check(_L.sv_expect_z_static(_ptr(dev_amplitudes), int(n_qubits), int(z_mask), _ptr(dev_out),
                                 _stream_ptr(stream)))


class BatchArgs:
    """Marshalled arrays for the sv_batch_* calls (keeps the IR arrays alive).

    Give either ``circuits`` (gate lists) or ``irs``: (sv_gate array, n_gates)
    pairs already marshalled with to_ir."""

    def __init__(self, circuits, n_qubits, shots, seeds, zmasks=None, irs=None):
        if irs is None:
            irs = [(to_ir(c)[0], len(c)) for c in circuits]
        self.irs = irs
        self.ptrs = np.array([ir.ctypes.data for ir, _ in irs], dtype=np.uint64)
        self.n_gates = np.array([ng for _, ng in irs], dtype=np.uint64)
        self.n_qubits = np.array(n_qubits, dtype=np.int32)
        self.shots = np.array(shots, dtype=np.uint64)
        self.seeds = np.array([int(x) & (2**64 - 1) for x in seeds], dtype=np.uint64)
        self.zmasks = np.array([int(z) for z in zmasks], dtype=np.uint64) if zmasks is not None else None
        self.n = len(irs)


def sv_batch_create(args: BatchArgs, opts=None, keep_states=False, stream=None):
    h = _P()
    _check(_L.sv_batch_create(args.n, args.ptrs.ctypes.data, args.n_gates.ctypes.data,
                              args.n_qubits.ctypes.data, args.shots.ctypes.data, args.seeds.ctypes.data,
                              args.zmasks.ctypes.data if args.zmasks is not None else None,
                              ctypes.byref(opts) if opts is not None else None, int(bool(keep_states)),
                              _stream_ptr(stream), ctypes.byref(h)))
    return h


def sv_batch_launch(h):
    _check(_L.sv_batch_launch(h))


def sv_batch_synchronize(h):
    _check(_L.sv_batch_synchronize(h))


def sv_batch_samples(h, circuit: int, out, on_device: bool = False):
    _check(_L.sv_batch_samples(h, int(circuit), _ptr(out), int(bool(on_device))))


def sv_batch_expectation(h, circuit: int):
    out = np.empty(2, dtype=np.float64)
    _check(_L.sv_batch_expectation(h, int(circuit), out.ctypes.data))
    return float(out[0]), float(out[1])


def sv_batch_amplitudes(h, circuit: int, out):
    _check(_L.sv_batch_amplitudes(h, int(circuit), _ptr(out)))


def sv_batch_stats(h):
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    _check(_L.sv_batch_stats(h, ctypes.byref(a), ctypes.byref(b)))
    return {"passes": a.value, "hbm_bytes": b.value}


def sv_batch_destroy(h):
    _check(_L.sv_batch_destroy(h))


def sv_batch_run(args: BatchArgs, outs, opts=None):
    ptrs = np.array([_ptr(o) or 0 for o in outs], dtype=np.uint64)
    _check(_L.sv_batch_run(args.ptrs.ctypes.data, args.n_gates.ctypes.data, args.n_qubits.ctypes.data, args.n,
                           args.shots.ctypes.data, args.seeds.ctypes.data, ptrs.ctypes.data,
                           ctypes.byref(opts) if opts is not None else None))


def sv_batch_autotune(args: BatchArgs, reps: int = 2):
    best = sv_opts()
    ms = ctypes.c_double()
    _check(_L.sv_batch_autotune(args.n, args.ptrs.ctypes.data, args.n_gates.ctypes.data,
                                args.n_qubits.ctypes.data, args.shots.ctypes.data, args.seeds.ctypes.data,
                                int(reps), ctypes.byref(best), ctypes.byref(ms)))
    return best, ms.value


def sv_profile_enable(h, on: bool = True):
    _check(_L.sv_profile_enable(h, int(bool(on))))


def sv_profile_read(h) -> dict:
    cap = 32
    arr = (sv_kernel_stat * cap)()
    n = ctypes.c_int()
    _check(_L.sv_profile_read(h, ctypes.cast(arr, _P), cap, ctypes.byref(n)))
    return {arr[i].name.decode(): {"launches": int(arr[i].launches), "ms": float(arr[i].ms),
                                   "bytes": float(arr[i].bytes)} for i in range(min(n.value, cap))}
