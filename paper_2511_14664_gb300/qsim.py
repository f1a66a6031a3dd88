"""Python binding of libqsim (C ABI in include/qsim.h): argument marshalling only.

Every computation runs in the library's CUDA kernels. PyTorch supplies device memory (the state tensor)
and the CUDA stream. If the compiled library is missing it is built with nvcc on first use; if that is not
possible the binding raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from itertools import chain
from typing import Iterable, Optional, Sequence

import numpy as np

from . import build as _build

C64, C128 = 0, 1
PREC_SIMT, PREC_TF32X3, PREC_BF16X3, PREC_BF16X6, PREC_FP16X3 = 0, 1, 2, 3, 4
RUN_PLAIN, RUN_FUSED = 0, 1
MAX_TARGETS = MAX_CONTROLS = 8
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EUNSUPPORTED"}
PRECISIONS = {"simt": PREC_SIMT, "tf32x3": PREC_TF32X3, "bf16x3": PREC_BF16X3, "bf16x6": PREC_BF16X6,
              "fp16x3": PREC_FP16X3}


class QsimError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Gate(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("nc", ctypes.c_int32),
                ("targets", ctypes.c_int32 * MAX_TARGETS), ("controls", ctypes.c_int32 * MAX_CONTROLS),
                ("matrix", ctypes.POINTER(ctypes.c_double))]


class Circuit(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("num_gates", ctypes.c_int32), ("gates", ctypes.POINTER(Gate))]


class RunOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("max_fused", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("tc_min_k", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("local_qubits", ctypes.c_int32),
                ("dry_run", ctypes.c_int32), ("batch_tc_min_n", ctypes.c_int32),
                ("plan_effort", ctypes.c_int32), ("pair_blocks", ctypes.c_int32),
                ("launch_per_pass", ctypes.c_int32)]


class PassInfo(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("k", ctypes.c_int32), ("nc", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("gates", ctypes.c_int64), ("algorithmic_bytes", ctypes.c_double),
                ("targets", ctypes.c_int32 * 8), ("controls", ctypes.c_int32 * 8),
                ("launches", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class SpillOpts(ctypes.Structure):
    _fields_ = [("window_qubits", ctypes.c_int32), ("global_slots", ctypes.c_int32), ("run", RunOpts)]


class SpillInfo(ctypes.Structure):
    _fields_ = [("segments", ctypes.c_int64), ("windows", ctypes.c_int64), ("passes", ctypes.c_int64),
                ("host_bytes", ctypes.c_double), ("elapsed_ms", ctypes.c_double), ("host_plan_ms", ctypes.c_double),
                ("window_qubits", ctypes.c_int32), ("global_slots", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


PASS_KINDS = {0: "dense_small", 1: "diag", 2: "dense_tile", 3: "tc", 4: "reorder", 5: "phase", 6: "tc_pair"}


class PlanInfo(ctypes.Structure):
    _fields_ = [("input_gates", ctypes.c_int64), ("passes", ctypes.c_int64), ("dense_blocks", ctypes.c_int64),
                ("tc_blocks", ctypes.c_int64), ("diag_blocks", ctypes.c_int64), ("reorders", ctypes.c_int64),
                ("algorithmic_bytes", ctypes.c_double), ("host_plan_ms", ctypes.c_double),
                ("resident", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None
# Every entry point the header declares, with its argument types.
_P, _vp, _i, _u64, _i64, _sz = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_int64, ctypes.c_size_t
SIGNATURES = {
    "qsim_abi_version": ([], _i),
    "qsim_last_error": ([], ctypes.c_char_p),
    "qsim_state_bytes": ([_i, _i, _P(_sz)], _i),
    "qsim_create": ([_i, _i, _vp, _sz, _vp, _P(_vp)], _i),
    "qsim_destroy": ([_vp], _i),
    "qsim_set_stream": ([_vp, _vp], _i),
    "qsim_num_qubits": ([_vp, _P(_i)], _i),
    "qsim_device_ptr": ([_vp, _P(_vp)], _i),
    "qsim_set_basis": ([_vp, _u64], _i),
    "qsim_set_state": ([_vp, _vp, _i], _i),
    "qsim_get_state": ([_vp, _vp, _i], _i),
    "qsim_synchronize": ([_vp], _i),
    "qsim_inject_device_error": ([_vp, ctypes.c_uint], _i),
    "qsim_apply_gate": ([_vp, _P(_i), _i, _P(_i), _i, _P(ctypes.c_double)], _i),
    "qsim_apply_fused": ([_vp, _P(_i), _i, _P(ctypes.c_double), _i], _i),
    "qsim_swap_qubits": ([_vp, _P(_i), _P(_i), _i], _i),
    "qsim_plan_create": ([_P(Circuit), _i, _P(RunOpts), _vp, _P(_vp), _P(PlanInfo)], _i),
    "qsim_plan_execute": ([_vp, _vp], _i),
    "qsim_plan_destroy": ([_vp], _i),
    "qsim_plan_cache_clear": ([], _i),
    "qsim_plan_num_passes": ([_vp, _P(_i64)], _i),
    "qsim_plan_pass_info": ([_vp, _i64, _P(PassInfo)], _i),
    "qsim_plan_execute_from_basis": ([_vp, _vp, _u64, _i64], _i),
    "qsim_plan_execute_range": ([_vp, _vp, _i64, _i64], _i),
    "qsim_run": ([_vp, _P(Circuit), _P(RunOpts), _P(PlanInfo)], _i),
    "qsim_norm": ([_vp, _P(ctypes.c_double)], _i),
    "qsim_probs": ([_vp, _P(_i), _i, _P(ctypes.c_double)], _i),
    "qsim_expect_pauli": ([_vp, ctypes.c_char_p, _P(ctypes.c_double)], _i),
    "qsim_expect_z": ([_vp, _P(ctypes.c_double), _P(ctypes.c_double)], _i),
    "qsim_sample": ([_vp, _u64, _i64, _P(_u64)], _i),
    "qsim_sample_uniforms": ([_vp, _P(ctypes.c_double), _i64, _P(_u64)], _i),
    "qsim_expect_z_and_sample": ([_vp, _P(ctypes.c_double), _P(ctypes.c_double), _u64, _i64, _P(_u64)], _i),
    "qsim_inner": ([_vp, _vp, _P(ctypes.c_double)], _i),
    "qsim_sample_noalloc": ([_vp, _i, _i, _u64, _i64, _vp, _vp], _i),
    "qsim_spill_run": ([_vp, _P(Circuit), _i, _P(SpillOpts), _vp, _P(SpillInfo)], _i),
    "qsim_spill_segments": ([_P(Circuit), _i, _i, _P(ctypes.c_int32), _P(_u64), _P(_i64)], _i),
    "qsim_spill_sample": ([_vp, _i, _i, _i, _u64, _i64, _P(_u64), _P(ctypes.c_double)], _i),
    "qsim_tc_peak": ([_i, _i, ctypes.c_double, _P(ctypes.c_double), _P(ctypes.c_double)], _i),
    "qsim_fp64_peak": ([ctypes.c_double, _P(ctypes.c_double), _P(ctypes.c_double)], _i),
    "qsim_batch_workspace_bytes": ([_P(Circuit), _i, _P(_sz)], _i),
    "qsim_batch_plan_create": ([_P(Circuit), _i, _P(RunOpts), _vp, _P(_vp), _P(PlanInfo)], _i),
    "qsim_batch_execute": ([_vp, _vp, _sz, _vp, _i], _i),
    "qsim_batch_results": ([_vp, _vp, _P(ctypes.c_double), _P(ctypes.c_double)], _i),
    "qsim_batch_destroy": ([_vp], _i),
    "qsim_batch_run": ([_P(Circuit), _i, _P(RunOpts), _vp, _sz, _vp, _P(ctypes.c_double), _P(ctypes.c_double),
                        _P(PlanInfo)], _i),
    "qsim_batch_autotune": ([_P(Circuit), _i, _vp, _P(_i)], _i),
    "qsim_batch_autotune_threshold": ([_P(Circuit), _i, _i, _vp, _P(_i)], _i),
    "qsim_batch_tune_save": ([ctypes.c_char_p], _i),
    "qsim_batch_tune_load": ([ctypes.c_char_p], _i),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libqsim (building it with nvcc if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        for name, (args, res) in SIGNATURES.items():
            f = getattr(L, name, None)
            if f is None:
                continue
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(rc: int) -> None:
    if rc != 0:
        raise QsimError(rc, lib().qsim_last_error().decode())


def _ints(xs: Iterable[int]):
    xs = [int(x) for x in xs]
    return (ctypes.c_int * max(1, len(xs)))(*xs), len(xs)


def _mat(U) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(U, dtype=np.complex128))


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _stream_ptr(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def state_bytes(n: int, dtype: int) -> int:
    out = ctypes.c_size_t()
    _check(lib().qsim_state_bytes(n, dtype, ctypes.byref(out)))
    return out.value


class State:
    """An n-qubit state whose amplitudes live in a torch tensor on the current CUDA device."""

    def __init__(self, n: int, dtype: int = C64, tensor=None, stream=None):
        import torch
        self.n = n
        self.dtype = dtype
        tdt = torch.complex64 if dtype == C64 else torch.complex128
        if tensor is None:
            tensor = torch.empty(1 << n, dtype=tdt, device="cuda")
        if tensor.dtype != tdt or tensor.numel() != (1 << n) or not tensor.is_cuda or not tensor.is_contiguous():
            raise ValueError("state tensor must be a contiguous CUDA tensor of 2^n amplitudes of the state dtype")
        self.tensor = tensor
        self._stream = stream
        h = ctypes.c_void_p()
        _check(lib().qsim_create(n, dtype, ctypes.c_void_p(tensor.data_ptr()),
                                 tensor.numel() * tensor.element_size(), ctypes.c_void_p(_stream_ptr(stream)),
                                 ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().qsim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- state ----------------------------------------------------------------------------------------
    def set_basis(self, x: int = 0):
        _check(lib().qsim_set_basis(self.h, int(x)))
        return self

    def set_state(self, psi: np.ndarray):
        dt = np.complex64 if self.dtype == C64 else np.complex128
        a = np.ascontiguousarray(psi, dtype=dt)
        _check(lib().qsim_set_state(self.h, ctypes.c_void_p(a.ctypes.data), 0))
        return self

    def get_state(self) -> np.ndarray:
        dt = np.complex64 if self.dtype == C64 else np.complex128
        out = np.empty(1 << self.n, dtype=dt)
        _check(lib().qsim_get_state(self.h, ctypes.c_void_p(out.ctypes.data), 0))
        return out

    def synchronize(self):
        _check(lib().qsim_synchronize(self.h))

    # -- gates ------------------------------------------------------------------------------------------
    def apply_gate(self, targets: Sequence[int], controls: Sequence[int], U):
        t, k = _ints(targets)
        c, nc = _ints(controls)
        m = _mat(U)
        _check(lib().qsim_apply_gate(self.h, t, k, c, nc, _dptr(m)))
        return self

    def apply_fused(self, targets: Sequence[int], U, precision: int = PREC_SIMT):
        t, k = _ints(targets)
        m = _mat(U)
        _check(lib().qsim_apply_fused(self.h, t, k, _dptr(m), int(precision)))
        return self

    def swap_qubits(self, a: Sequence[int], b: Sequence[int]):
        pa, p = _ints(a)
        pb, _ = _ints(b)
        _check(lib().qsim_swap_qubits(self.h, pa, pb, p))
        return self

    def run(self, circuit, mode: int = RUN_PLAIN, max_fused: int = 5, precision: int = PREC_SIMT,
            tc_min_k: int = 5, local_qubits: int = 0, plan_effort: int = 0, pair_blocks: bool = False,
            launch_per_pass: bool = False):
        cc = CircuitArgs(circuit)
        o = RunOpts(mode=mode, max_fused=max_fused, precision=precision, tc_min_k=tc_min_k, use_graph=0,
                    local_qubits=local_qubits, plan_effort=plan_effort, pair_blocks=1 if pair_blocks else 0,
                    launch_per_pass=1 if launch_per_pass else 0)
        info = PlanInfo()
        _check(lib().qsim_run(self.h, ctypes.byref(cc.c), ctypes.byref(o), ctypes.byref(info)))
        return info.as_dict()

    # -- readout ----------------------------------------------------------------------------------------
    def norm(self) -> float:
        out = ctypes.c_double()
        _check(lib().qsim_norm(self.h, ctypes.byref(out)))
        return out.value

    def probs(self, qubits: Sequence[int]) -> np.ndarray:
        q, nq = _ints(qubits)
        out = np.zeros(1 << nq, dtype=np.float64)
        _check(lib().qsim_probs(self.h, q, nq, _dptr(out)))
        return out

    def expect_pauli(self, paulis: str) -> complex:
        out = np.zeros(2, dtype=np.float64)
        _check(lib().qsim_expect_pauli(self.h, paulis.encode(), _dptr(out)))
        return complex(out[0], out[1])

    def expect_z(self):
        zi = np.zeros(self.n, dtype=np.float64)
        zz = np.zeros(max(1, self.n - 1), dtype=np.float64)
        _check(lib().qsim_expect_z(self.h, _dptr(zi), _dptr(zz)))
        return zi, zz[: self.n - 1]

    def sample(self, seed: int, shots: int) -> np.ndarray:
        out = np.zeros(shots, dtype=np.uint64)
        _check(lib().qsim_sample(self.h, seed & (2**64 - 1), shots,
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
        return out

    def expect_z_and_sample(self, seed: int, shots: int):
        """(<Z_i>, <Z_i Z_i+1>, samples) with one read of the state."""
        zi = np.zeros(self.n)
        zz = np.zeros(max(1, self.n - 1))
        out = np.zeros(max(1, shots), dtype=np.uint64)
        _check(lib().qsim_expect_z_and_sample(self.h, _dptr(zi), _dptr(zz), seed & (2**64 - 1), shots,
                                              out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
        return zi, zz[: max(0, self.n - 1)], out[:shots]

    def sample_uniforms(self, u: np.ndarray) -> np.ndarray:
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.zeros(len(u), dtype=np.uint64)
        _check(lib().qsim_sample_uniforms(self.h, _dptr(u), len(u),
                                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
        return out

    def inner(self, other: "State") -> complex:
        out = np.zeros(2, dtype=np.float64)
        _check(lib().qsim_inner(self.h, other.h, _dptr(out)))
        return complex(out[0], out[1])


# numpy image of the qsim_gate struct, so that a whole gate list is packed with array operations
_GATE_NP = np.dtype({"names": ["k", "nc", "targets", "controls", "matrix"],
                     "formats": ["<i4", "<i4", ("<i4", (MAX_TARGETS,)), ("<i4", (MAX_CONTROLS,)), "<u8"],
                     "offsets": [Gate.k.offset, Gate.nc.offset, Gate.targets.offset, Gate.controls.offset,
                                 Gate.matrix.offset],
                     "itemsize": ctypes.sizeof(Gate)})


def _pack_gates(gs):
    """Gate records in the qsim_gate layout for the list `gs`, plus the matrix arrays they point into (one
    per gate width, so that all gates of a width are copied with one array operation). Three passes over
    the gate objects to collect their fields; the rest is array work."""
    G = len(gs)
    rec = np.zeros(max(1, G), dtype=_GATE_NP)
    pools = []
    if G:
        tg = [g.targets for g in gs]
        ct = [g.controls for g in gs]
        mt = [g.matrix for g in gs]
        ks = np.fromiter(map(len, tg), dtype=np.int32, count=G)
        # (any() stops at the first gate with controls; without any, no per-gate lengths are needed)
        ncs = np.fromiter(map(len, ct), dtype=np.int32, count=G) if any(map(len, ct)) else np.zeros(G, dtype=np.int32)
        if int(ks.max()) > MAX_TARGETS or int(ncs.max()) > MAX_CONTROLS:
            raise ValueError("a gate has more than %d targets or controls" % MAX_TARGETS)
        rec["k"][:G] = ks
        rec["nc"][:G] = ncs
        ids = np.fromiter(map(id, mt), dtype=np.int64, count=G)

        def fill(field, lists, lens):
            # all lists chained into one array, then each gate's entries gathered by its offset
            flat = np.fromiter(chain.from_iterable(lists), dtype=np.int32, count=int(lens.sum()))
            off = np.zeros(G, dtype=np.int64)
            np.cumsum(lens[:-1], out=off[1:])
            for k in np.unique(lens):
                k = int(k)
                if k:
                    idx = np.nonzero(lens == k)[0]
                    rec[field][idx, :k] = flat[off[idx][:, None] + np.arange(k)]

        fill("targets", tg, ks)
        if int(ncs.max()):
            fill("controls", ct, ncs)
        for k in np.unique(ks):  # gates of one width share an array of matrices
            idx = np.nonzero(ks == k)[0]
            k = int(k)
            # one copy per distinct matrix object (circuits often reuse one array for many gates)
            uniq, first, inv = np.unique(ids[idx], return_index=True, return_inverse=True)
            M = np.ascontiguousarray(np.array([mt[idx[j]] for j in first], dtype=np.complex128))
            if M.shape[1:] != (1 << k, 1 << k):
                raise ValueError("a %d-qubit gate needs a %dx%d matrix" % (k, 1 << k, 1 << k))
            pools.append(M)
            rec["matrix"][idx] = M.ctypes.data + inv.astype(np.uint64).ravel() * np.uint64(M[0].nbytes)
    return rec, pools


class CircuitArgs:
    """A workloads.Circuit marshalled into qsim_gate structs: one record array for the gates and, per gate
    width, one array holding those gates' matrices (all kept alive here)."""

    def __init__(self, circuit):
        self.n = circuit.n
        self.rec, self.pools = _pack_gates(circuit.gates)
        self.gates = ctypes.cast(self.rec.ctypes.data, ctypes.POINTER(Gate))
        self.c = Circuit(n=circuit.n, num_gates=len(circuit.gates), gates=self.gates)


class CircuitsArgs:
    """Many circuits marshalled at once (all their gates packed in one pass): `arr` is the qsim_circuit array
    the batch entry points take."""

    def __init__(self, circuits):
        circuits = list(circuits)
        allg = [g for c in circuits for g in c.gates]
        self.rec, self.pools = _pack_gates(allg)
        base = self.rec.ctypes.data
        size = ctypes.sizeof(Gate)
        self.arr = (Circuit * max(1, len(circuits)))()
        off = 0
        for i, c in enumerate(circuits):
            G = len(c.gates)
            self.arr[i] = Circuit(n=c.n, num_gates=G, gates=ctypes.cast(base + off * size, ctypes.POINTER(Gate)))
            off += G
        self.count = len(circuits)


class Plan:
    """A planned circuit (fusion, kernel choice, FP64 block composition done once)."""

    def __init__(self, circuit, dtype: int = C64, mode: int = RUN_PLAIN, max_fused: int = 5,
                 precision: int = PREC_SIMT, tc_min_k: int = 5, use_graph: bool = False, stream=None,
                 local_qubits: int = 0, dry_run: bool = False, plan_effort: int = 0, pair_blocks: bool = False,
                 launch_per_pass: bool = False):
        """dry_run: plan on the host only (no device needed); the plan lists its passes but cannot run.
        plan_effort 1: also try fusion with one block of look-ahead, keep the grouping with fewer blocks.
        pair_blocks (with PREC_FP16X3): two consecutive 6-qubit blocks per pass where they fit a tile.
        launch_per_pass: one launch per pass even where the plan could run in one resident launch (states of
        at most 16 qubits, CUDA-core passes only)."""
        self.args = CircuitArgs(circuit)
        o = RunOpts(mode=mode, max_fused=max_fused, precision=precision, tc_min_k=tc_min_k,
                    use_graph=1 if use_graph else 0, local_qubits=local_qubits, dry_run=1 if dry_run else 0,
                    plan_effort=plan_effort, pair_blocks=1 if pair_blocks else 0,
                    launch_per_pass=1 if launch_per_pass else 0)
        info = PlanInfo()
        p = ctypes.c_void_p()
        _check(lib().qsim_plan_create(ctypes.byref(self.args.c), dtype, ctypes.byref(o),
                                      ctypes.c_void_p(0 if dry_run else _stream_ptr(stream)), ctypes.byref(p),
                                      ctypes.byref(info)))
        self.p = p
        self.info = info.as_dict()

    def execute(self, state: State):
        _check(lib().qsim_plan_execute(state.h, self.p))

    def execute_from_basis(self, state: State, x: int = 0, count: int = -1):
        """set_basis(x), then passes [0, count) (all for count < 0); a first tensor-core block generates |x>
        itself instead of reading it."""
        _check(lib().qsim_plan_execute_from_basis(state.h, self.p, int(x), int(count)))

    def execute_range(self, state: State, first: int, count: int):
        _check(lib().qsim_plan_execute_range(state.h, self.p, int(first), int(count)))

    def passes(self):
        """Per-pass descriptions: kind, k, controls, precision, merged gates, algorithmic bytes, qubits."""
        num = ctypes.c_int64()
        _check(lib().qsim_plan_num_passes(self.p, ctypes.byref(num)))
        out = []
        for i in range(num.value):
            pi = PassInfo()
            _check(lib().qsim_plan_pass_info(self.p, i, ctypes.byref(pi)))
            out.append({"kind": PASS_KINDS[pi.kind], "k": pi.k, "nc": pi.nc, "precision": pi.precision,
                        "gates": pi.gates, "algorithmic_bytes": pi.algorithmic_bytes,
                        "targets": list(pi.targets[:pi.k]), "controls": list(pi.controls[:pi.nc]),
                        "launches": pi.launches})
        return out

    def close(self):
        if getattr(self, "p", None):
            lib().qsim_plan_destroy(self.p)
            self.p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _host_ptr(state) -> int:
    """Address of a host state: a numpy array or a CPU torch tensor (page-locked ones let copies overlap)."""
    if isinstance(state, np.ndarray):
        if not state.flags.c_contiguous:
            raise ValueError("host state must be contiguous")
        return state.ctypes.data
    if getattr(state, "is_cuda", False) or not state.is_contiguous():
        raise ValueError("host state must be a contiguous CPU tensor or numpy array")
    return state.data_ptr()


def spill_run(host_state, circuit, dtype: int = C64, window_qubits: int = 28, global_slots: int = 0,
              mode: int = RUN_FUSED, max_fused: int = 6, precision: int = PREC_TF32X3, tc_min_k: int = 5,
              plan_effort: int = 0, stream=None) -> dict:
    """Run `circuit` in place on a state held in host memory, streamed through device windows of
    2^window_qubits amplitudes (three of them); returns the run's counters (segments, windows, bytes, ms)."""
    cc = CircuitArgs(circuit)
    o = SpillOpts(window_qubits=window_qubits, global_slots=global_slots,
                  run=RunOpts(mode=mode, max_fused=max_fused, precision=precision, tc_min_k=tc_min_k,
                              plan_effort=plan_effort))
    info = SpillInfo()
    _check(lib().qsim_spill_run(ctypes.c_void_p(_host_ptr(host_state)), ctypes.byref(cc.c), dtype, ctypes.byref(o),
                                ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(info)))
    return info.as_dict()


def spill_segments(circuit, window_qubits: int, global_slots: int = 0):
    """Host-only segmentation of an out-of-core run: (segment of every gate, top-bit qubit mask per segment)."""
    cc = CircuitArgs(circuit)
    G = len(circuit.gates)
    seg = (ctypes.c_int32 * max(1, G))()
    used = (ctypes.c_uint64 * max(1, G))()
    ns = ctypes.c_int64()
    _check(lib().qsim_spill_segments(ctypes.byref(cc.c), int(window_qubits), int(global_slots), seg, used,
                                     ctypes.byref(ns)))
    return np.array(seg[:G], dtype=np.int64), [int(used[i]) for i in range(ns.value)]


def spill_sample(host_state, n: int, dtype: int, window_qubits: int, seed: int, shots: int):
    """Samples (and the squared norm) of a host state, streamed through the device by slices."""
    out = np.zeros(max(1, shots), dtype=np.uint64)
    nrm = ctypes.c_double()
    _check(lib().qsim_spill_sample(ctypes.c_void_p(_host_ptr(host_state)), int(n), int(dtype), int(window_qubits),
                                   seed & (2**64 - 1), int(shots), out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                   ctypes.byref(nrm)))
    return out[:shots], nrm.value


def plan_cache_clear():
    """Empty the planner's cache of groupings by circuit structure (qsim_plan_cache_clear)."""
    _check(lib().qsim_plan_cache_clear())


def tc_peak(kind: str = "tf32", n_cols: int = 128, seconds: float = 1.0):
    """Measured dense tensor-core rate (TFLOP/s, elapsed ms) of an MMA-only loop on every SM."""
    k = {"tf32": 0, "bf16": 1, "fp16": 2}[kind]
    t, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().qsim_tc_peak(k, int(n_cols), float(seconds), ctypes.byref(t), ctypes.byref(ms)))
    return t.value, ms.value


def fp64_peak(seconds: float = 1.0):
    """Measured FP64 FMA rate (TFLOP/s, elapsed ms) of independent FMA chains on every SM."""
    t, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().qsim_fp64_peak(float(seconds), ctypes.byref(t), ctypes.byref(ms)))
    return t.value, ms.value


class Batch:
    """Many independent circuits (each from |0...0>, complex64) in one persistent launch; returns the
    per-circuit <Z_q> and <Z_q Z_{q+1}>. With a tensor-core precision, circuits of at least tc_min_n qubits
    (0 = 20) run as fused tensor-core plans in the same enqueue."""

    def __init__(self, circuits, max_fused: int = 0, stream=None, precision: int = 0, tc_min_n: int = 0):
        import torch
        self.circuits = list(circuits)
        self.args = CircuitsArgs(self.circuits)
        arr = self.args.arr
        ws = ctypes.c_size_t()
        _check(lib().qsim_batch_workspace_bytes(arr, self.args.count, ctypes.byref(ws)))
        self.ws_bytes = ws.value
        self.ws = torch.empty(max(1, self.ws_bytes // 8), dtype=torch.complex64, device="cuda")
        o = RunOpts(mode=RUN_FUSED, max_fused=max_fused, precision=precision, batch_tc_min_n=tc_min_n)
        info = PlanInfo()
        b = ctypes.c_void_p()
        _check(lib().qsim_batch_plan_create(arr, self.args.count, ctypes.byref(o),
                                            ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(b), ctypes.byref(info)))
        self.b = b
        self.info = info.as_dict()
        self.stream = stream
        self.nzi = sum(c.n for c in self.circuits)
        self.nzz = sum(max(0, c.n - 1) for c in self.circuits)

    def execute(self, use_graph: bool = False):
        _check(lib().qsim_batch_execute(self.b, ctypes.c_void_p(self.ws.data_ptr()), self.ws_bytes,
                                        ctypes.c_void_p(_stream_ptr(self.stream)), 1 if use_graph else 0))

    def results(self):
        zi = np.zeros(max(1, self.nzi))
        zz = np.zeros(max(1, self.nzz))
        _check(lib().qsim_batch_results(self.b, ctypes.c_void_p(_stream_ptr(self.stream)), _dptr(zi), _dptr(zz)))
        out, a, b = [], 0, 0
        for c in self.circuits:
            out.append((zi[a:a + c.n].copy(), zz[b:b + c.n - 1].copy()))
            a += c.n
            b += max(0, c.n - 1)
        return out

    def close(self):
        if getattr(self, "b", None):
            lib().qsim_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_run(circuits, max_fused: int = 0, precision: int = 0, tc_min_n: int = 0, stream=None):
    """Plan, run and read out a batch in one call (qsim_batch_run): the GPU starts on the circuits already
    planned while the host plans the others. Returns (per-circuit (<Z_q>, <Z_q Z_{q+1}>), plan info)."""
    import torch
    circuits = list(circuits)
    args = CircuitsArgs(circuits)
    ws = ctypes.c_size_t()
    _check(lib().qsim_batch_workspace_bytes(args.arr, args.count, ctypes.byref(ws)))
    buf = torch.empty(max(1, ws.value // 8), dtype=torch.complex64, device="cuda") if ws.value else None
    o = RunOpts(mode=RUN_FUSED, max_fused=max_fused, precision=precision, batch_tc_min_n=tc_min_n)
    nzi = sum(c.n for c in circuits)
    nzz = sum(max(0, c.n - 1) for c in circuits)
    zi = np.zeros(max(1, nzi))
    zz = np.zeros(max(1, nzz))
    info = PlanInfo()
    _check(lib().qsim_batch_run(args.arr, args.count, ctypes.byref(o),
                                ctypes.c_void_p(buf.data_ptr() if buf is not None else 0), ws.value,
                                ctypes.c_void_p(_stream_ptr(stream)), _dptr(zi), _dptr(zz), ctypes.byref(info)))
    out, a, b = [], 0, 0
    for c in circuits:
        out.append((zi[a:a + c.n].copy(), zz[b:b + c.n - 1].copy()))
        a += c.n
        b += max(0, c.n - 1)
    return out, info.as_dict()


def batch_autotune(circuits, stream=None):
    """Tune the batched fusion width per qubit count; returns the k each circuit now gets."""
    args = CircuitsArgs(circuits)
    chosen = (ctypes.c_int * max(1, args.count))()
    _check(lib().qsim_batch_autotune(args.arr, args.count, ctypes.c_void_p(_stream_ptr(stream)), chosen))
    return list(chosen)[:args.count]


def batch_autotune_threshold(circuits, precision: int = PREC_TF32X3, stream=None) -> int:
    """Tune (and keep process-wide) the width from which batched circuits run as tensor-core plans."""
    args = CircuitsArgs(circuits)
    best = ctypes.c_int()
    _check(lib().qsim_batch_autotune_threshold(args.arr, args.count, int(precision),
                                               ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(best)))
    return best.value


def batch_tune_save(path: str) -> None:
    _check(lib().qsim_batch_tune_save(os.fsencode(path)))


def batch_tune_load(path: str) -> None:
    _check(lib().qsim_batch_tune_load(os.fsencode(path)))
