"""FP64 oracle: a plain, slow, obviously correct CPU state-vector simulator (C, via ctypes).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The GPU library neither imports nor links it.

Every function computes the plain definition of its quantity (see ``oracle.c``):
  * ``run`` / ``apply_gate``  -- the per-gate operator I (x) U (x) I with controls (paper Sec. 2.1,
    "State-Vector Simulation");
  * ``dense_operator``        -- the same operator built as a full 2^n x 2^n matrix (n <= 10), an
    independent brute-force path;
  * ``probs``, ``norm2``, ``expect_pauli``, ``inner`` -- observables (Sec. 2.1 "Measurement and
    Sampling"; Sec. 2.5 "sampling and calculation of expectation values");
  * ``sample`` -- inverse-CDF sampling from |psi_x|^2 given uniforms; ``uniforms`` -- SplitMix64.
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, Sequence

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        c_int, c_dbl, c_u64, c_i64 = ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_int64
        vp = ctypes.c_void_p
        L.oracle_apply_gate.argtypes = [c_int, vp, c_int, P(c_int), c_int, P(c_int), vp]
        L.oracle_apply_gate.restype = c_int
        L.oracle_dense_operator.argtypes = [c_int, c_int, P(c_int), c_int, P(c_int), vp, vp]
        L.oracle_dense_operator.restype = c_int
        L.oracle_dense_matvec.argtypes = [c_int, vp, vp]
        L.oracle_dense_matvec.restype = c_int
        L.oracle_norm2.argtypes = [c_int, vp]
        L.oracle_norm2.restype = c_dbl
        L.oracle_probs.argtypes = [c_int, vp, c_int, P(c_int), vp]
        L.oracle_probs.restype = c_int
        L.oracle_expect_pauli.argtypes = [c_int, vp, ctypes.c_char_p, vp]
        L.oracle_expect_pauli.restype = c_int
        L.oracle_inner.argtypes = [c_int, vp, vp, vp]
        L.oracle_inner.restype = None
        L.oracle_splitmix64.argtypes = [c_u64, c_u64]
        L.oracle_splitmix64.restype = c_u64
        L.oracle_uniforms.argtypes = [c_u64, c_i64, vp]
        L.oracle_uniforms.restype = None
        L.oracle_sample.argtypes = [c_int, vp, c_i64, vp, vp]
        L.oracle_sample.restype = c_int
        L.oracle_num_threads.argtypes = []
        L.oracle_num_threads.restype = c_int
        L.oracle_set_num_threads.argtypes = [c_int]
        L.oracle_set_num_threads.restype = None
        _lib = L
    return _lib


def _ints(xs: Iterable[int]):
    xs = list(xs)
    arr = (ctypes.c_int * max(1, len(xs)))(*xs)
    return arr, len(xs)


def _state(psi: np.ndarray) -> np.ndarray:
    if psi.dtype != np.complex128 or not psi.flags.c_contiguous:
        raise TypeError("oracle states are C-contiguous complex128 arrays")
    return psi


def num_threads() -> int:
    return lib().oracle_num_threads()


def set_num_threads(t: int) -> None:
    lib().oracle_set_num_threads(int(t))


def basis(n: int, x: int = 0) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[x] = 1.0
    return psi


def apply_gate(psi: np.ndarray, n: int, targets: Sequence[int], controls: Sequence[int], U: np.ndarray) -> None:
    """In place: psi <- (U on targets, controlled on controls = 1) psi."""
    _state(psi)
    U = np.ascontiguousarray(U, dtype=np.complex128)
    t, k = _ints(targets)
    c, nc = _ints(controls)
    if U.shape != (1 << k, 1 << k):
        raise ValueError("matrix shape does not match the number of targets")
    rc = lib().oracle_apply_gate(n, psi.ctypes.data, k, t, nc, c, U.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle_apply_gate rejected targets={tuple(targets)} controls={tuple(controls)}")


def run(circuit, psi: np.ndarray | None = None, basis_state: int = 0) -> np.ndarray:
    """Apply every gate of ``circuit`` (a workloads.Circuit) in order; returns the state (new array
    unless ``psi`` is given, which is updated in place)."""
    n = circuit.n
    if psi is None:
        psi = basis(n, basis_state)
    for g in circuit.gates:
        apply_gate(psi, n, g.targets, g.controls, g.matrix)
    return psi


def dense_operator(n: int, targets, controls, U) -> np.ndarray:
    U = np.ascontiguousarray(U, dtype=np.complex128)
    t, k = _ints(targets)
    c, nc = _ints(controls)
    G = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    rc = lib().oracle_dense_operator(n, k, t, nc, c, U.ctypes.data, G.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_dense_operator rejected its arguments")
    return G


def dense_run(circuit, psi: np.ndarray | None = None) -> np.ndarray:
    """Brute force: each gate as a full 2^n x 2^n operator times the vector (n <= 10)."""
    n = circuit.n
    if psi is None:
        psi = basis(n, 0)
    for g in circuit.gates:
        G = dense_operator(n, g.targets, g.controls, g.matrix)
        rc = lib().oracle_dense_matvec(n, G.ctypes.data, psi.ctypes.data)
        if rc != 0:
            raise ValueError("oracle_dense_matvec failed")
    return psi


def norm2(psi: np.ndarray, n: int) -> float:
    return float(lib().oracle_norm2(n, _state(psi).ctypes.data))


def probs(psi: np.ndarray, n: int, qubits: Sequence[int]) -> np.ndarray:
    q, nq = _ints(qubits)
    out = np.zeros(1 << nq, dtype=np.float64)
    rc = lib().oracle_probs(n, _state(psi).ctypes.data, nq, q, out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_probs rejected its arguments")
    return out


def expect_pauli(psi: np.ndarray, n: int, paulis: str) -> complex:
    if len(paulis) != n:
        raise ValueError("Pauli string length must equal n")
    out = np.zeros(2, dtype=np.float64)
    rc = lib().oracle_expect_pauli(n, _state(psi).ctypes.data, paulis.encode(), out.ctypes.data)
    if rc != 0:
        raise ValueError("bad Pauli string")
    return complex(out[0], out[1])


def z_string(n: int, qubits: Sequence[int]) -> str:
    s = ["I"] * n
    for q in qubits:
        s[q] = "Z"
    return "".join(s)


def expect_z_chain(psi: np.ndarray, n: int):
    """<Z_i> for every qubit and <Z_i Z_{i+1}> for every bond of the open chain."""
    zi = np.array([expect_pauli(psi, n, z_string(n, [i])).real for i in range(n)])
    zz = np.array([expect_pauli(psi, n, z_string(n, [i, i + 1])).real for i in range(n - 1)])
    return zi, zz


def inner(a: np.ndarray, b: np.ndarray, n: int) -> complex:
    out = np.zeros(2, dtype=np.float64)
    lib().oracle_inner(n, _state(a).ctypes.data, _state(b).ctypes.data, out.ctypes.data)
    return complex(out[0], out[1])


def splitmix64(seed: int, i: int) -> int:
    return int(lib().oracle_splitmix64(seed & (2**64 - 1), i))


def uniforms(seed: int, count: int) -> np.ndarray:
    out = np.zeros(count, dtype=np.float64)
    lib().oracle_uniforms(seed & (2**64 - 1), int(count), out.ctypes.data)
    return out


def sample(psi: np.ndarray, n: int, u: np.ndarray) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(len(u), dtype=np.uint64)
    rc = lib().oracle_sample(n, _state(psi).ctypes.data, len(u), u.ctypes.data, out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_sample rejected its arguments")
    return out


def infidelity(psi_a: np.ndarray, psi_b: np.ndarray, n: int, normalised: bool = True) -> float:
    """1 - |<a|b>|^2, normalised by the two norms when ``normalised`` (the state-fidelity reading)."""
    ov = inner(psi_a, psi_b, n)
    f = abs(ov) ** 2
    if normalised:
        f /= norm2(psi_a, n) * norm2(psi_b, n)
    return 1.0 - f
