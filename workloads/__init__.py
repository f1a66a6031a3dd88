"""Seeded synthetic circuit generators.

This module produces *inputs* only: gate lists (targets, controls, FP64 unitary matrices) and basis-state
indices. It performs no state-vector arithmetic, so both the FP64 oracle and the GPU library consume its
output as plain data.

Conventions (the paper does not fix them; these are the readings used throughout):
  * qubit q is bit q of the amplitude index (little-endian);
  * for a gate on targets (t_0, ..., t_{k-1}) the matrix row/column index is m = sum_j bit_{t_j} * 2^j;
  * matrices are 2^k x 2^k complex128, row-major; controls fire on |1>.

Workloads follow the paper's benchmark descriptions (Sec. 2.2 "Benchmarks"): random circuits with CZ and
single-qubit rotations, Trotterised transverse-field Ising evolution (Eq. 1), and the QFT that sits inside
QPE. All randomness comes from numpy's PCG64 generator seeded explicitly.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

__all__ = [
    "Gate", "Circuit", "haar_unitary", "H", "X", "Y", "Z", "RX", "RY", "RZ", "CZ", "CP", "RZZ", "SWAP",
    "brickwork", "qft", "tfim_chain", "random_pairs", "rcs", "ghz", "random_gate", "inverse",
    "tfim_batch", "basis_index", "qpe",
]


@dataclass
class Gate:
    targets: Tuple[int, ...]
    controls: Tuple[int, ...]
    matrix: np.ndarray  # (2^k, 2^k) complex128
    name: str = "u"

    @property
    def k(self) -> int:
        return len(self.targets)

    @property
    def qubits(self) -> Tuple[int, ...]:
        return tuple(self.targets) + tuple(self.controls)


@dataclass
class Circuit:
    n: int
    gates: List[Gate] = field(default_factory=list)
    name: str = ""

    def __len__(self) -> int:
        return len(self.gates)

    def append(self, g: Gate) -> None:
        self.gates.append(g)


# ---------------------------------------------------------------------------------------------------------
# Gate matrices (standard textbook forms; the paper defers to the CUDA-Q documentation, Sec. 2.2 "Random
# Circuits", which is not available, so the usual definitions are used).
# ---------------------------------------------------------------------------------------------------------
_S2 = 1.0 / math.sqrt(2.0)


def H() -> np.ndarray:
    return np.array([[_S2, _S2], [_S2, -_S2]], dtype=np.complex128)


def X() -> np.ndarray:
    return np.array([[0, 1], [1, 0]], dtype=np.complex128)


def Y() -> np.ndarray:
    return np.array([[0, -1j], [1j, 0]], dtype=np.complex128)


def Z() -> np.ndarray:
    return np.array([[1, 0], [0, -1]], dtype=np.complex128)


def RX(theta: float) -> np.ndarray:
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)


def RY(theta: float) -> np.ndarray:
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def RZ(theta: float) -> np.ndarray:
    return np.diag([np.exp(-0.5j * theta), np.exp(0.5j * theta)]).astype(np.complex128)


def CZ() -> np.ndarray:
    return np.diag([1, 1, 1, -1]).astype(np.complex128)


def CP(lam: float) -> np.ndarray:
    """Phase gate diag(1, e^{i lam}) — used with one control qubit to form the controlled phase."""
    return np.diag([1, np.exp(1j * lam)]).astype(np.complex128)


def RZZ(theta: float) -> np.ndarray:
    """exp(-i theta Z(x)Z / 2): the Ising coupling term of Eq. 1 under a Trotter step."""
    a, b = np.exp(-0.5j * theta), np.exp(0.5j * theta)
    return np.diag([a, b, b, a]).astype(np.complex128)


def SWAP() -> np.ndarray:
    m = np.zeros((4, 4), dtype=np.complex128)
    m[0, 0] = m[3, 3] = 1
    m[1, 2] = m[2, 1] = 1
    return m


def haar_unitary(d: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed U(d): QR of a complex Ginibre matrix with the phases of diag(R) divided out
    (Mezzadri, Notices AMS 54, 2007)."""
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return (q * ph[None, :]).astype(np.complex128)


def inverse(c: Circuit) -> Circuit:
    """The adjoint circuit: gates in reverse order with conjugate-transposed matrices (paper Sec. 2.1:
    every unitary is reversible, A^-1 = A^dagger)."""
    out = Circuit(c.n, name=c.name + "^dagger")
    for g in reversed(c.gates):
        out.append(Gate(g.targets, g.controls, np.ascontiguousarray(g.matrix.conj().T), g.name + "^dg"))
    return out


# ---------------------------------------------------------------------------------------------------------
# Circuit families
# ---------------------------------------------------------------------------------------------------------
def brickwork(n: int, depth: int, seed: int, both_pairs: bool = False) -> Circuit:
    """Random brickwork: each layer applies a Haar U(2) to every qubit, then CZ on nearest-neighbour pairs.
    Even layers use pairs (0,1),(2,3),...; odd layers use (1,2),(3,4),... (both sets per layer when
    ``both_pairs``). Stands in for the paper's random-circuit benchmark (Sec. 2.2)."""
    rng = np.random.default_rng(seed)
    c = Circuit(n, name=f"brickwork_n{n}_d{depth}_s{seed}")
    for layer in range(depth):
        for q in range(n):
            c.append(Gate((q,), (), haar_unitary(2, rng), "u2"))
        starts = (0, 1) if both_pairs else ((layer % 2),)
        for s in starts:
            for a in range(s, n - 1, 2):
                c.append(Gate((a, a + 1), (), CZ(), "cz"))
    return c


def qft(n: int, swaps: bool = True) -> Circuit:
    """QFT|x> = 2^{-n/2} sum_y exp(+2 pi i x y / 2^n) |y>. For q = n-1 down to 0: H(q), then the
    controlled phase CP(pi / 2^{q-j}) with control j and target q for j = q-1 down to 0; finally
    SWAP(q, n-1-q) for q < n/2. The inverse of this circuit is the inverse QFT used by QPE (Sec. 2.2)."""
    c = Circuit(n, name=f"qft_n{n}")
    for q in range(n - 1, -1, -1):
        c.append(Gate((q,), (), H(), "h"))
        for j in range(q - 1, -1, -1):
            c.append(Gate((q,), (j,), CP(math.pi / (1 << (q - j))), "cp"))
    if swaps:
        for q in range(n // 2):
            c.append(Gate((q, n - 1 - q), (), SWAP(), "swap"))
    return c


def basis_index(n: int, seed: int) -> int:
    """A seeded random computational basis state index in [0, 2^n)."""
    rng = np.random.default_rng(seed)
    return int(rng.integers(0, 1 << 62, dtype=np.int64)) % (1 << n)


def tfim_chain(n: int, steps: int, theta: float, phi: float) -> Circuit:
    """First-order Trotterisation of Eq. 1 on an open 1-D chain: each step applies RZZ(theta) on every
    bond (i, i+1), then RX(phi) on every qubit (theta = 2 J dt, phi = 2 h dt)."""
    c = Circuit(n, name=f"tfim_n{n}_s{steps}")
    zz, rx = RZZ(theta), RX(phi)
    for _ in range(steps):
        for i in range(n - 1):
            c.append(Gate((i, i + 1), (), zz, "rzz"))
        for i in range(n):
            c.append(Gate((i,), (), rx, "rx"))
    return c


def tfim_batch(count: int, seed: int, nmin: int = 10, nmax: int = 24, smin: int = 8, smax: int = 32):
    """``count`` TFIM chains with widths ~ U{nmin..nmax}, Trotter steps ~ U{smin..smax} and angles
    theta, phi ~ U(0, pi), one (theta, phi) per circuit. Returns a list of (Circuit, theta, phi)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        s = int(rng.integers(smin, smax + 1))
        th = float(rng.uniform(0.0, math.pi))
        ph = float(rng.uniform(0.0, math.pi))
        out.append((tfim_chain(n, s, th, ph), th, ph))
    return out


def triangular_bonds(lx: int, ly: int) -> List[Tuple[int, int]]:
    """Bonds of an lx x ly triangular lattice with periodic boundaries (site (x, y) is qubit y * lx + x):
    each site couples to (x+1, y), (x, y+1) and (x+1, y+1), wrapping around; duplicate bonds of narrow
    lattices are kept once. 3 lx ly bonds when lx, ly >= 3."""
    bonds = []
    seen = set()
    for y in range(ly):
        for x in range(lx):
            a = y * lx + x
            for dx, dy in ((1, 0), (0, 1), (1, 1)):
                b = ((y + dy) % ly) * lx + (x + dx) % lx
                key = (min(a, b), max(a, b))
                if a != b and key not in seen:
                    seen.add(key)
                    bonds.append(key)
    return bonds


def tfim_lattice(lx: int, ly: int, steps: int, theta: float, phi: float) -> Circuit:
    """First-order Trotter evolution under Eq. 1 on a periodic triangular lattice (Sec. 2.2's HamLib TFIM is
    a 2-D lattice of this kind; its data file is not available): each step applies RZZ(theta) on every bond,
    then RX(phi) on every site (theta = 2 J dt, phi = 2 h dt), from |0...0>."""
    n = lx * ly
    c = Circuit(n, name=f"tfim_tri_{lx}x{ly}_s{steps}")
    zz, rx = RZZ(theta), RX(phi)
    bonds = triangular_bonds(lx, ly)
    for _ in range(steps):
        for a, b in bonds:
            c.append(Gate((a, b), (), zz, "rzz"))
        for q in range(n):
            c.append(Gate((q,), (), rx, "rx"))
    return c


def random_pairs(n: int, depth: int, seed: int) -> Circuit:
    """Each layer is a seeded random perfect matching of the n qubits (n even; one qubit idles when odd)
    with a Haar U(4) on every pair, so most gates span high-order qubits."""
    rng = np.random.default_rng(seed)
    c = Circuit(n, name=f"pairs_n{n}_d{depth}_s{seed}")
    for _ in range(depth):
        perm = rng.permutation(n)
        for i in range(0, n - 1, 2):
            a, b = int(perm[i]), int(perm[i + 1])
            c.append(Gate((a, b), (), haar_unitary(4, rng), "u4"))
    return c


def rcs(n: int, seed: int, gates_per_qubit: int = 30) -> Circuit:
    """The paper's random-circuit script (Sec. 2.2): 30n gates on random qubits; a CZ with probability
    0.25, otherwise one of H, RX, RY, RZ. Rotation angles ~ U(0, 2 pi) (the paper does not state them)."""
    rng = np.random.default_rng(seed)
    c = Circuit(n, name=f"rcs_n{n}_s{seed}")
    for _ in range(gates_per_qubit * n):
        if n > 1 and rng.random() < 0.25:
            a, b = rng.choice(n, size=2, replace=False)
            c.append(Gate((int(a), int(b)), (), CZ(), "cz"))
        else:
            q = int(rng.integers(0, n))
            kind = int(rng.integers(0, 4))
            if kind == 0:
                c.append(Gate((q,), (), H(), "h"))
            else:
                th = float(rng.uniform(0.0, 2 * math.pi))
                m = (RX, RY, RZ)[kind - 1](th)
                c.append(Gate((q,), (), m, ("rx", "ry", "rz")[kind - 1]))
    return c


def ghz(n: int) -> Circuit:
    """H on qubit 0, then CNOT(0 -> i) for i = 1..n-1."""
    c = Circuit(n, name=f"ghz_n{n}")
    c.append(Gate((0,), (), H(), "h"))
    for i in range(1, n):
        c.append(Gate((i,), (0,), X(), "cx"))
    return c


def random_gate(n: int, rng: np.random.Generator, kmax: int = 3, cmax: int = 2, diag_prob: float = 0.0) -> Gate:
    """A random gate: k ~ U{1..kmax} targets in random (unsorted) order, c ~ U{0..cmax} controls, Haar U(2^k)
    or, with probability ``diag_prob``, a random diagonal unitary with some entries exactly 1."""
    k = int(rng.integers(1, min(kmax, n) + 1))
    c = int(rng.integers(0, min(cmax, n - k) + 1))
    qs = rng.permutation(n)[: k + c]
    t = tuple(int(x) for x in qs[:k])
    ctl = tuple(int(x) for x in qs[k:])
    if rng.random() < diag_prob:
        ph = np.exp(1j * rng.uniform(0, 2 * math.pi, size=1 << k))
        ph[rng.random(1 << k) < 0.5] = 1.0
        m = np.diag(ph).astype(np.complex128)
        return Gate(t, ctl, m, "diag")
    return Gate(t, ctl, haar_unitary(1 << k, rng), "u")


def qpe(n_count: int, phase_numerator: int) -> Tuple[Circuit, int]:
    """Quantum phase estimation with an exactly representable phase phi = a / 2^t (Sec. 2.2 "QPE"):
    t = n_count counting qubits (0..t-1) and one eigenstate qubit t prepared in |1> of U = P(2 pi phi).
    Controlled-U^(2^j) by counting qubit j, then the inverse QFT on the counting register. Returns the
    circuit and the expected outcome a of the counting register."""
    t = n_count
    n = t + 1
    phi = phase_numerator / float(1 << t)
    c = Circuit(n, name=f"qpe_t{t}_a{phase_numerator}")
    c.append(Gate((t,), (), X(), "x"))
    for j in range(t):
        c.append(Gate((j,), (), H(), "h"))
    for j in range(t):
        lam = 2 * math.pi * phi * (1 << j)
        c.append(Gate((t,), (j,), CP(lam), "cu"))
    inv = inverse(qft(t, swaps=True))
    for g in inv.gates:
        c.append(g)
    return c, phase_numerator % (1 << t)
