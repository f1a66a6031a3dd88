"""Shared test helpers: build golden circuits from their JSON description, compare states."""
import json
import math
import os

import numpy as np

import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(name="closed_forms.json"):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def golden_circuit(case):
    """Turn a golden case's gate list ([name, targets, controls, params]) into a workloads.Circuit."""
    n = case["n"]
    c = W.Circuit(n, name=case["name"])
    for name, t, ctl, par in case["gates"]:
        t, ctl = tuple(t), tuple(ctl)
        if name == "qft":
            for g in W.qft(n).gates:
                c.append(g)
            continue
        if name == "qpe":
            qc, _ = W.qpe(int(par[0]), int(par[1]))
            for g in qc.gates:
                c.append(g)
            continue
        m = {
            "h": lambda: W.H(), "x": lambda: W.X(), "y": lambda: W.Y(), "z": lambda: W.Z(),
            "swap": lambda: W.SWAP(), "cz": lambda: W.CZ(),
            "cp": lambda: W.CP(par[0]), "rz": lambda: W.RZ(par[0]), "rx": lambda: W.RX(par[0]),
            "ry": lambda: W.RY(par[0]), "rzz": lambda: W.RZZ(par[0]),
        }[name]()
        c.append(W.Gate(t, ctl, m, name))
    return c


def golden_amps(case):
    return np.array([complex(a, b) for a, b in case["amps"]], dtype=np.complex128)


def qft_closed_form(n, x):
    """QFT|x> amplitudes with the phase reduced exactly in integers: 2 pi ((x*y) mod 2^n) / 2^n."""
    N = 1 << n
    y = np.arange(N, dtype=np.uint64)
    ph = (np.uint64(x) * y) & np.uint64(N - 1)  # exact: x*y < 2^64 for n <= 32
    return np.exp(2j * math.pi * ph.astype(np.float64) / N) / math.sqrt(N)


def random_state(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return (v / np.linalg.norm(v)).astype(np.complex128)


def pauli_dense(paulis):
    """Dense Pauli-string operator via numpy kron; character q acts on qubit q (bit q), so the
    leftmost Kronecker factor is qubit n-1."""
    mats = {"I": np.eye(2), "X": W.X(), "Y": W.Y(), "Z": W.Z()}
    op = np.array([[1.0 + 0j]])
    for ch in reversed(paulis):
        op = np.kron(op, mats[ch])
    return op
