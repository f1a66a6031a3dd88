"""The phase pass: runs of 1- and 2-qubit diagonal gates on any qubits in one pass (a quadratic form of the
index bits per amplitude), against the FP64 oracle through the C ABI.

Tolerances: complex64 max |amplitude error| <= 1e-5 and normalised infidelity <= 1e-9; complex128 max
|amplitude error| <= 1e-12.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qsim(gpu_lib):
    from paper_2511_14664_gb300 import qsim as q
    return q


def diag2(rng):
    return np.diag(np.exp(1j * rng.uniform(0, 2 * math.pi, size=4))).astype(np.complex128)


def diagonal_run(n, count, rng):
    """`count` random diagonal gates of every kind the phase pass takes, on qubits drawn from the whole
    register (lane bits 0-4, bits 5-9 and the high bits of the kernel's ranges all appear)."""
    gates = []
    for _ in range(count):
        a, b = (int(x) for x in rng.choice(n, size=2, replace=False))
        kind = int(rng.integers(0, 7))
        th = float(rng.uniform(0, 2 * math.pi))
        if kind == 0:
            gates.append(W.Gate((a, b), (), W.CZ(), "cz"))
        elif kind == 1:  # controlled phase as a 2-target diagonal
            gates.append(W.Gate((a, b), (), np.diag([1.0, 1.0, 1.0, np.exp(1j * th)]).astype(np.complex128), "cp"))
        elif kind == 2:  # controlled phase written as a control and a 1-qubit diagonal target
            gates.append(W.Gate((b,), (a,), W.CP(th), "cphase"))
        elif kind == 3:
            gates.append(W.Gate((a,), (), W.RZ(th), "rz"))
        elif kind == 4:
            gates.append(W.Gate((a, b), (), W.RZZ(th), "rzz"))
        elif kind == 5:
            gates.append(W.Gate((b,), (a,), W.RZ(th), "crz"))
        else:
            gates.append(W.Gate((a, b), (), diag2(rng), "diag2"))
    return gates


def circuit_with_runs(n, seed):
    rng = np.random.default_rng(seed)
    c = W.Circuit(n, name=f"phase_runs_n{n}")
    for q in range(n):
        c.append(W.Gate((q,), (), W.haar_unitary(2, rng), "u"))
    for g in diagonal_run(n, 40, rng):
        c.append(g)
    for q in range(0, n, 3):
        c.append(W.Gate((q,), (), W.H(), "h"))
    for g in diagonal_run(n, 25, rng):
        c.append(g)
    return c


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n", [10, 13, 17])
def test_phase_pass_against_oracle(qsim, dtype, n):
    c = circuit_with_runs(n, seed=n * 3 + dtype)
    p = qsim.Plan(c, dtype, mode=qsim.RUN_FUSED, max_fused=3)
    kinds = [q["kind"] for q in p.passes()]
    assert "phase" in kinds, kinds
    st = qsim.State(n, dtype)
    st.set_basis(0)
    p.execute(st)
    g = st.get_state().astype(np.complex128)
    ref = oracle.run(c)
    err = float(np.max(np.abs(g - ref)))
    if dtype == 0:
        assert err <= 1e-5, err
        assert oracle.infidelity(np.ascontiguousarray(g), ref, n) <= 1e-9
    else:
        assert err <= 1e-12, err


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_phase_pass_graph_replay_and_qft(qsim, prec):
    """The QFT's controlled phases gather in phase passes, each folded into the epilogue of the tensor-core
    block before it (3xTF32, BF16x3; BF16x6 keeps them as passes); a replayed graph gives the closed form."""
    n = 16
    x = W.basis_index(n, 4)
    c = W.qft(n)
    p = qsim.Plan(c, qsim.C64, mode=qsim.RUN_FUSED, max_fused=6, precision=prec, tc_min_k=5, use_graph=True)
    kinds = [q["kind"] for q in p.passes()]
    assert sum(q["gates"] for q in p.passes()) == len(c)
    if prec == 3:
        assert "phase" in kinds
    else:
        assert len(kinds) < 13 and "tc" in kinds, kinds
    st = qsim.State(n, qsim.C64)
    y = np.arange(1 << n, dtype=np.uint64)
    ph = (np.uint64(x) * y) & np.uint64((1 << n) - 1)
    ref = np.exp(2j * math.pi * ph.astype(np.float64) / (1 << n)) / math.sqrt(1 << n)
    for _ in range(3):
        st.set_basis(x)
        p.execute(st)
        got = st.get_state().astype(np.complex128)
        assert float(np.max(np.abs(got - ref))) <= 1e-5


def layers_then_diagonals(n, seed, rounds=3):
    """Rounds of a Haar U(2) on every qubit followed by a run of random diagonal gates on any qubits: the
    fused plan puts 6-qubit tensor-core blocks right before phase passes, which become their epilogues."""
    rng = np.random.default_rng(seed)
    c = W.Circuit(n, name=f"layers_diag_n{n}")
    for _ in range(rounds):
        for q in range(n):
            c.append(W.Gate((q,), (), W.haar_unitary(2, rng), "u"))
        for g in diagonal_run(n, 50, rng):
            c.append(g)
    return c


@pytest.mark.parametrize("prec,inf_tol", [(1, 1e-9), (2, 1e-6)])
@pytest.mark.parametrize("n", [13, 21])
def test_phase_epilogue_on_tensor_core_blocks(qsim, prec, inf_tol, n):
    c = layers_then_diagonals(n, seed=n + 10 * prec)
    p = qsim.Plan(c, qsim.C64, mode=qsim.RUN_FUSED, max_fused=6, precision=prec, tc_min_k=5)
    passes = p.passes()
    assert sum(q["gates"] for q in passes) == len(c)
    assert "tc" in [q["kind"] for q in passes]
    st = qsim.State(n, qsim.C64)
    st.set_basis(0)
    p.execute(st)
    g = st.get_state().astype(np.complex128)
    ref = oracle.run(c)
    assert float(np.max(np.abs(g - ref))) <= 1e-5
    assert oracle.infidelity(np.ascontiguousarray(g), ref, n) <= inf_tol


@pytest.mark.parametrize("targets", [(0, 1, 2, 3, 4, 5), (0, 2, 4, 6, 8, 10), (7, 8, 9, 10, 11, 12), (1, 3, 9, 14, 15, 20)])
def test_phase_epilogue_each_data_path(qsim, targets):
    """One 6-qubit block (32-byte, 16-byte and 8-byte data paths) followed by diagonal gates on every kind of
    bit (rows, columns, the half bit, tile bits): the epilogue against the oracle."""
    n = 21
    rng = np.random.default_rng(sum(targets))
    c = W.Circuit(n, name="block_then_phase")
    c.append(W.Gate(targets, (), W.haar_unitary(64, rng), "u64"))
    for g in diagonal_run(n, 60, rng):
        c.append(g)
    p = qsim.Plan(c, qsim.C64, mode=qsim.RUN_FUSED, max_fused=6, precision=1, tc_min_k=5)
    kinds = [q["kind"] for q in p.passes()]
    assert kinds == ["tc"], kinds
    st = qsim.State(n, qsim.C64)
    psi0 = np.random.default_rng(4).standard_normal((1 << n, 2)) @ np.array([1, 1j])
    psi0 = (psi0 / np.linalg.norm(psi0)).astype(np.complex128)
    st.set_state(psi0)
    p.execute(st)
    ref = psi0.copy()
    for gt in c.gates:
        oracle.apply_gate(ref, n, gt.targets, gt.controls, gt.matrix)
    g = st.get_state().astype(np.complex128)
    assert float(np.max(np.abs(g - ref))) <= 1e-5
    assert oracle.infidelity(np.ascontiguousarray(g), ref, n) <= 1e-9


def test_plain_plans_keep_one_pass_per_gate(qsim):
    n = 12
    c = circuit_with_runs(n, seed=8)
    p = qsim.Plan(c, qsim.C64, mode=qsim.RUN_PLAIN, max_fused=1)
    kinds = [q["kind"] for q in p.passes()]
    assert len(kinds) == len(c) and "phase" not in kinds


def test_phase_pass_not_used_with_global_qubits(qsim):
    """Plans with global qubits keep diagonal blocks within the fusion width (their tables name physical
    positions, which reorder passes move)."""
    n = 14
    c = circuit_with_runs(n, seed=5)
    p = qsim.Plan(c, qsim.C64, mode=qsim.RUN_FUSED, max_fused=3, local_qubits=11)
    assert all(q["kind"] != "phase" for q in p.passes())
    st = qsim.State(n, qsim.C64)
    st.set_basis(0)
    p.execute(st)
    g = st.get_state().astype(np.complex128)
    ref = oracle.run(c)
    assert float(np.max(np.abs(g - ref))) <= 1e-5
