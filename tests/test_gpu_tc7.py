"""Seven-qubit tensor-core blocks (QSIM_PREC_FP16X3 with k = 7: FP16 split products, B stacked as
[Im U; Re U; -Im U]) against the FP64 oracle, at the complex64 bar: max |amplitude error| <= 1e-5 and
normalised infidelity <= 1e-9.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from helpers import random_state

pytestmark = pytest.mark.gpu

FP16X3, TF32X3 = 4, 1


@pytest.fixture(scope="module")
def qsim(gpu_lib):
    from paper_2511_14664_gb300 import qsim as q
    return q


def check(psi_gpu, ref, n):
    g = np.ascontiguousarray(psi_gpu.astype(np.complex128))
    err = float(np.max(np.abs(g - ref)))
    inf = oracle.infidelity(g, ref, n)
    assert err <= 1e-5, f"max amplitude error {err:.3e}"
    assert inf <= 1e-9, f"infidelity {inf:.3e}"
    return err, inf


# target lists (in the order given, which fixes U's column bits) for each data path of the kernel
TARGETS = {
    "rows_high": (7, 8, 9, 10, 11, 12, 13),   # rows are qubits 0..6: whole 256-byte runs per warp access
    "rows_q3": (3, 4, 6, 8, 10, 12, 13),      # targets from qubit 3 up (the planner's 7-qubit blocks)
    "rows_mixed": (2, 5, 8, 9, 11, 3, 13),    # unsorted, qubits 2 and 3 among them
    "rows_q1": (1, 4, 6, 8, 10, 12, 13),      # qubit 1 but not 0
    "rows_q0_later": (5, 0, 1, 7, 9, 11, 13), # qubit 0 a target but not the first: rows path
    "pairs": (0, 2, 3, 5, 9, 12, 13),         # qubit 0 first: 16-byte pairs
    "quads": (0, 1, 4, 6, 7, 10, 13),         # qubits 0, 1 first: 32-byte quads
    "low7": (0, 1, 2, 3, 4, 5, 6),
    "descending": (13, 12, 11, 10, 9, 8, 7),
}


@pytest.mark.parametrize("name", list(TARGETS))
@pytest.mark.parametrize("n", [14, 15, 21])
def test_single_block_against_oracle(qsim, name, n):
    """One tile (n = 14), two tiles, and one tile per CTA (n = 21)."""
    t = TARGETS[name]
    rng = np.random.default_rng(n * 11 + len(name))
    U = W.haar_unitary(128, rng)
    psi0 = random_state(n, 5)
    st = qsim.State(n, qsim.C64)
    st.set_state(psi0)
    st.apply_fused(t, U, FP16X3)
    ref = psi0.copy()
    oracle.apply_gate(ref, n, t, (), U)
    check(st.get_state(), ref, n)


@pytest.mark.parametrize("name", ["rows_mixed", "quads", "pairs", "rows_high", "rows_q3"])
def test_single_block_many_tiles_per_cta(qsim, name):
    """23 qubits: 512 tiles, several per CTA (the accumulator and A planes reused across tiles)."""
    n = 23
    t = TARGETS[name]
    rng = np.random.default_rng(23)
    U = W.haar_unitary(128, rng)
    psi0 = random_state(n, 7)
    st = qsim.State(n, qsim.C64)
    st.set_state(psi0)
    st.apply_fused(t, U, FP16X3)
    ref = psi0.copy()
    oracle.apply_gate(ref, n, t, (), U)
    check(st.get_state(), ref, n)


def test_diagonal_and_permutation_blocks(qsim):
    """Structured 7-qubit matrices (a diagonal of phases, a permutation): exact zeros in B must stay zeros."""
    n = 16
    rng = np.random.default_rng(4)
    diag = np.diag(np.exp(1j * rng.uniform(0, 2 * np.pi, 128)))
    perm = np.eye(128)[rng.permutation(128)].astype(np.complex128)
    for U, t in ((diag, TARGETS["rows_high"]), (perm, TARGETS["quads"])):
        psi0 = random_state(n, 9)
        st = qsim.State(n, qsim.C64)
        st.set_state(psi0)
        st.apply_fused(t, U, FP16X3)
        ref = psi0.copy()
        oracle.apply_gate(ref, n, t, (), U)
        check(st.get_state(), ref, n)


def test_k7_needs_fp16x3(qsim):
    """Other tensor-core precisions have no 7-qubit block: the call is refused before any launch."""
    n = 15
    st = qsim.State(n, qsim.C64)
    st.set_basis(0)
    U = W.haar_unitary(128, np.random.default_rng(1))
    with pytest.raises(qsim.QsimError):
        st.apply_fused(TARGETS["rows_high"], U, TF32X3)
    st13 = qsim.State(13, qsim.C64)
    with pytest.raises(qsim.QsimError):  # n < k + 7
        st13.apply_fused((0, 1, 2, 3, 4, 5, 6), U, FP16X3)
    with pytest.raises(qsim.QsimError):  # plans: other precisions stop at 6 qubits
        qsim.Plan(W.brickwork(n, 4, seed=1), qsim.C64, mode=1, max_fused=7, precision=TF32X3, tc_min_k=5)


K7 = dict(mode=1, max_fused=7, precision=FP16X3, tc_min_k=5)


@pytest.mark.parametrize("seed", [3, 4])
def test_brickwork_20q_depth40_k7(qsim, seed):
    """The 20-qubit instance of the benchmark generator planned with 7-qubit blocks."""
    n = 20
    c = W.brickwork(n, 40, seed=seed)
    p = qsim.Plan(c, qsim.C64, **K7)
    ks = [q["k"] for q in p.passes() if q["kind"] == "tc"]
    assert ks.count(7) >= 20
    st = qsim.State(n, qsim.C64)
    p.execute_from_basis(st, 0)
    check(st.get_state(), oracle.run(c), n)


def test_k7_first_block_generates_the_basis_state(qsim):
    n = 17
    rng = np.random.default_rng(8)
    c = W.Circuit(n)
    c.append(W.Gate((3, 4, 5, 6, 7, 8, 9), (), W.haar_unitary(128, rng), "u7"))
    c.append(W.Gate((0, 1, 10, 11, 12, 13, 14), (), W.haar_unitary(128, rng), "u7"))
    p = qsim.Plan(c, qsim.C64, **K7)
    assert [(q["kind"], q["k"]) for q in p.passes()] == [("tc", 7), ("tc", 7)]
    x = 0b10110011100101011
    st = qsim.State(n, qsim.C64)
    st.set_state(random_state(n, 1))  # garbage the first pass must not read
    p.execute_from_basis(st, x)
    check(st.get_state(), oracle.run(c, basis_state=x), n)


@pytest.mark.parametrize("make", [lambda: W.rcs(18, seed=5), lambda: W.tfim_lattice(5, 3, 4, 0.27, 0.74),
                                  lambda: W.qft(18)])
def test_paper_workloads_k7(qsim, make):
    c = make()
    n = c.n
    st = qsim.State(n, qsim.C64)
    st.set_basis(0)
    info = st.run(c, **K7)
    assert info["tc_blocks"] > 0
    check(st.get_state(), oracle.run(c), n)


def test_full_size_k7_forward_inverse(qsim):
    """At the benchmark size (30 qubits) the circuit and its inverse, both with 7-qubit blocks, return
    |0...0>."""
    n = 30
    c = W.brickwork(n, 6, seed=3)
    st = qsim.State(n, qsim.C64)
    st.set_basis(0)
    st.run(c, **K7)
    info = st.run(W.inverse(c), **K7)
    norm = st.norm()
    assert abs(norm - 1.0) <= 1e-6 * 2 * info["tc_blocks"], (norm, info["tc_blocks"])
    p = st.probs([0, 1, 2, 3, 29])
    assert p[0] / norm >= 1.0 - 1e-6


def test_structure_cache_reuses_grouping_with_new_matrices(qsim):
    """Groupings are cached by circuit structure (qubits, diagonal or not), not by matrices: a second chain
    with the same structure and other angles is grouped like the first (its plan comes from the cache) and
    is still computed with its own matrices."""
    n = 16
    qsim.plan_cache_clear()
    c1 = W.tfim_chain(n, 4, 0.3, 0.7)
    c2 = W.tfim_chain(n, 4, 1.1, 0.2)
    p1 = qsim.Plan(c1, qsim.C64, **K7)
    p2 = qsim.Plan(c2, qsim.C64, **K7)
    assert [(q["kind"], q["targets"], q["gates"]) for q in p1.passes()] == \
           [(q["kind"], q["targets"], q["gates"]) for q in p2.passes()]
    for p, c in ((p2, c2), (p1, c1)):
        st = qsim.State(n, qsim.C64)
        p.execute_from_basis(st, 0)
        check(st.get_state(), oracle.run(c), n)
    qsim.plan_cache_clear()


@pytest.mark.parametrize("kw", [K7, dict(mode=0, max_fused=1), dict(mode=1, max_fused=4)])
def test_empty_circuit_plans(qsim, kw):
    """A circuit without gates plans to no passes: run from a basis state it leaves |x>, run on a state it
    leaves the state as it was."""
    n = 15
    c = W.Circuit(n)
    p = qsim.Plan(c, qsim.C64, **kw)
    assert p.passes() == []
    st = qsim.State(n, qsim.C64)
    p.execute_from_basis(st, 12345)
    psi = st.get_state()
    want = np.zeros(1 << n, dtype=np.complex128)
    want[12345] = 1.0
    assert np.array_equal(psi.astype(np.complex128), want)
    psi0 = random_state(n, 4)
    st.set_state(psi0)
    p.execute(st)
    assert np.array_equal(st.get_state(), psi0.astype(np.complex64))
