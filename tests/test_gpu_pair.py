"""Two fused 6-qubit blocks in one pass (QSIM_PREC_FP16X3 with pair_blocks: FP16 split products, the second
block applied while the tile is still on chip) against the FP64 oracle, at the complex64 bar: max |amplitude
error| <= 1e-5 and normalised infidelity <= 1e-9.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from helpers import random_state

pytestmark = pytest.mark.gpu

FP16X3 = 4


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


def two_blocks(n, t1, t2, seed):
    rng = np.random.default_rng(seed)
    c = W.Circuit(n)
    c.append(W.Gate(tuple(t1), (), W.haar_unitary(64, rng), "u6"))
    c.append(W.Gate(tuple(t2), (), W.haar_unitary(64, rng), "u6"))
    return c


CASES = [
    (14, [4, 5, 6, 7, 8, 9], [0, 1, 2, 3, 4, 5]),         # overlapping, the second on the lowest qubits
    (16, [8, 9, 10, 11, 12, 13], [12, 13, 14, 15, 2, 3]), # overlapping, unsorted second targets
    (15, [0, 1, 2, 3, 4, 5], [9, 10, 11, 12, 13, 14]),    # disjoint
    (14, [1, 3, 5, 7, 9, 11], [0, 2, 4, 6, 8, 10]),       # interleaved, union of 12
    (13, [0, 1, 2, 3, 4, 5], [6, 7, 8, 9, 10, 11]),       # the smallest state: one tile
    (21, [14, 15, 16, 17, 18, 19], [17, 18, 19, 20, 0, 1]),  # many tiles per CTA
]


@pytest.mark.parametrize("n,t1,t2", CASES)
def test_pair_of_blocks_against_oracle(qsim, n, t1, t2):
    c = two_blocks(n, t1, t2, n)
    p = qsim.Plan(c, qsim.C64, mode=1, max_fused=6, precision=FP16X3, tc_min_k=5, pair_blocks=True)
    ps = p.passes()
    assert [q["kind"] for q in ps] == ["tc_pair"]
    assert ps[0]["targets"] == sorted(t1) and sorted(ps[0]["controls"]) == sorted(t2)
    psi0 = random_state(n, 3)
    st = qsim.State(n, qsim.C64)
    st.set_state(psi0)
    p.execute(st)
    check(st.get_state(), oracle.run(c, psi=psi0.copy()), n)


def test_pair_generates_the_basis_state(qsim):
    """A plan starting with a pair generates |x> in its first tile loads (no set-up pass, no reads)."""
    n = 17
    c = two_blocks(n, [2, 3, 4, 5, 6, 7], [6, 7, 8, 9, 10, 11], 5)
    p = qsim.Plan(c, qsim.C64, mode=1, max_fused=6, precision=FP16X3, tc_min_k=5, pair_blocks=True)
    st = qsim.State(n, qsim.C64)
    x = 0b10110011100101011
    st.set_state(random_state(n, 1))  # garbage the first pass must not read
    p.execute_from_basis(st, x)
    check(st.get_state(), oracle.run(c, basis_state=x), n)


@pytest.mark.parametrize("seed", [3, 4])
def test_brickwork_20q_depth40_with_pairs(qsim, seed):
    """The 20-qubit instance of the benchmark generator with pairing: complex64 bar against the oracle."""
    n = 20
    c = W.brickwork(n, 40, seed=seed)
    p = qsim.Plan(c, qsim.C64, mode=1, max_fused=6, precision=FP16X3, tc_min_k=5, pair_blocks=True)
    kinds = [q["kind"] for q in p.passes()]
    assert kinds.count("tc_pair") >= 10
    st = qsim.State(n, qsim.C64)
    p.execute_from_basis(st, 0)
    check(st.get_state(), oracle.run(c), n)


def test_paper_random_circuit_with_pairs(qsim):
    n = 18
    c = W.rcs(n, seed=5)
    st = qsim.State(n, qsim.C64)
    st.set_basis(0)
    info = st.run(c, mode=1, max_fused=6, precision=FP16X3, tc_min_k=5, pair_blocks=True)
    assert info["tc_blocks"] > 0
    check(st.get_state(), oracle.run(c), n)


def test_full_size_pairs_forward_inverse(qsim):
    """At the benchmark size (30 qubits) the paired circuit followed by its paired inverse returns |0...0>."""
    n = 30
    c = W.brickwork(n, 4, seed=3)
    st = qsim.State(n, qsim.C64)
    st.set_basis(0)
    kw = dict(mode=1, max_fused=6, precision=FP16X3, tc_min_k=5, pair_blocks=True)
    st.run(c, **kw)
    info = st.run(W.inverse(c), **kw)
    norm = st.norm()
    assert abs(norm - 1.0) <= 1e-6 * 2 * info["tc_blocks"], (norm, info["tc_blocks"])
    p = st.probs([0, 1, 2, 3, 29])
    assert p[0] / norm >= 1.0 - 1e-6
