"""qsim_plan_execute_from_basis: a plan run from a basis state, where a first tensor-core block generates
|x> in registers instead of reading a set-up state. Its result must equal set_basis(x) followed by execute
bit for bit (the block sees the same exact inputs, 1 and 0), on every data path of the block kernel (rows,
16-byte pairs, 32-byte quads) and with a phase epilogue; other plans fall back to set_basis + execute.
Against the FP64 oracle: complex64 bar (max |amplitude error| <= 1e-5, normalised infidelity <= 1e-9)."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TC6 = dict(mode=1, max_fused=6, precision=1, tc_min_k=5)


@pytest.fixture(scope="module")
def qsim(gpu_lib):
    from paper_2511_14664_gb300 import qsim as q
    return q


def block_circuit(n, targets, rng, extra=()):
    """One dense 6-qubit block on `targets` (a product of random 2-qubit unitaries), then `extra` gates."""
    c = W.Circuit(n)
    t = list(targets)
    for i in range(0, len(t), 2):
        c.append(W.Gate((t[i], t[i + 1]), (), W.haar_unitary(4, rng), "u4"))
    for i in range(1, len(t) - 1, 2):
        c.append(W.Gate((t[i], t[i + 1]), (), W.haar_unitary(4, rng), "u4"))
    for g in extra:
        c.append(g)
    return c


def run_both(qsim, c, plan_kw, x, count=-1):
    n = c.n
    p = qsim.Plan(c, qsim.C64, **plan_kw)
    a = qsim.State(n, qsim.C64)
    a.set_basis((x + 1) % (1 << n))  # stale contents the generated block must overwrite
    p.execute_from_basis(a, x, count)
    b = qsim.State(n, qsim.C64)
    b.set_basis(x)
    if count < 0:
        p.execute(b)
    else:
        p.execute_range(b, 0, count)
    return p, a.get_state(), b.get_state()


@pytest.mark.parametrize("targets", [(8, 9, 10, 11, 12, 13),    # rows path
                                     (0, 5, 9, 12, 14, 17),     # 16-byte pairs (qubit 0 first)
                                     (0, 1, 2, 3, 4, 5),        # 32-byte quads (qubits 0, 1 first)
                                     (13, 3, 17, 1, 7, 10)])    # scattered
def test_generated_input_matches_set_basis(qsim, targets):
    n = 18
    rng = np.random.default_rng(sum(targets))
    c = block_circuit(n, targets, rng)
    for x in (0, 1, 0b101101, (1 << n) - 1, int(rng.integers(0, 1 << n))):
        p, got, want = run_both(qsim, c, TC6, x)
        ps = p.passes()
        assert len(ps) == 1 and ps[0]["kind"] == "tc"
        assert np.array_equal(got, want), x
        ref = oracle.run(c, basis_state=x)
        g = got.astype(np.complex128)
        assert float(np.max(np.abs(g - ref))) <= 1e-5
        assert oracle.infidelity(np.ascontiguousarray(g), ref, n) <= 1e-9


def test_generated_input_with_phase_epilogue(qsim):
    """A 6-qubit block followed by controlled phases to lower qubits: the block carries them in its epilogue."""
    n = 17
    rng = np.random.default_rng(11)
    extra = [W.Gate((q,), (c_,), W.CP(float(rng.uniform(0, 6.28))), "cp")
             for q in (10, 11, 12, 13) for c_ in (0, 3, 6)]
    c = block_circuit(n, (10, 11, 12, 13, 14, 15), rng, extra)
    x = 0b10110011001011101
    p, got, want = run_both(qsim, c, TC6, x)
    ps = p.passes()
    assert ps[0]["kind"] == "tc" and ps[0]["launches"] == 2 and ps[0]["gates"] == len(c)
    assert np.array_equal(got, want)
    ref = oracle.run(c, basis_state=x)
    assert float(np.max(np.abs(got.astype(np.complex128) - ref))) <= 1e-5


@pytest.mark.parametrize("prec", [1, 2])
def test_brickwork_from_basis_and_partial_range(qsim, prec):
    """The 20-qubit instance of the benchmark generator: all passes, and the first pass alone followed by the
    rest through execute_range (the benchmark's per-pass timing)."""
    n = 20
    c = W.brickwork(n, 40, seed=3)
    kw = dict(TC6, precision=prec)
    p, got, want = run_both(qsim, c, kw, 0)
    assert p.passes()[0]["kind"] == "tc"
    assert np.array_equal(got, want)
    st = qsim.State(n, qsim.C64)
    st.set_basis(5)
    p.execute_from_basis(st, 0, 1)
    p.execute_range(st, 1, len(p.passes()) - 1)
    assert np.array_equal(st.get_state(), want)
    if prec == 1:
        ref = oracle.run(c)
        assert oracle.infidelity(np.ascontiguousarray(got.astype(np.complex128)), ref, n) <= 1e-9


@pytest.mark.parametrize("kw", [dict(mode=0, max_fused=1), dict(mode=1, max_fused=5),
                                dict(mode=1, max_fused=6, precision=3, tc_min_k=5)])
def test_fallback_plans(qsim, kw):
    """Plain, CUDA-core and BF16x6 plans take the set-up pass first; results equal set_basis + execute."""
    n = 14
    c = W.brickwork(n, 6, seed=2)
    for count in (-1, 1, 0):
        p, got, want = run_both(qsim, c, kw, 77, count)
        assert np.array_equal(got, want)


def test_basis_index_out_of_range(qsim):
    n = 12
    c = W.brickwork(n, 2, seed=1)
    p = qsim.Plan(c, qsim.C64, **TC6)
    st = qsim.State(n, qsim.C64)
    with pytest.raises(Exception):
        p.execute_from_basis(st, 1 << n)
    with pytest.raises(Exception):
        p.execute_from_basis(st, 0, len(p.passes()) + 1)
