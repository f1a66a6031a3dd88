"""Small-state plans run as one resident cooperative launch (every pass inside one kernel, grid barriers
between passes) against the FP64 oracle and against the same plan launched pass by pass.

Tolerances: complex64 -- max |amplitude error| <= 1e-5 and normalised infidelity <= 1e-9; complex128 -- max
|amplitude error| <= 1e-12 and infidelity <= 1e-12. Resident and per-pass launches of dense blocks of up to 4
qubits and of diagonals do the same arithmetic per amplitude (the same FMA chains), so their complex128 states
must be identical; complex64 per-pass plans take a warp-shuffle kernel for single-qubit gates on qubits 1..5,
and 5-qubit blocks a shared-memory kernel, so those are compared within the tolerance.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from helpers import random_state

pytestmark = pytest.mark.gpu

TOL = {0: (1e-5, 1e-9), 1: (1e-12, 1e-12)}
C64, C128 = 0, 1


@pytest.fixture(scope="module")
def qsim(gpu_lib):
    from paper_2511_14664_gb300 import qsim as q
    return q


def close(psi_gpu, ref, n, dtype):
    at, it = TOL[dtype]
    g = np.ascontiguousarray(psi_gpu.astype(np.complex128))
    err = float(np.max(np.abs(g - ref)))
    inf = oracle.infidelity(g, ref, n)
    assert err <= at, f"max amplitude error {err:.3e}"
    assert inf <= it, f"infidelity {inf:.3e}"


def random_circuit(n, gates, seed, kmax=3, cmax=2, diag_prob=0.3):
    rng = np.random.default_rng(seed)
    c = W.Circuit(n)
    for _ in range(gates):
        c.append(W.random_gate(n, rng, kmax=min(kmax, n), cmax=cmax, diag_prob=diag_prob))
    return c


def run_both(qsim, c, dtype, psi0, **kw):
    """The plan executed resident and launched pass by pass, from the same state."""
    out = []
    for lpp in (False, True):
        p = qsim.Plan(c, dtype, launch_per_pass=lpp, **kw)
        assert p.info["resident"] == (0 if lpp else 1)
        st = qsim.State(c.n, dtype)
        st.set_state(psi0)
        p.execute(st)
        out.append(st.get_state())
        p.close()
    return out


@pytest.mark.parametrize("dtype", [C64, C128])
@pytest.mark.parametrize("n", [1, 2, 5, 9, 14, 16])
@pytest.mark.parametrize("kw", [dict(mode=0, max_fused=1), dict(mode=1, max_fused=2), dict(mode=1, max_fused=4),
                                dict(mode=1, max_fused=5)])
def test_random_circuits_against_oracle(qsim, dtype, n, kw):
    """Dense gates with controls and diagonal gates (some entries exactly 1), per-gate and fused plans; n = 1 and
    2 leave most lanes of a warp idle in every pass."""
    c = random_circuit(n, 60, seed=7 * n + kw["max_fused"], kmax=3 if n >= 3 else n, cmax=2 if n >= 4 else 0)
    psi0 = random_state(n, n + 100)
    res, per = run_both(qsim, c, dtype, psi0, **kw)
    ref = oracle.run(c, psi=psi0.copy())
    close(res, ref, n, dtype)
    close(per, ref, n, dtype)
    if dtype == C128 and kw["max_fused"] <= 4:
        assert np.array_equal(res, per)


@pytest.mark.parametrize("dtype", [C64, C128])
@pytest.mark.parametrize("k", [4, 5])
def test_brickwork_14q_complex128_config(qsim, dtype, k):
    """The 14-qubit random brickwork (20 layers, 410 gates) fused at k = 4 and 5, from |0>: the resident plan
    against the oracle."""
    c = W.brickwork(14, 20, seed=1)
    p = qsim.Plan(c, dtype, mode=1, max_fused=k)
    assert p.info["resident"] == 1 and p.info["passes"] > 10
    st = qsim.State(14, dtype)
    p.execute_from_basis(st, 0)
    close(st.get_state(), oracle.run(c), 14, dtype)


def test_from_basis_and_repeated_execution(qsim):
    """The resident launch sets |x> itself; executing the plan three times applies it three times (the barrier
    word restarts with every launch)."""
    n = 12
    c = random_circuit(n, 40, seed=3, kmax=4, cmax=1)
    x = 0b101101110001
    p = qsim.Plan(c, C128, mode=1, max_fused=4)
    assert p.info["resident"] == 1
    st = qsim.State(n, C128)
    st.set_state(random_state(n, 9))  # garbage the launch must overwrite
    p.execute_from_basis(st, x)
    ref = oracle.run(c, basis_state=x)
    close(st.get_state(), ref, n, C128)
    p.execute(st)
    p.execute(st)
    ref3 = oracle.run(c, psi=oracle.run(c, psi=ref.copy()))
    close(st.get_state(), ref3, n, C128)


def test_many_passes_and_graph_option(qsim):
    """A per-gate plan of 400 passes (400 grid barriers in one launch), also with use_graph (a resident plan
    is one launch and is not captured)."""
    n = 10
    c = random_circuit(n, 400, seed=11, kmax=2, cmax=1)
    psi0 = random_state(n, 5)
    ref = oracle.run(c, psi=psi0.copy())
    for ug in (False, True):
        p = qsim.Plan(c, C128, mode=0, max_fused=1, use_graph=ug)
        assert p.info["resident"] == 1 and p.info["passes"] == 400
        st = qsim.State(n, C128)
        for _ in range(2):
            st.set_state(psi0)
            p.execute(st)
        close(st.get_state(), ref, n, C128)
        p.close()


def test_eligibility(qsim):
    """Resident only for states of at most 16 qubits whose passes are all CUDA-core dense blocks (k <= 5),
    diagonals or phase passes; a pass range still launches pass by pass and matches."""
    c17 = W.brickwork(17, 4, seed=2)
    assert qsim.Plan(c17, C128, mode=1, max_fused=4).info["resident"] == 0
    c = W.brickwork(14, 6, seed=2)
    assert qsim.Plan(c, C64, mode=1, max_fused=6, precision=1, tc_min_k=5).info["resident"] == 0  # tensor cores
    assert qsim.Plan(c, C128, mode=1, max_fused=6).info["resident"] == 0                           # 6-qubit SIMT
    assert qsim.Plan(c, C128, mode=1, max_fused=4, local_qubits=12).info["resident"] == 0           # reorders
    p = qsim.Plan(c, C128, mode=1, max_fused=5)
    assert p.info["resident"] == 1
    psi0 = random_state(14, 2)
    st = qsim.State(14, C128)
    st.set_state(psi0)
    npass = p.info["passes"]
    p.execute_range(st, 0, npass // 2)
    p.execute_range(st, npass // 2, npass - npass // 2)
    close(st.get_state(), oracle.run(c, psi=psi0.copy()), 14, C128)
    info = qsim.State(14, C128).run(c, mode=1, max_fused=4)
    assert info["resident"] == 1


@pytest.mark.parametrize("dtype", [C64, C128])
@pytest.mark.parametrize("make", [lambda: W.qft(12), lambda: W.qft(16), lambda: W.qpe(11, 1234)[0]])
def test_phase_passes(qsim, dtype, make):
    """Plans with phase passes (runs of controlled phases: a quadratic form of the index bits, summed per
    amplitude in fixed-point turns) against the oracle and against the per-pass launches."""
    c = make()
    n = c.n
    p = qsim.Plan(c, dtype, mode=1, max_fused=4)
    assert p.info["resident"] == 1
    assert "phase" in [q["kind"] for q in p.passes()]
    psi0 = random_state(n, 21)
    res, per = run_both(qsim, c, dtype, psi0, mode=1, max_fused=4)
    ref = oracle.run(c, psi=psi0.copy())
    close(res, ref, n, dtype)
    close(per, ref, n, dtype)


def test_fp64_rate_probe(qsim):
    """The FP64 rate probe (the resident runner's roofline denominator) reports a plausible rate for its
    elapsed time: positive, below the FP64 rate of any GPU of this class (~100 TFLOP/s), and the run lasts
    about as long as asked."""
    tf, ms = qsim.fp64_peak(0.2)
    assert 0.05 < tf < 100.0, tf
    assert 50.0 < ms < 2000.0, ms
