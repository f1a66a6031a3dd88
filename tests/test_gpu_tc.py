"""Tensor-core fused blocks (tcgen05, split precision) against the FP64 oracle.

Tolerances: 3xTF32 and BF16x6 are held to the complex64 bar (max |amplitude error| <= 1e-5, normalised
infidelity <= 1e-9). BF16x3 is a reduced-accuracy precision (~16 significant bits per product): a single
block on a random state is held to max error <= 1e-5 and infidelity <= 1e-8, and the 20-qubit depth-40
benchmark circuit (64 blocks) to the complex64 bar of 1e-9.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from helpers import random_state

pytestmark = pytest.mark.gpu

PRECS = {"tf32x3": 1, "bf16x3": 2, "bf16x6": 3, "fp16x3": 4}
BLOCK_TOL = {"tf32x3": (1e-5, 1e-9), "bf16x3": (1e-5, 1e-8), "bf16x6": (1e-5, 1e-9), "fp16x3": (1e-5, 1e-9)}


@pytest.fixture(scope="module")
def qsim(gpu_lib):
    from paper_2511_14664_gb300 import qsim as q
    return q


def check(psi_gpu, ref, n, amp_tol, inf_tol):
    g = psi_gpu.astype(np.complex128)
    err = float(np.max(np.abs(g - ref)))
    inf = oracle.infidelity(np.ascontiguousarray(g), ref, n)
    assert err <= amp_tol, f"max amplitude error {err:.3e}"
    assert inf <= inf_tol, f"infidelity {inf:.3e}"
    return err, inf


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("k", [5, 6])
@pytest.mark.parametrize("targets", ["high", "low", "mixed", "top"])
def test_single_block(qsim, prec, k, targets):
    n = 15
    rng = np.random.default_rng(k * 7 + len(targets))
    if targets == "high":
        t = tuple(int(x) for x in rng.permutation(np.arange(7, n))[:k])
    elif targets == "low":
        t = tuple(range(k))
    elif targets == "top":
        t = tuple(range(n - 1, n - 1 - k, -1))
    else:
        t = tuple(int(x) for x in rng.permutation(n)[:k])
    U = W.haar_unitary(1 << k, rng)
    psi0 = random_state(n, 3)
    st = qsim.State(n, qsim.C64)
    st.set_state(psi0)
    st.apply_fused(t, U, PRECS[prec])
    ref = psi0.copy()
    oracle.apply_gate(ref, n, t, (), U)
    check(st.get_state(), ref, n, *BLOCK_TOL[prec])


# Target patterns that take the block kernel's different data paths: with qubit 0 not a target but one of
# qubits 1..3 a target, pair rows (3xTF32: 16x256b TMEM fragments whose two rows differ in qubit 0, lanes
# l % 4 on the two lowest targets); lanes on rows with 8-byte accesses (targets from qubit 4 up, or BF16x3);
# 16-byte pairs (qubit 0 the first target), 32-byte quads
# (qubits 0 and 1 the first two), line groups (qubits 0..3 the first four, 3xTF32: four lanes per row,
# permuted column order), and low runs from qubit 0, 1 or 2 given in scrambled order (rows interleaved with
# targets in the lowest address bits).
PATH_TARGETS = {
    "from3": (8, 3, 5, 4, 7, 6),
    "run_from0_in_order": (0, 1, 2, 3, 4, 5),
    "lines_spread": (0, 1, 2, 3, 19, 11),
    "quads_spread": (0, 1, 9, 4, 20, 13),
    "almost_lines": (0, 1, 2, 4, 3, 5),
    "even_from0": (0, 2, 4, 6, 8, 10),
    "run_from0": (3, 0, 5, 1, 4, 2),
    "run_from1": (6, 1, 2, 3, 4, 5),
    "run_from2": (2, 7, 3, 4, 6, 5),
    "low_and_high": (1, 21, 3, 4, 17, 2),
    "pair_rows_low": (2, 3, 8, 9, 14, 15),
    "rows_high": (4, 9, 12, 15, 18, 21),
}


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("path", list(PATH_TARGETS))
def test_block_paths_many_tiles(qsim, prec, path):
    """23 qubits: 1024 tiles, so every CTA runs several tiles through the pipeline (two accumulators, the
    epilogue of tile i-1 behind the MMAs of tile i) and some CTAs run one more than others."""
    n = 23
    t = PATH_TARGETS[path]
    rng = np.random.default_rng(len(path) * 11 + PRECS[prec])
    U = W.haar_unitary(64, rng)
    psi0 = random_state(n, 5)
    st = qsim.State(n, qsim.C64)
    st.set_state(psi0)
    st.apply_fused(t, U, PRECS[prec])
    ref = psi0.copy()
    oracle.apply_gate(ref, n, t, (), U)
    check(st.get_state(), ref, n, *BLOCK_TOL[prec])


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("path", ["from3", "run_from0_in_order", "lines_spread", "run_from0", "run_from1"])
def test_block_paths_k5(qsim, prec, path):
    n = 21
    t = PATH_TARGETS[path][:5]
    rng = np.random.default_rng(len(path) * 13 + PRECS[prec])
    U = W.haar_unitary(32, rng)
    psi0 = random_state(n, 6)
    st = qsim.State(n, qsim.C64)
    st.set_state(psi0)
    st.apply_fused(t, U, PRECS[prec])
    ref = psi0.copy()
    oracle.apply_gate(ref, n, t, (), U)
    check(st.get_state(), ref, n, *BLOCK_TOL[prec])


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("t", [(12, 0, 5, 9, 3, 7), (0, 1, 2, 3, 4, 5)])
def test_smallest_state_single_tile(qsim, prec, t):
    """n = k + 7: exactly one 128-row tile."""
    k, n = 6, 13
    rng = np.random.default_rng(1)
    U = W.haar_unitary(64, rng)
    psi0 = random_state(n, 8)
    st = qsim.State(n, qsim.C64)
    st.set_state(psi0)
    st.apply_fused(t, U, PRECS[prec])
    ref = psi0.copy()
    oracle.apply_gate(ref, n, t, (), U)
    check(st.get_state(), ref, n, *BLOCK_TOL[prec])


def test_too_small_state_is_rejected(qsim):
    st = qsim.State(12, qsim.C64)
    st.set_basis(0)
    with pytest.raises(qsim.QsimError) as e:
        st.apply_fused(tuple(range(6)), np.eye(64), PRECS["tf32x3"])
    assert e.value.code == 5
    st128 = qsim.State(14, qsim.C128)
    with pytest.raises(qsim.QsimError) as e:
        st128.apply_fused(tuple(range(6)), np.eye(64), PRECS["tf32x3"])
    assert e.value.code == 5


@pytest.mark.parametrize("prec", list(PRECS))
def test_brickwork_20q_depth40_fused_tc(qsim, prec):
    """The 20-qubit instance of the 30-qubit benchmark generator, fused into 6-qubit tensor-core blocks."""
    n = 20
    c = W.brickwork(n, 40, seed=3)
    ref = oracle.run(c)
    st = qsim.State(n, qsim.C64)
    st.set_basis(0)
    info = st.run(c, mode=qsim.RUN_FUSED, max_fused=6, precision=PRECS[prec], tc_min_k=5)
    assert info["tc_blocks"] > 0
    g = st.get_state().astype(np.complex128)
    inf = oracle.infidelity(g, ref, n)
    err = float(np.max(np.abs(g - ref)))
    assert inf <= 1e-9, inf
    assert err <= 1e-5, err


def test_repeated_launches_and_plan_reuse(qsim):
    """Many consecutive tensor-core passes (TMEM allocated and freed by every launch)."""
    n = 16
    c = W.brickwork(n, 12, seed=9)
    ref = oracle.run(c)
    p = qsim.Plan(c, mode=qsim.RUN_FUSED, max_fused=6, precision=PRECS["tf32x3"], tc_min_k=5, use_graph=True)
    assert p.info["tc_blocks"] > 0
    st = qsim.State(n, qsim.C64)
    for _ in range(3):
        st.set_basis(0)
        p.execute(st)
        check(st.get_state(), ref, n, 1e-5, 1e-9)
    st.synchronize()


def test_full_size_property_forward_inverse(qsim):
    """At the benchmark size (30 qubits, 8 GiB) the fused tensor-core circuit followed by its fused inverse
    returns |0...0>: a check that holds at any size, in the launch configuration the benchmark times."""
    n = 30
    c = W.brickwork(n, 4, seed=3)
    st = qsim.State(n, qsim.C64)
    st.set_basis(0)
    st.run(c, mode=qsim.RUN_FUSED, max_fused=6, precision=PRECS["tf32x3"], tc_min_k=5)
    info = st.run(W.inverse(c), mode=qsim.RUN_FUSED, max_fused=6, precision=PRECS["tf32x3"], tc_min_k=5)
    # The tensor cores accumulate FP32 with truncation (round towards zero), so each block shrinks the norm
    # by a few 1e-7; the bound below allows 1e-6 per tensor-core pass of the round trip.
    norm = st.norm()
    assert abs(norm - 1.0) <= 1e-6 * 2 * info["tc_blocks"], (norm, info["tc_blocks"])
    p = st.probs([0, 1, 2, 3, 29])
    assert p[0] / norm >= 1.0 - 1e-6  # normalised overlap with |0...0>
