"""The fusion planner (host C++) without a GPU: plans made with dry_run list their passes, so their structure
is checked here. Every plan keeps every input gate exactly once, each pass's qubits are valid, and the
benchmarked circuits get the pass structure the kernels are built around (tensor-core blocks of 6 qubits,
phase passes or epilogues for runs of diagonal gates)."""
import math

import numpy as np
import pytest

import workloads as W

TC6 = dict(mode=1, max_fused=6, precision=1, tc_min_k=5)


@pytest.fixture(scope="module")
def qsim():
    from paper_2511_14664_gb300 import qsim as q
    q.lib()  # builds and loads the library (no device needed for dry runs)
    return q


def plan(qsim, c, dtype=0, **kw):
    p = qsim.Plan(c, dtype, dry_run=True, **kw)
    ps = p.passes()
    assert sum(q["gates"] for q in ps) == len(c)
    for q in ps:
        # a pair pass lists its second block's targets as controls: each block's qubits are distinct
        groups = [q["targets"], q["controls"]] if q["kind"] == "tc_pair" else [q["targets"] + q["controls"]]
        for qubits in groups:
            assert len(set(qubits)) == len(qubits) and all(0 <= x < c.n for x in qubits)
    return p, ps


def test_plain_plan_is_one_pass_per_gate(qsim):
    c = W.qft(12)
    p, ps = plan(qsim, c, mode=0, max_fused=1)
    assert len(ps) == len(c)
    for q, g in zip(ps, c.gates):
        diag = np.allclose(g.matrix, np.diag(np.diag(g.matrix)))
        assert q["kind"] == ("diag" if diag else "dense_small")
        assert q["gates"] == 1


def test_brickwork_30q_tensor_core_blocks(qsim):
    """The benchmark's 30-qubit brickwork: every pass a 6-qubit tensor-core block, each moving the whole state
    once (the last one carries the final CZ layer in its epilogue; a 4-qubit block is padded to 6)."""
    c = W.brickwork(30, 40, seed=3)
    p, ps = plan(qsim, c, **TC6)
    assert all(q["kind"] == "tc" and q["k"] == 6 for q in ps)
    assert len(ps) <= 64
    full = 2 * 8 * 2.0 ** 30
    assert all(q["algorithmic_bytes"] == full for q in ps)
    assert p.info["algorithmic_bytes"] == full * len(ps)


def test_qft_phases_fold_into_blocks(qsim):
    """28-qubit QFT: the controlled phases that link a block to lower qubits ride on the block's epilogue;
    no separate phase or diagonal pass remains."""
    c = W.qft(28)
    p, ps = plan(qsim, c, **TC6)
    assert all(q["kind"] == "tc" for q in ps)
    assert len(ps) <= 9
    # without tensor cores the phases need passes of their own
    p2, ps2 = plan(qsim, c, mode=1, max_fused=6)
    assert any(q["kind"] == "phase" for q in ps2) and len(ps2) > len(ps)


def test_qpe_33q_passes(qsim):
    c, _ = W.qpe(32, W.basis_index(32, 7))
    p, ps = plan(qsim, c, **TC6)
    assert len(ps) <= 18 and all(q["kind"] == "tc" for q in ps)


def test_lattice_tfim_one_phase_per_step(qsim):
    """The 33-site triangular lattice: the 99 RZZ gates of a Trotter step gather in one phase pass (or an
    epilogue); the RX layers go to 6-qubit blocks."""
    c = W.tfim_lattice(11, 3, 10, 0.27, 0.74)
    p, ps = plan(qsim, c, **TC6)
    assert len(ps) <= 63
    assert sum(1 for q in ps if q["kind"] == "phase") <= 10


def test_phase_pass_any_width(qsim):
    """A run of diagonal gates on 20 qubits after CUDA-core blocks: one phase pass (no epilogue without
    tensor cores) carrying those the dense blocks did not take in (a gate whose qubits both lie in a
    block's window may join that block)."""
    rng = np.random.default_rng(1)
    n = 20
    c = W.Circuit(n)
    for q in range(n):
        c.append(W.Gate((q,), (), W.haar_unitary(2, rng), "u"))
    diag = 0
    for _ in range(40):
        a, b = (int(x) for x in rng.choice(n, size=2, replace=False))
        c.append(W.Gate((a, b), (), W.RZZ(float(rng.uniform(0, math.pi))), "rzz"))
        diag += 1
    p, ps = plan(qsim, c, mode=1, max_fused=4)
    phases = [q for q in ps if q["kind"] == "phase"]
    assert len(phases) == 1 and phases[0]["gates"] >= diag // 2 and phases[0]["k"] == 0
    assert phases[0]["algorithmic_bytes"] == 2 * 8 * 2.0 ** n


def test_four_qubit_block_padded_for_tensor_cores(qsim):
    n = 16
    rng = np.random.default_rng(2)
    c = W.Circuit(n)
    for _ in range(3):
        for q in (3, 4, 5, 6):
            c.append(W.Gate((q,), (), W.haar_unitary(2, rng), "u"))
        c.append(W.Gate((3, 4), (), W.haar_unitary(4, rng), "u4"))
        c.append(W.Gate((5, 6), (), W.haar_unitary(4, rng), "u4"))
    p, ps = plan(qsim, c, **TC6)
    assert len(ps) == 1 and ps[0]["kind"] == "tc" and ps[0]["k"] == 6
    assert set(ps[0]["targets"]) == {3, 4, 5, 6, 14, 15}
    p2, ps2 = plan(qsim, c, mode=1, max_fused=6)  # CUDA cores: stays a 4-qubit pass
    assert len(ps2) == 1 and ps2[0]["kind"] == "dense_small" and ps2[0]["k"] == 4


def test_global_qubits_plan(qsim):
    """local_qubits: before a pass touches a global qubit a reorder brings it in; every non-reorder pass
    then works on local positions only, and diagonal runs stay within the fusion width."""
    n, L = 24, 20
    c = W.random_pairs(n, 4, seed=5)
    p, ps = plan(qsim, c, mode=1, max_fused=4, local_qubits=L)
    assert any(q["kind"] == "reorder" for q in ps)
    for q in ps:
        if q["kind"] != "reorder":
            assert all(x < L for x in q["targets"] + q["controls"])
        else:  # exchanged index-bit pairs (the passes that restore the identity order may pair two local bits)
            assert q["k"] == q["nc"] >= 1
            assert any((a >= L) != (b >= L) for a, b in zip(q["targets"], q["controls"])) or q is ps[-1] or \
                all(x["kind"] == "reorder" for x in ps[ps.index(q):])
        assert q["kind"] != "phase"


def test_dry_run_needs_no_device_and_reports_info(qsim):
    c = W.brickwork(14, 6, seed=1)
    p, ps = plan(qsim, c, 1, mode=1, max_fused=4)
    assert p.info["passes"] == len(ps) and p.info["input_gates"] == len(c)
    assert p.info["host_plan_ms"] >= 0.0


def test_plan_effort_lookahead_never_more_passes(qsim):
    """plan_effort 1 adds groupings with one block of look-ahead and keeps the one with the fewest blocks:
    never more passes than greedy fusion, every gate still placed once; on the 33-site lattice TFIM it
    saves passes."""
    cases = [W.tfim_lattice(11, 3, 10, 0.27, 0.74), W.brickwork(20, 40, seed=3), W.qft(16), W.rcs(18, seed=3)]
    for c in cases:
        _, ps0 = plan(qsim, c, **TC6)
        _, ps1 = plan(qsim, c, plan_effort=1, **TC6)
        assert len(ps1) <= len(ps0)
    _, a = plan(qsim, cases[0], **TC6)
    _, b = plan(qsim, cases[0], plan_effort=1, **TC6)
    assert len(b) < len(a)


def test_plan_effort_beam_never_more_passes_and_places_every_gate(qsim):
    """plan_effort 2 adds a beam search over groupings (the partial groupings that placed the most gates)
    and keeps the grouping with the fewest blocks: never more passes than greedy or look-ahead fusion, the
    merged gate counts add up to the circuit's, and on the 30-qubit brickwork it saves passes."""
    cases = [W.brickwork(30, 40, seed=3), W.rcs(20, seed=3), W.qft(18)]
    for c in cases:
        _, ps1 = plan(qsim, c, plan_effort=1, **TC6)
        _, ps2 = plan(qsim, c, plan_effort=2, **TC6)
        assert len(ps2) <= len(ps1)
        assert sum(q["gates"] for q in ps2) == len(c)
    _, a = plan(qsim, cases[0], **TC6)
    _, b = plan(qsim, cases[0], plan_effort=2, **TC6)
    assert len(b) < len(a)


@pytest.mark.parametrize("make", [lambda: W.brickwork(30, 40, seed=3), lambda: W.rcs(33, seed=3), lambda: W.qft(28),
                                  lambda: W.tfim_lattice(11, 3, 10, 0.27, 0.74)])
def test_pairs_are_consecutive_blocks_of_the_tf32_plan(qsim, make):
    """A QSIM_PREC_FP16X3 plan with pair_blocks pairs consecutive 6-qubit blocks: with every pair unrolled into its two
    blocks, the pass sequence is exactly the 3xTF32 plan's, each pair's targets span at most 12 qubits,
    and the merged gate counts add up."""
    c = make()
    _, single = plan(qsim, c, **TC6)
    _, paired = plan(qsim, c, mode=1, max_fused=6, precision=4, tc_min_k=5, pair_blocks=True)
    unrolled = []
    for q in paired:
        if q["kind"] == "tc_pair":
            assert q["k"] == 6 and q["nc"] == 6 and len(set(q["targets"]) | set(q["controls"])) <= 12
            unrolled.append(("tc", q["targets"]))
            unrolled.append(("tc", q["controls"]))
        else:
            unrolled.append((q["kind"], q["targets"]))
    assert unrolled == [(q["kind"], q["targets"]) for q in single]
    # without pair_blocks, the same plan has no pairs, and its blocks keep 3xTF32 exactly where their 3xTF32
    # form has a line-group or pair-rows path
    _, fp16 = plan(qsim, c, mode=1, max_fused=6, precision=4, tc_min_k=5)
    assert [(q["kind"], q["targets"]) for q in fp16] == [(q["kind"], q["targets"]) for q in single]
    for q in fp16:
        if q["kind"] == "tc":
            t = q["targets"]
            epi = q["launches"] == 2  # a phase epilogue: neither 3xTF32 path exists, the block stays FP16
            keep_tf32 = not epi and (t[:4] == [0, 1, 2, 3] or (0 not in t and any(x in t for x in (1, 2, 3))))
            assert q["precision"] == (1 if keep_tf32 else 4), (t, q["precision"])
    assert sum(q["gates"] for q in paired) == len(c)
    # (blocks with a phase epilogue do not pair)
    assert sum(1 for q in paired if q["kind"] == "tc_pair") >= len(single) // 5


def test_seven_qubit_blocks(qsim):
    """max_fused = 7 with QSIM_PREC_FP16X3: 7-qubit tensor-core blocks in FP16 (no 3xTF32 form, no phase
    epilogue) that keep off qubits 0..2, every gate placed once; the 30-qubit brickwork takes 50 passes instead
    of 64; where the 6-qubit grouping is cheaper (the QFT) it is kept."""
    c = W.brickwork(30, 40, seed=3)
    _, ps = plan(qsim, c, mode=1, max_fused=7, precision=4, tc_min_k=5)
    k7 = [q for q in ps if q["kind"] == "tc" and q["k"] == 7]
    assert len(ps) <= 50 and len(k7) >= 40
    assert all(min(q["targets"]) >= 3 for q in k7)
    assert all(q["k"] <= 6 for q in ps if q["kind"] == "tc" and min(q["targets"]) < 3)
    assert all(q["precision"] == 4 and q["launches"] == 1 for q in k7)
    assert all(q["algorithmic_bytes"] == 2 * 8 * 2.0 ** 30 for q in k7)
    # the QFT's phases ride on 6-qubit blocks as epilogues, which 7-qubit blocks cannot carry: width 7 keeps the
    # (cheaper) 6-qubit grouping
    c = W.qft(20)
    _, p6 = plan(qsim, c, mode=1, max_fused=6, precision=4, tc_min_k=5)
    _, p7 = plan(qsim, c, mode=1, max_fused=7, precision=4, tc_min_k=5)
    assert [(q["kind"], q["targets"]) for q in p7] == [(q["kind"], q["targets"]) for q in p6]
    assert not any(q["kind"] == "phase" for q in p7)


@pytest.mark.parametrize("L", [16, 18, 22])
def test_global_qubit_reorders_restore_identity(qsim, L):
    """Following a plan's reorder passes as exchanges of index bits, every gate pass must find its qubits
    at local positions and the order must be the identity again after the last pass; the exchanges use
    positions >= 4 and at most 4 pairs per pass (the direct exchange kernel)."""
    n = 24
    c = W.random_pairs(n, 6, seed=7)
    for kw in (dict(mode=1, max_fused=6, precision=1, tc_min_k=5), dict(mode=0, max_fused=2)):
        p, ps = plan(qsim, c, local_qubits=L, **kw)
        logi = list(range(n))  # position -> logical qubit
        for q in ps:
            if q["kind"] == "reorder":
                assert 1 <= q["k"] <= 4
                for a, b in zip(q["targets"], q["controls"]):
                    assert a >= 4 and b >= 4
                    logi[a], logi[b] = logi[b], logi[a]
            else:
                assert all(x < L for x in q["targets"] + q["controls"])
        assert logi == list(range(n))
