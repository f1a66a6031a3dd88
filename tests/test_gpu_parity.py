"""GPU parity: every kernel against the FP64 oracle on the same seeded inputs, through the C ABI.

Tolerances (stated per result): complex64 -- max |amplitude error| <= 1e-5 and normalised infidelity
1 - |<a|b>|^2 / (|a|^2 |b|^2) <= 1e-9; complex128 -- max |amplitude error| <= 1e-12 (and infidelity
<= 1e-12). Integer results (samples) are compared exactly.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from helpers import qft_closed_form, random_state

pytestmark = pytest.mark.gpu

TOL = {0: (1e-5, 1e-9), 1: (1e-12, 1e-12)}


def close(psi_gpu, psi_ref, n, dtype, amp_tol=None, inf_tol=None):
    at, it = TOL[dtype]
    at = amp_tol if amp_tol is not None else at
    it = inf_tol if inf_tol is not None else it
    g = psi_gpu.astype(np.complex128)
    err = float(np.max(np.abs(g - psi_ref)))
    inf = oracle.infidelity(np.ascontiguousarray(g), psi_ref, n)
    assert err <= at, f"max amplitude error {err:.3e} > {at:.0e}"
    assert inf <= it, f"infidelity {inf:.3e} > {it:.0e}"
    return err, inf


def make_state(qsim, n, dtype, psi0=None, basis=0):
    st = qsim.State(n, dtype)
    if psi0 is None:
        st.set_basis(basis)
    else:
        st.set_state(psi0)
    return st


@pytest.fixture(scope="module")
def qsim(gpu_lib):
    from paper_2511_14664_gb300 import qsim as q
    return q


DT = [0, 1]


# ---- basics ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", DT)
def test_set_basis_and_roundtrip(qsim, dtype):
    for n, x in [(1, 1), (5, 17), (13, 4095), (20, 777777)]:
        st = make_state(qsim, n, dtype, basis=x)
        psi = st.get_state()
        ref = oracle.basis(n, x)
        assert np.array_equal(psi.astype(np.complex128), ref)
    psi0 = random_state(9, 1)
    st = make_state(qsim, 9, dtype, psi0=psi0)
    np.testing.assert_allclose(st.get_state(), psi0.astype(st.get_state().dtype), atol=0)


# ---- single gates on every target ---------------------------------------------------------------------
@pytest.mark.parametrize("dtype", DT)
@pytest.mark.parametrize("n", [3, 7, 13])
def test_single_qubit_every_target(qsim, dtype, n):
    rng = np.random.default_rng(n)
    psi0 = random_state(n, n + 10)
    for q in range(n):
        U = W.haar_unitary(2, rng)
        st = make_state(qsim, n, dtype, psi0=psi0)
        st.apply_gate((q,), (), U)
        ref = psi0.copy()
        oracle.apply_gate(ref, n, (q,), (), U)
        close(st.get_state(), ref, n, dtype)


@pytest.mark.parametrize("dtype", DT)
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7, 8])
def test_dense_gates_with_controls(qsim, dtype, k):
    n = 12
    rng = np.random.default_rng(100 + k)
    for trial in range(4):
        nc = int(rng.integers(0, 3))
        qs = rng.permutation(n)[: k + nc]
        t, c = tuple(int(x) for x in qs[:k]), tuple(int(x) for x in qs[k:])
        U = W.haar_unitary(1 << k, rng)
        psi0 = random_state(n, 1000 * k + trial)
        st = make_state(qsim, n, dtype, psi0=psi0)
        st.apply_gate(t, c, U)
        ref = psi0.copy()
        oracle.apply_gate(ref, n, t, c, U)
        close(st.get_state(), ref, n, dtype)


@pytest.mark.parametrize("dtype", DT)
def test_wide_gates_single_group_diagonal_and_fused(qsim, dtype):
    """7- and 8-qubit gates: one group only (n = k), a diagonal 7-qubit gate (dense path), and the
    SIMT single-block entry point."""
    rng = np.random.default_rng(78)
    for n, k in ((7, 7), (8, 8), (9, 8)):
        t = tuple(int(x) for x in rng.permutation(n)[:k])
        U = W.haar_unitary(1 << k, rng)
        psi0 = random_state(n, 11 * n + k)
        st = make_state(qsim, n, dtype, psi0=psi0)
        st.apply_gate(t, (), U)
        ref = psi0.copy()
        oracle.apply_gate(ref, n, t, (), U)
        close(st.get_state(), ref, n, dtype)
    n = 13
    dg = np.diag(np.exp(1j * rng.uniform(0, 2 * np.pi, size=128)))
    t = (12, 0, 5, 3, 9, 1, 7)
    psi0 = random_state(n, 3)
    st = make_state(qsim, n, dtype, psi0=psi0)
    st.apply_gate(t, (2,), dg)
    ref = psi0.copy()
    oracle.apply_gate(ref, n, t, (2,), dg)
    close(st.get_state(), ref, n, dtype)
    U = W.haar_unitary(128, rng)
    st = make_state(qsim, n, dtype, psi0=psi0)
    st.apply_fused(t, U, qsim.PREC_SIMT)
    ref = psi0.copy()
    oracle.apply_gate(ref, n, t, (), U)
    close(st.get_state(), ref, n, dtype)


@pytest.mark.parametrize("dtype", DT)
@pytest.mark.parametrize("mode", [0, 1])
def test_plans_with_wide_gates(qsim, dtype, mode):
    """Circuits mixing 7- and 8-qubit gates with small ones, plain and fused (wider gates than max_fused
    become passes of their own)."""
    n = 14
    rng = np.random.default_rng(4 + mode)
    c = W.Circuit(n)
    for i in range(30):
        c.append(W.random_gate(n, rng, kmax=2, cmax=1, diag_prob=0.3))
        if i % 10 == 4:
            k = 7 + (i // 10) % 2
            qs = rng.permutation(n)[: k + 1]
            c.append(W.Gate(tuple(int(x) for x in qs[:k]), (int(qs[k]),) if i == 14 else (),
                            W.haar_unitary(1 << k, rng), f"u{k}"))
    psi0 = random_state(n, 40 + mode)
    st = make_state(qsim, n, dtype, psi0=psi0)
    st.run(c, mode=mode, max_fused=4)
    close(st.get_state(), oracle.run(c, psi=psi0.copy()), n, dtype)


@pytest.mark.parametrize("dtype", DT)
def test_low_targets_and_ragged_small_states(qsim, dtype):
    """Targets in the vector lanes (bit 0), in the warp (1..5) and above; n below a warp chunk."""
    rng = np.random.default_rng(5)
    for n in (1, 2, 4, 6, 9):
        for q in range(n):
            for ctl in ([], [(q + 1) % n] if n > 1 else []):
                U = W.haar_unitary(2, rng)
                psi0 = random_state(n, 7 * n + q)
                st = make_state(qsim, n, dtype, psi0=psi0)
                st.apply_gate((q,), tuple(ctl), U)
                ref = psi0.copy()
                oracle.apply_gate(ref, n, (q,), tuple(ctl), U)
                close(st.get_state(), ref, n, dtype)


@pytest.mark.parametrize("dtype", DT)
def test_diagonal_gates(qsim, dtype):
    n = 11
    rng = np.random.default_rng(9)
    psi0 = random_state(n, 3)
    cases = [((0, 1), (), W.CZ()), ((4, 9), (), W.CZ()), ((3,), (0,), W.CP(0.3)), ((0,), (7,), W.CP(1.1)),
             ((2, 5), (), W.RZZ(0.7)), ((6,), (), W.RZ(0.4)), ((1, 8), (3, 10), W.RZZ(2.2))]
    for _ in range(4):
        g = W.random_gate(n, rng, kmax=4, cmax=2, diag_prob=1.0)
        cases.append((g.targets, g.controls, g.matrix))
    for t, c, U in cases:
        st = make_state(qsim, n, dtype, psi0=psi0)
        st.apply_gate(t, c, U)
        ref = psi0.copy()
        oracle.apply_gate(ref, n, t, c, U)
        close(st.get_state(), ref, n, dtype)


# ---- qubit reorder --------------------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", DT)
@pytest.mark.parametrize("pairs", [[(0, 13)], [(2, 3)], [(0, 5), (1, 14), (2, 9)], [(10, 11), (12, 13)],
                                   [(4, 9), (5, 14), (15, 6)], [(3, 8), (4, 9), (5, 10), (6, 11)],
                                   [(0, 8), (1, 9), (2, 10), (3, 11), (4, 12), (5, 13), (6, 14), (7, 15)]])
def test_swap_qubits_matches_swap_gates(qsim, dtype, pairs):
    n = 16
    psi0 = random_state(n, 44)
    st = make_state(qsim, n, dtype, psi0=psi0)
    st.swap_qubits([a for a, _ in pairs], [b for _, b in pairs])
    ref = psi0.copy()
    for a, b in pairs:
        oracle.apply_gate(ref, n, (a, b), (), W.SWAP())
    # a permutation moves values without arithmetic: bit-exact
    assert np.array_equal(st.get_state().astype(np.complex128), ref.astype(st.get_state().dtype).astype(np.complex128))


def test_reorder_then_local_gate_equals_global_gate(qsim):
    """The paper's global/local split (Sec. 2.1): the top qubits act as 'global'; swapping one down,
    applying the gate locally and swapping back equals applying it in place."""
    n, dtype = 15, 0
    rng = np.random.default_rng(8)
    U = W.haar_unitary(4, rng)
    psi0 = random_state(n, 12)
    a = make_state(qsim, n, dtype, psi0=psi0)
    a.apply_gate((14, 3), (), U)
    b = make_state(qsim, n, dtype, psi0=psi0)
    b.swap_qubits([14], [5])
    b.apply_gate((5, 3), (), U)
    b.swap_qubits([14], [5])
    assert np.array_equal(a.get_state(), b.get_state())


# ---- circuits ----------------------------------------------------------------------------------------------
def test_brickwork_14q_complex128_plain(qsim):
    """14-qubit random brickwork, 20 layers, complex128, plain per-gate path: full state vs oracle."""
    c = W.brickwork(14, 20, seed=1)
    st = make_state(qsim, 14, 1)
    info = st.run(c, mode=qsim.RUN_PLAIN)
    assert info["input_gates"] == len(c) == 410
    close(st.get_state(), oracle.run(c), 14, 1)


@pytest.mark.parametrize("dtype", DT)
def test_ghz(qsim, dtype):
    n = 18
    st = make_state(qsim, n, dtype)
    st.run(W.ghz(n))
    psi = st.get_state()
    assert abs(psi[0] - 1 / math.sqrt(2)) <= TOL[dtype][0]
    assert abs(psi[-1] - 1 / math.sqrt(2)) <= TOL[dtype][0]
    assert np.max(np.abs(psi[1:-1])) == 0


@pytest.mark.parametrize("mode,k", [(0, 0), (1, 2), (1, 4), (1, 5), (1, 6)])
def test_qft_closed_form(qsim, mode, k):
    n = 16
    x = W.basis_index(n, 2)
    st = make_state(qsim, n, 0, basis=x)
    st.run(W.qft(n), mode=mode, max_fused=max(k, 1))
    close(st.get_state(), qft_closed_form(n, x), n, 0)


def test_full_size_qft28_tensor_cores_closed_form(qsim):
    """The 28-qubit QFT of the benchmark (2 GiB complex64), in the configuration it times (6-qubit 3xTF32
    blocks with phase epilogues and phase passes): 8192 sampled amplitudes against the closed form."""
    import torch
    n = 28
    x = W.basis_index(n, 2)
    p = qsim.Plan(W.qft(n), qsim.C64, mode=1, max_fused=6, precision=1, tc_min_k=5, use_graph=True)
    st = make_state(qsim, n, 0, basis=x)
    p.execute(st)
    rng = np.random.default_rng(5)
    ys = np.sort(rng.choice(1 << n, size=8192, replace=False))
    got = st.tensor[torch.from_numpy(ys).cuda()].cpu().numpy().astype(np.complex128)
    ph = (np.uint64(x) * ys.astype(np.uint64)) & np.uint64((1 << n) - 1)
    ref = np.exp(2j * math.pi * ph.astype(np.float64) / (1 << n)) / math.sqrt(1 << n)
    # relative 1e-5 of the amplitudes' magnitude 2^-14 (6.1e-10 absolute), and the normalised infidelity of
    # the sampled sub-vector
    assert float(np.max(np.abs(got - ref))) <= 1e-5 * 2.0 ** (-n / 2)
    ov = np.vdot(ref, got)
    assert 1.0 - abs(ov) ** 2 / (np.vdot(ref, ref).real * np.vdot(got, got).real) <= 1e-9
    assert abs(st.norm() - 1.0) <= 1e-4


def test_brickwork_14q_complex128_fused_graph(qsim):
    """The 14-qubit complex128 brickwork in the benchmark's configuration (4-qubit SIMT fusion, CUDA graph
    replay): full state against the oracle at the complex128 bar, twice in a row."""
    n = 14
    c = W.brickwork(n, 20, seed=1)
    ref = oracle.run(c)
    p = qsim.Plan(c, 1, mode=1, max_fused=4, use_graph=True)
    st = make_state(qsim, n, 1)
    for _ in range(2):
        st.set_basis(0)
        p.execute(st)
        close(st.get_state(), ref, n, 1)


@pytest.mark.parametrize("dtype", DT)
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_fused_simt_random_circuit(qsim, dtype, k):
    n = 13
    rng = np.random.default_rng(k)
    c = W.Circuit(n)
    for _ in range(80):
        c.append(W.random_gate(n, rng, kmax=2, cmax=1, diag_prob=0.3))
    for g in W.brickwork(n, 3, seed=k).gates:
        c.append(g)
    psi0 = random_state(n, k)
    st = make_state(qsim, n, dtype, psi0=psi0)
    info = st.run(c, mode=qsim.RUN_FUSED, max_fused=k, precision=qsim.PREC_SIMT)
    assert info["passes"] <= len(c)
    close(st.get_state(), oracle.run(c, psi=psi0.copy()), n, dtype)


def test_fused_reduces_passes_on_brickwork(qsim):
    c = W.brickwork(20, 10, seed=3)
    plain = qsim.Plan(c, mode=qsim.RUN_PLAIN)
    fused = qsim.Plan(c, mode=qsim.RUN_FUSED, max_fused=5)
    assert plain.info["passes"] == len(c)
    assert fused.info["passes"] < len(c) / 4
    st = make_state(qsim, 20, 0)
    fused.execute(st)
    close(st.get_state(), oracle.run(c), 20, 0)


def test_plan_graph_replay(qsim):
    c = W.brickwork(16, 6, seed=4)
    ref = oracle.run(c)
    p = qsim.Plan(c, mode=qsim.RUN_FUSED, max_fused=4, use_graph=True)
    st = make_state(qsim, 16, 0)
    for _ in range(3):  # capture on first execution, replay afterwards
        st.set_basis(0)
        p.execute(st)
        close(st.get_state(), ref, 16, 0)


@pytest.mark.parametrize("mode,k", [(0, 1), (1, 4)])
def test_complex128_large_state_elementwise(qsim, mode, k):
    """Complex128 at 21 qubits, where dense gates on up to 4 targets (without controls) leave 2^17 or more
    groups and so take the large-state register-gather kernel rather than the lane-split one: every
    amplitude against the oracle at the complex128 bar, per-gate and fused."""
    n = 21
    rng = np.random.default_rng(210 + k)
    c = W.Circuit(n)
    for _ in range(24):
        c.append(W.random_gate(n, rng, kmax=4, cmax=0, diag_prob=0.0))
    for _ in range(12):
        c.append(W.random_gate(n, rng, kmax=2, cmax=1, diag_prob=0.3))
    for g in W.brickwork(n, 4, seed=k).gates:
        c.append(g)
    psi0 = random_state(n, 5)
    st = make_state(qsim, n, 1, psi0=psi0)
    st.run(c, mode=mode, max_fused=k)
    close(st.get_state(), oracle.run(c, psi=psi0.copy()), n, 1)


def test_circuit_then_inverse_large(qsim):
    """A property that holds at any size: the circuit followed by its inverse returns |0...0>."""
    n = 26
    c = W.brickwork(n, 6, seed=11)
    st = make_state(qsim, n, 0)
    st.run(c, mode=qsim.RUN_FUSED, max_fused=5)
    st.run(W.inverse(c), mode=qsim.RUN_FUSED, max_fused=5)
    assert abs(st.norm() - 1.0) <= 1e-5
    p = st.probs([0, 1, 2, 3])
    assert abs(p[0] - 1.0) <= 1e-5


# ---- readout -------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", DT)
@pytest.mark.parametrize("n", [3, 11, 12, 17])
def test_norm_probs_expectations(qsim, dtype, n):
    psi = random_state(n, 70 + n)
    st = make_state(qsim, n, dtype, psi0=psi)
    ref = st.get_state().astype(np.complex128)  # the exact values the GPU holds
    assert abs(st.norm() - oracle.norm2(ref, n)) <= 1e-13
    rng = np.random.default_rng(n)
    for qs in ([0], [n - 1], list(range(min(n, 5))), list(rng.permutation(n)[: min(n, 7)]), [n - 1, 0]):
        got = st.probs([int(q) for q in qs])
        np.testing.assert_allclose(got, oracle.probs(ref, n, qs), atol=1e-14, rtol=0)
    for _ in range(6):
        P = "".join(rng.choice(list("IXYZ"), size=n))
        got = st.expect_pauli(P)
        exp = oracle.expect_pauli(ref, n, P)
        assert abs(got - exp) <= 1e-13, (P, got, exp)
    zi, zz = st.expect_z()
    rzi, rzz = oracle.expect_z_chain(ref, n)
    np.testing.assert_allclose(zi, rzi, atol=1e-13, rtol=0)
    np.testing.assert_allclose(zz, rzz, atol=1e-13, rtol=0)


def test_expect_z_large_segments(qsim):
    """Bits above the 4096-amplitude segment go through the segment-sum path."""
    n = 22
    c = W.tfim_chain(n, 3, 0.9, 0.4)
    st = make_state(qsim, n, 0)
    st.run(c)
    ref = st.get_state().astype(np.complex128)
    zi, zz = st.expect_z()
    rzi, rzz = oracle.expect_z_chain(ref, n)
    np.testing.assert_allclose(zi, rzi, atol=1e-12, rtol=0)
    np.testing.assert_allclose(zz, rzz, atol=1e-12, rtol=0)


@pytest.mark.parametrize("dtype", DT)
def test_rx_product_closed_form(qsim, dtype):
    n, phi = 14, 0.83
    c = W.Circuit(n)
    for q in range(n):
        c.append(W.Gate((q,), (), W.RX(phi), "rx"))
    st = make_state(qsim, n, dtype)
    st.run(c)
    zi, zz = st.expect_z()
    tol = 1e-6 if dtype == 0 else 1e-13
    np.testing.assert_allclose(zi, math.cos(phi), atol=tol)
    np.testing.assert_allclose(zz, math.cos(phi) ** 2, atol=tol)


@pytest.mark.parametrize("dtype", DT)
@pytest.mark.parametrize("n", [1, 6, 12, 15, 23])
def test_sampling_matches_oracle(qsim, dtype, n):
    psi = random_state(n, 5 + n)
    psi[np.arange(0, 1 << n, 5)] = 0
    st = make_state(qsim, n, dtype, psi0=psi)
    ref = st.get_state().astype(np.complex128)
    u = oracle.uniforms(99 + n, 5000)
    got = st.sample_uniforms(u)
    exp = oracle.sample(ref, n, u)
    mism = int(np.sum(got != exp))
    assert mism == 0, f"{mism} of {len(u)} samples differ"
    got2 = st.sample(99 + n, 5000)  # device-side SplitMix64 gives the same uniforms
    assert np.array_equal(got2, exp)


@pytest.mark.parametrize("dtype", DT)
@pytest.mark.parametrize("n", [9, 12, 17, 21])
def test_expect_z_and_sample_one_pass(qsim, dtype, n):
    """The combined readout equals the separate calls: <Z> exactly, and the shots are the oracle's inverse
    CDF on the GPU's own state with the same uniforms (segment sums from the <Z> pass)."""
    c = W.brickwork(n, 6, seed=n)
    st = make_state(qsim, n, dtype)
    st.run(c, mode=1, max_fused=4)
    zi, zz, smp = st.expect_z_and_sample(17, 700)
    zi2, zz2 = st.expect_z()
    assert np.array_equal(zi, zi2) and np.array_equal(zz, zz2)
    psi = np.ascontiguousarray(st.get_state().astype(np.complex128))
    assert np.array_equal(smp, oracle.sample(psi, n, oracle.uniforms(17, 700)))
    assert np.array_equal(st.sample(17, 700), smp)


def test_inner_product(qsim):
    n = 15
    a, b = random_state(n, 1), random_state(n, 2)
    sa, sb = make_state(qsim, n, 0, psi0=a), make_state(qsim, n, 0, psi0=b)
    ra, rb = sa.get_state().astype(np.complex128), sb.get_state().astype(np.complex128)
    assert abs(sa.inner(sb) - oracle.inner(ra, rb, n)) <= 1e-13


# ---- argument errors -----------------------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", DT)
@pytest.mark.parametrize("n,qs", [
    (17, "perm13"),      # 12 low marginal bits + 1 high: one bin group per high value, chunked (S > 1)
    (17, "perm17"),      # the whole distribution in a permuted bit order (no fold, S = 1)
    (25, "high13"),      # all marginal bits above the 4096-amplitude segment: every low bit folded
    (20, "mixed15"),     # a mix of low and high marginal bits in random order
])
def test_probs_wide_marginals(qsim, dtype, n, qs):
    """Marginals over more than 12 qubits (bins beyond shared memory) against the FP64 oracle."""
    psi = random_state(n, 300 + n)
    st = make_state(qsim, n, dtype, psi0=psi)
    ref = st.get_state().astype(np.complex128)
    rng = np.random.default_rng(len(qs) + n)
    if qs == "perm13":
        q = [int(x) for x in rng.permutation(12)] + [int(rng.integers(12, n))]
    elif qs == "perm17":
        q = [int(x) for x in rng.permutation(n)]
    elif qs == "high13":
        q = [int(x) for x in rng.permutation(np.arange(12, n))]
    else:
        q = [int(x) for x in rng.permutation(n)[:15]]
    got = st.probs(q)
    np.testing.assert_allclose(got, oracle.probs(ref, n, q), atol=1e-14, rtol=0)
    if len(q) == n:
        # the full distribution is |psi|^2 with the index bits permuted
        m = np.arange(1 << n, dtype=np.int64)
        x = np.zeros_like(m)
        for j, qj in enumerate(q):
            x |= ((m >> j) & 1) << qj
        np.testing.assert_allclose(got, np.abs(ref[x]) ** 2, atol=1e-15, rtol=0)


@pytest.mark.parametrize("dtype", DT)
def test_probs_small_state_many_bins(qsim, dtype):
    """n < 12 with 8..11 marginal qubits (more results than the fixed-size result buffer holds)."""
    n = 11
    psi = random_state(n, 5)
    st = make_state(qsim, n, dtype, psi0=psi)
    ref = st.get_state().astype(np.complex128)
    rng = np.random.default_rng(9)
    for nq in (8, 11):
        q = [int(x) for x in rng.permutation(n)[:nq]]
        np.testing.assert_allclose(st.probs(q), oracle.probs(ref, n, q), atol=1e-14, rtol=0)


def test_probs_limits(qsim):
    st = make_state(qsim, 14, 0)
    with pytest.raises(qsim.QsimError) as e:
        st.probs(list(range(14)) + [3])
    assert e.value.code == 1
    with pytest.raises(qsim.QsimError) as e:
        st.probs(list(range(15)))  # more qubits than the state has
    assert e.value.code == 1
    p = st.probs(list(range(14)))  # |0...0>: all weight in bin 0
    assert p[0] == 1.0 and p[1:].sum() == 0.0


def test_errors(qsim):
    st = make_state(qsim, 6, 0)
    for t, c in [((6,), ()), ((1, 1), ()), ((2,), (2,)), ((-1,), ())]:
        with pytest.raises(qsim.QsimError) as e:
            st.apply_gate(t, c, np.eye(1 << len(t)))
        assert e.value.code == 1
    with pytest.raises(qsim.QsimError) as e:
        st.apply_gate((0,), (), np.array([[1, 1], [0, 1]]))
    assert e.value.code == 1
    with pytest.raises(qsim.QsimError):
        st.probs([0, 0])
    with pytest.raises(qsim.QsimError) as e:
        st.apply_gate(tuple(range(6)) + (0,), (), np.eye(128))
    assert e.value.code in (1, 5)
    with pytest.raises(qsim.QsimError):
        st.expect_pauli("XXQXXX")
    with pytest.raises(qsim.QsimError):
        st.set_basis(64)
    # state unchanged by rejected calls
    st.set_basis(3)
    with pytest.raises(qsim.QsimError):
        st.apply_gate((9,), (), np.eye(2))
    assert st.get_state()[3] == 1


# ---- global / local index bits: reorder passes before gates on "global" qubits -------------------------------
@pytest.mark.parametrize("mode,k,local", [(0, 1, 12), (0, 1, 10), (1, 4, 12), (1, 2, 9)])
def test_local_qubits_reorder_plan(qsim, mode, k, local):
    """Random U(4) layers on seeded matchings (most pairs span high qubits), run with the top qubits treated
    as global index bits: the plan inserts reorder passes, and the result equals the oracle's."""
    n = 16
    c = W.random_pairs(n, 6, seed=5)
    st = make_state(qsim, n, 0)
    info = st.run(c, mode=mode, max_fused=k, local_qubits=local)
    assert info["reorders"] > 0
    close(st.get_state(), oracle.run(c), n, 0)


@pytest.mark.parametrize("prec,k", [(1, 6), (4, 6), (4, 7)])
def test_local_qubits_with_tensor_cores(qsim, prec, k):
    """Global-qubit plans (reorder passes) with 3xTF32 or FP16X3 blocks (width 7 stays 6 with global qubits)."""
    n = 17
    c = W.brickwork(n, 8, seed=6)
    st = make_state(qsim, n, 0)
    info = st.run(c, mode=1, max_fused=k, precision=prec, tc_min_k=5, local_qubits=14)
    assert info["reorders"] > 0 and info["tc_blocks"] > 0
    close(st.get_state(), oracle.run(c), n, 0)


def test_full_size_34q_reorder_and_sampling(qsim):
    """At the 34-qubit size (128 GiB complex64), in the configuration the benchmark times (top 4 qubits
    global, reorder passes): properties that hold at any size -- the norm stays 1 and 10^5 samples follow
    the GPU's own 8-qubit marginal (chi-square), and their indices are valid."""
    import torch
    from scipy.stats import chisquare
    free = torch.cuda.mem_get_info()[0]
    if free < (2**34) * 8 + (4 << 30):
        pytest.skip("needs 132 GiB of free device memory")
    n = 34
    c = W.random_pairs(n, 2, seed=5)
    st = make_state(qsim, n, 0)
    info = st.run(c, mode=0, max_fused=2, local_qubits=30)
    assert info["reorders"] > 0
    assert abs(st.norm() - 1.0) <= 1e-4
    qs = [0, 5, 11, 17, 22, 28, 31, 33]
    marg = st.probs(qs)
    s = st.sample(6, 100000).astype(np.int64)
    assert s.max() < 2**n
    idx = np.zeros(len(s), dtype=np.int64)
    for j, q in enumerate(qs):
        idx |= ((s >> q) & 1) << j
    counts = np.bincount(idx, minlength=256)
    expected = marg / marg.sum() * len(s)
    keep = expected > 5
    assert chisquare(counts[keep], expected[keep] * counts[keep].sum() / expected[keep].sum()).pvalue > 1e-4
    del st
    torch.cuda.empty_cache()
