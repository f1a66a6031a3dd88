"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics (no GPU).

Each test checks the oracle against something other than itself: hand-derived amplitudes, closed forms,
library routines (numpy einsum / kron, scipy expm, numpy searchsorted), brute-force dense operators,
and invariants (unitarity, norm, reversibility).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from helpers import (golden_amps, golden_circuit, load_golden, pauli_dense, qft_closed_form,
                     random_state)


# ---- golden hand-derived cases -------------------------------------------------------------------
@pytest.mark.parametrize("case", load_golden()["cases"], ids=lambda c: c["name"])
def test_golden_closed_forms(case):
    c = golden_circuit(case)
    psi = oracle.run(c, basis_state=case["init"])
    np.testing.assert_allclose(psi, golden_amps(case), atol=1e-14, rtol=0)


# ---- GHZ -------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [2, 3, 5, 8, 12])
def test_ghz_amplitudes(n):
    psi = oracle.run(W.ghz(n))
    ref = np.zeros(1 << n, dtype=np.complex128)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    np.testing.assert_allclose(psi, ref, atol=1e-15, rtol=0)


# ---- QFT closed form -------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 4, 7, 10, 13])
def test_qft_closed_form(n):
    x = W.basis_index(n, 100 + n)
    psi = oracle.run(W.qft(n), basis_state=x)
    np.testing.assert_allclose(np.abs(psi), 2 ** (-n / 2), atol=1e-13, rtol=0)
    np.testing.assert_allclose(psi, qft_closed_form(n, x), atol=1e-12, rtol=0)


# ---- reversibility and norm ------------------------------------------------------------------------
def test_brickwork_then_inverse_returns_zero_state():
    c = W.brickwork(10, 8, seed=7)
    psi = oracle.run(c)
    oracle.run(W.inverse(c), psi=psi)
    ref = oracle.basis(10, 0)
    assert np.max(np.abs(psi - ref)) <= 1e-12


def test_random_gates_then_inverse_restore_state():
    n = 9
    rng = np.random.default_rng(11)
    c = W.Circuit(n)
    for _ in range(60):
        c.append(W.random_gate(n, rng, kmax=3, cmax=2, diag_prob=0.3))
    psi0 = random_state(n, 3)
    psi = oracle.run(c, psi=psi0.copy())
    oracle.run(W.inverse(c), psi=psi)
    assert np.max(np.abs(psi - psi0)) <= 1e-12


def test_norm_preserved():
    psi = oracle.run(W.brickwork(12, 6, seed=5))
    assert abs(oracle.norm2(psi, 12) - 1.0) <= 1e-12
    assert abs(np.vdot(psi, psi).real - 1.0) <= 1e-12


# ---- brute-force dense operators ---------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(6))
def test_per_gate_matches_dense_operator(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 8))
    c = W.Circuit(n)
    for _ in range(25):
        c.append(W.random_gate(n, rng, kmax=3, cmax=2, diag_prob=0.25))
    psi0 = random_state(n, seed + 50)
    a = oracle.run(c, psi=psi0.copy())
    b = oracle.dense_run(c, psi=psi0.copy())
    assert np.max(np.abs(a - b)) <= 1e-12


def test_dense_operator_is_unitary_and_controlled_identity():
    n = 5
    U = W.haar_unitary(4, np.random.default_rng(1))
    G = oracle.dense_operator(n, (3, 1), (0,), U)
    np.testing.assert_allclose(G @ G.conj().T, np.eye(1 << n), atol=1e-13)
    for x in range(1 << n):
        if not (x & 1):  # control qubit 0 clear -> identity column
            col = np.zeros(1 << n)
            col[x] = 1
            np.testing.assert_array_equal(G[:, x], col)


# ---- library routines: einsum on reshaped views --------------------------------------------------------
@pytest.mark.parametrize("q", range(9))
def test_single_qubit_gate_matches_einsum(q):
    n = 9
    U = W.haar_unitary(2, np.random.default_rng(q))
    psi0 = random_state(n, 20 + q)
    a = psi0.copy()
    oracle.apply_gate(a, n, (q,), (), U)
    v = psi0.reshape(1 << (n - q - 1), 2, 1 << q)
    b = np.einsum("ij,ajb->aib", U, v).reshape(-1)
    assert np.max(np.abs(a - b)) <= 1e-14


@pytest.mark.parametrize("t0,t1", [(0, 1), (1, 0), (2, 6), (6, 2), (0, 7)])
def test_two_qubit_gate_matches_tensordot(t0, t1):
    """Pins the target-order convention: matrix index m = b_{t0} + 2 b_{t1}."""
    n = 8
    U = W.haar_unitary(4, np.random.default_rng(t0 * 10 + t1))
    psi0 = random_state(n, 99)
    a = psi0.copy()
    oracle.apply_gate(a, n, (t0, t1), (), U)
    T = psi0.reshape([2] * n)  # axis n-1-q is qubit q
    U4 = U.reshape(2, 2, 2, 2)  # [out_b1, out_b0, in_b1, in_b0]
    ax0, ax1 = n - 1 - t0, n - 1 - t1
    out = np.tensordot(U4, T, axes=([2, 3], [ax1, ax0]))  # new axes: out_b1, out_b0, rest...
    rest = [ax for ax in range(n) if ax not in (ax0, ax1)]
    perm = np.empty(n, dtype=int)
    perm[ax1], perm[ax0] = 0, 1
    for i, ax in enumerate(rest):
        perm[ax] = 2 + i
    b = np.transpose(out, perm).reshape(-1)
    assert np.max(np.abs(a - b)) <= 1e-14


# ---- TFIM Trotter circuit vs scipy expm of Eq. 1's terms ---------------------------------------------
def test_tfim_trotter_matches_expm():
    from scipy.linalg import expm
    n, steps, th, ph = 5, 4, 0.7, 1.3
    psi = oracle.run(W.tfim_chain(n, steps, th, ph))
    Hzz = sum(pauli_dense("".join("Z" if q in (i, i + 1) else "I" for q in range(n))) for i in range(n - 1))
    Hx = sum(pauli_dense("".join("X" if q == i else "I" for q in range(n))) for i in range(n))
    Ustep = expm(-0.5j * ph * Hx) @ expm(-0.5j * th * Hzz)
    ref = np.zeros(1 << n, dtype=np.complex128)
    ref[0] = 1
    for _ in range(steps):
        ref = Ustep @ ref
    assert np.max(np.abs(psi - ref)) <= 1e-12


@pytest.mark.parametrize("lx,ly", [(3, 3), (4, 2)])
def test_tfim_lattice_trotter_matches_expm(lx, ly):
    """The periodic triangular-lattice TFIM: bonds (each site's three forward neighbours, wrapping; every
    site of a lattice with lx, ly >= 3 has six neighbours) and the Trotter circuit against expm of Eq. 1's
    two terms built from those bonds."""
    from scipy.linalg import expm
    n, steps, th, ph = lx * ly, 3, 0.9, 0.35
    bonds = W.triangular_bonds(lx, ly)
    if lx >= 3 and ly >= 3:
        assert len(bonds) == 3 * n
        deg = np.bincount(np.array(bonds).ravel(), minlength=n)
        assert np.all(deg == 6)
    assert len(set(bonds)) == len(bonds) and all(a < b for a, b in bonds)
    psi = oracle.run(W.tfim_lattice(lx, ly, steps, th, ph))
    Hzz = sum(pauli_dense("".join("Z" if q in (a, b) else "I" for q in range(n))) for a, b in bonds)
    Hx = sum(pauli_dense("".join("X" if q == i else "I" for q in range(n))) for i in range(n))
    Ustep = expm(-0.5j * ph * Hx) @ expm(-0.5j * th * Hzz)
    ref = np.zeros(1 << n, dtype=np.complex128)
    ref[0] = 1
    for _ in range(steps):
        ref = Ustep @ ref
    assert np.max(np.abs(psi - ref)) <= 1e-12


# ---- observables ------------------------------------------------------------------------------------
@pytest.mark.parametrize("phi", [0.0, 0.4, 1.1, 2.9])
def test_rx_product_expectations(phi):
    n = 6
    c = W.Circuit(n)
    for q in range(n):
        c.append(W.Gate((q,), (), W.RX(phi), "rx"))
    psi = oracle.run(c)
    zi, zz = oracle.expect_z_chain(psi, n)
    np.testing.assert_allclose(zi, math.cos(phi), atol=1e-14)
    np.testing.assert_allclose(zz, math.cos(phi) ** 2, atol=1e-14)
    for q in range(n):
        y = oracle.expect_pauli(psi, n, "".join("Y" if i == q else "I" for i in range(n)))
        x = oracle.expect_pauli(psi, n, "".join("X" if i == q else "I" for i in range(n)))
        assert abs(y - (-math.sin(phi))) <= 1e-14
        assert abs(x) <= 1e-14


@pytest.mark.parametrize("seed", range(5))
def test_pauli_expectation_matches_dense_kron(seed):
    rng = np.random.default_rng(seed)
    n = 6
    psi = random_state(n, seed)
    paulis = "".join(rng.choice(list("IXYZ"), size=n))
    ref = np.vdot(psi, pauli_dense(paulis) @ psi)
    got = oracle.expect_pauli(psi, n, paulis)
    assert abs(got - ref) <= 1e-14


def test_marginals_of_product_state():
    n = 7
    alphas = np.linspace(0.3, 2.8, n)
    c = W.Circuit(n)
    for q in range(n):
        c.append(W.Gate((q,), (), W.RY(alphas[q]), "ry"))
    psi = oracle.run(c)
    p1 = np.sin(alphas / 2) ** 2  # P(qubit q = 1)
    for qs in [(0,), (3, 1), (6, 2, 4), tuple(range(n))]:
        got = oracle.probs(psi, n, qs)
        ref = np.ones(1 << len(qs))
        for m in range(1 << len(qs)):
            for j, q in enumerate(qs):
                ref[m] *= p1[q] if (m >> j) & 1 else 1 - p1[q]
        np.testing.assert_allclose(got, ref, atol=1e-14)
    assert abs(oracle.probs(psi, n, range(n)).sum() - 1) <= 1e-14


# ---- sampling -------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 5, 10])
def test_sampler_matches_searchsorted(n):
    psi = random_state(n, n)
    psi[np.arange(0, 1 << n, 3)] = 0  # zero-probability indices must never be drawn
    u = oracle.uniforms(1234 + n, 4000)
    got = oracle.sample(psi, n, u)
    p = np.abs(psi) ** 2
    cdf = np.cumsum(p)
    ref = np.searchsorted(cdf, u * cdf[-1], side="right")
    assert np.array_equal(got, ref.astype(np.uint64))
    assert np.all(p[got.astype(np.int64)] > 0)


def test_sampler_frequencies_chi2():
    from scipy.stats import chisquare
    n = 6
    psi = random_state(n, 77)
    p = np.abs(psi) ** 2
    u = oracle.uniforms(42, 200_000)
    s = oracle.sample(psi, n, u).astype(np.int64)
    counts = np.bincount(s, minlength=1 << n)
    assert chisquare(counts, p * len(s)).pvalue > 1e-4


def test_splitmix64_uniforms():
    from scipy.stats import kstest
    u = oracle.uniforms(2024, 100_000)
    assert np.all((u >= 0) & (u < 1))
    assert len(np.unique(u)) == len(u)
    assert kstest(u, "uniform").pvalue > 1e-4
    assert oracle.splitmix64(2024, 5) >> 11 == int(round(u[5] * 2**53))


def test_splitmix64_published_vector():
    """The oracle's generator against the published SplitMix64 outputs for seed 1234567 (a wrong increment,
    shift or finaliser constant changes every one of them), and the uniforms as their top 53 bits."""
    g = load_golden("splitmix64.json")
    want = [int(v) for v in g["outputs"]]
    assert [oracle.splitmix64(g["seed"], i) for i in range(len(want))] == want
    u = oracle.uniforms(g["seed"], len(want))
    assert [int(x * 2**53) for x in u] == [v >> 11 for v in want]


# ---- inner product and infidelity (the checker behind every GPU parity bound) ------------------------------
def test_inner_hand_values():
    """<a|b> = sum_x conj(a_x) b_x (Sec. 2.1: amplitudes of basis states), on values fixed by hand: the
    conjugate sits on the left operand, so <a|i a> = +i and <i a|a> = -i."""
    s = 1 / math.sqrt(2)
    zero = np.array([1, 0], dtype=np.complex128)
    plus = np.array([s, s], dtype=np.complex128)
    assert abs(oracle.inner(zero, plus, 1) - s) <= 1e-16
    a = np.array([0.6, 0.8j], dtype=np.complex128)      # |a|^2 = 1
    assert abs(oracle.inner(a, a, 1) - 1.0) <= 1e-15
    assert abs(oracle.inner(a, 1j * a, 1) - 1j) <= 1e-15
    assert abs(oracle.inner(1j * a, a, 1) + 1j) <= 1e-15
    b = np.array([1, 1j], dtype=np.complex128)          # <a|b> = 0.6 + conj(0.8 i) i = 0.6 + 0.8
    assert abs(oracle.inner(a, b, 1) - 1.4) <= 1e-15
    c = np.array([1j, 0], dtype=np.complex128)          # <a|c> = 0.6 i, <c|a> = -0.6 i
    assert abs(oracle.inner(a, c, 1) - 0.6j) <= 1e-15
    assert abs(oracle.inner(c, a, 1) + 0.6j) <= 1e-15


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_inner_matches_numpy_vdot(seed):
    n = 9
    a, b = random_state(n, seed), random_state(n, seed + 100) * (0.3 - 0.7j)
    assert abs(oracle.inner(a, b, n) - np.vdot(a, b)) <= 1e-13


def test_infidelity_special_cases():
    """1 - |<a|b>|^2 / (<a|a><b|b>) (normalised) and 1 - |<a|b>|^2 (unnormalised) on closed forms."""
    zero = np.array([1, 0], dtype=np.complex128)
    one = np.array([0, 1], dtype=np.complex128)
    assert oracle.infidelity(zero, one, 1) == pytest.approx(1.0, abs=1e-15)         # orthogonal
    psi = random_state(8, 5)
    assert oracle.infidelity(psi, np.exp(0.7j) * psi, 8) <= 1e-14                   # global phase
    for th in (0.0, 0.3, 1.0, math.pi / 3):
        v = np.array([math.cos(th), math.sin(th)], dtype=np.complex128)
        assert oracle.infidelity(v, zero, 1) == pytest.approx(math.sin(th) ** 2, abs=1e-15)
    two = 2.0 * psi                                                                  # norms 1 and 4
    assert oracle.infidelity(psi, two, 8) <= 1e-14
    assert oracle.infidelity(psi, two, 8, normalised=False) == pytest.approx(1.0 - 4.0, abs=1e-12)


# ---- QPE with exactly representable phases ------------------------------------------------------------
@pytest.mark.parametrize("t,a", [(3, 5), (5, 17), (7, 100), (8, 255)])
def test_qpe_exact_phase(t, a):
    c, expect = W.qpe(t, a)
    psi = oracle.run(c)
    p = oracle.probs(psi, c.n, range(t))
    assert abs(p[expect] - 1.0) <= 1e-12


# ---- invalid input ---------------------------------------------------------------------------------------
def test_oracle_rejects_bad_qubits():
    psi = oracle.basis(3)
    with pytest.raises(ValueError):
        oracle.apply_gate(psi, 3, (0, 0), (), np.eye(4))
    with pytest.raises(ValueError):
        oracle.apply_gate(psi, 3, (3,), (), np.eye(2))
    with pytest.raises(ValueError):
        oracle.apply_gate(psi, 3, (1,), (1,), np.eye(2))


def test_paper_gate_count_rcs():
    facts = load_golden()["paper_facts"]
    for n in (4, 9, 33):
        assert len(W.rcs(n, seed=1)) == facts["rcs_gates_per_qubit"] * n
