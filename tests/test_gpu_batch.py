"""Batched circuits in one persistent launch (clusters for large circuits, shared memory for small ones)
against the FP64 oracle: per-circuit <Z_i> and <Z_i Z_{i+1}> within 1e-5 (complex64 states, FP32 fused
matrices)."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qsim(gpu_lib):
    from paper_2511_14664_gb300 import qsim as q
    return q


def oracle_z(c):
    psi = oracle.run(c)
    return oracle.expect_z_chain(psi, c.n)


def check(results, circuits, tol=1e-5):
    for (zi, zz), c in zip(results, circuits):
        rzi, rzz = oracle_z(c)
        np.testing.assert_allclose(zi, rzi, atol=tol, rtol=0)
        np.testing.assert_allclose(zz, rzz, atol=tol, rtol=0)


def tfim_mix(widths, steps, seed):
    rng = np.random.default_rng(seed)
    return [W.tfim_chain(n, s, float(rng.uniform(0, np.pi)), float(rng.uniform(0, np.pi)))
            for n, s in zip(widths, steps)]


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_tfim_batch_small_and_large(qsim, k):
    widths = [10, 11, 12, 13, 14, 15, 16, 17, 10, 14, 12, 16]
    steps = [3, 2, 4, 2, 3, 2, 2, 3, 5, 1, 2, 2]
    cs = tfim_mix(widths, steps, seed=k)
    b = qsim.Batch(cs, max_fused=k)
    assert b.info["input_gates"] == sum(len(c) for c in cs)
    b.execute()
    check(b.results(), cs)


def test_workspace_is_only_for_large_circuits(qsim):
    cs = tfim_mix([10, 13, 14, 20], [1, 1, 1, 1], seed=0)
    b = qsim.Batch(cs, max_fused=3)
    assert b.ws_bytes == 8 * (2**14 + 2**20)


def test_general_gates_with_controls(qsim):
    rng = np.random.default_rng(5)
    cs = []
    for n in (9, 12, 13, 15, 18):
        c = W.Circuit(n)
        for _ in range(40):
            c.append(W.random_gate(n, rng, kmax=2, cmax=1, diag_prob=0.3))
        cs.append(c)
    b = qsim.Batch(cs, max_fused=4)
    b.execute()
    check(b.results(), cs)


def test_segment_high_bits_and_graph_replay(qsim):
    cs = tfim_mix([22, 11, 19], [2, 3, 2], seed=9)
    b = qsim.Batch(cs, max_fused=4)
    b.execute(use_graph=True)
    r1 = b.results()
    b.execute(use_graph=True)  # replay of the captured graph
    r2 = b.results()
    for (a1, b1), (a2, b2) in zip(r1, r2):
        assert np.array_equal(a1, a2) and np.array_equal(b1, b2)
    check(r1, cs)


def test_autotune_then_default_width(qsim):
    cs = tfim_mix([12, 15, 17], [2, 2, 2], seed=3)
    chosen = qsim.batch_autotune(cs)
    assert all(1 <= k <= 4 for k in chosen)
    b = qsim.Batch(cs, max_fused=0)
    b.execute()
    check(b.results(), cs)


def test_rx_product_closed_form_many_widths(qsim):
    """RX(phi) on every qubit: <Z_i> = cos(phi), <Z_i Z_{i+1}> = cos(phi)^2, for widths 1..20."""
    phi = 0.7
    cs = []
    for n in range(1, 21):
        c = W.Circuit(n)
        for q in range(n):
            c.append(W.Gate((q,), (), W.RX(phi), "rx"))
        cs.append(c)
    b = qsim.Batch(cs, max_fused=4)
    b.execute()
    for (zi, zz), c in zip(b.results(), cs):
        np.testing.assert_allclose(zi, np.cos(phi), atol=1e-6)
        np.testing.assert_allclose(zz, np.cos(phi) ** 2, atol=1e-6)


def test_batch_rejects_bad_input(qsim):
    with pytest.raises(qsim.QsimError):
        qsim.Batch([W.Circuit(27)])
    c = W.Circuit(6)
    c.append(W.Gate((0, 1, 2), (3, 4), np.eye(8), "wide"))
    with pytest.raises(qsim.QsimError):
        qsim.Batch([c])
    # the one-shot call validates every circuit before any launch, and the library stays usable after it
    ok = tfim_mix([12, 20], [2, 2], seed=3)
    with pytest.raises(qsim.QsimError):
        qsim.batch_run(ok + [c], max_fused=3, precision=4, tc_min_n=16)
    r, _ = qsim.batch_run(ok, max_fused=3, precision=4, tc_min_n=16)
    check(r, ok)


def test_full_size_batch_256_tfim_chains(qsim):
    """The benchmark's batch (256 chains, 10-24 qubits, 8-32 Trotter steps, seed 4) in one launch: every
    <Z> in [-1, 1] and finite, and the circuits of up to 16 qubits against the oracle."""
    batch = W.tfim_batch(256, seed=4, nmax=24)
    cs = [c for c, _, _ in batch]
    b = qsim.Batch(cs, max_fused=0)
    b.execute(use_graph=True)
    res = b.results()
    for (zi, zz), c in zip(res, cs):
        assert np.all(np.isfinite(zi)) and np.all(np.abs(zi) <= 1 + 1e-5)
        assert np.all(np.isfinite(zz)) and np.all(np.abs(zz) <= 1 + 1e-5)
    small = [i for i, c in enumerate(cs) if c.n <= 16][:24]
    assert len(small) >= 10
    check([res[i] for i in small], [cs[i] for i in small])


@pytest.mark.parametrize("prec", [1, 4])
def test_full_size_batch_tensor_core_circuits_against_oracle(qsim, prec):
    """The same batch in the benchmark's configuration (tensor-core plans for the circuits of >= 20 qubits:
    3xTF32 with 6-qubit blocks, or FP16X3 with up to 7; on worker streams, graph replay): four of those
    circuits -- the two cheapest of 20-21 qubits and the two cheapest of 22-24 qubits -- and twelve
    persistent-launch circuits against the oracle."""
    batch = W.tfim_batch(256, seed=4, nmax=24)
    cs = [c for c, _, _ in batch]
    b = qsim.Batch(cs, max_fused=0, precision=prec, tc_min_n=20)
    assert b.info["tc_blocks"] > 0
    b.execute(use_graph=True)
    b.execute(use_graph=True)
    res = b.results()
    work = lambda i: len(cs[i]) * 2.0 ** cs[i].n
    mid = sorted((i for i, c in enumerate(cs) if 20 <= c.n <= 21), key=work)[:2]
    top = sorted((i for i, c in enumerate(cs) if c.n >= 22), key=work)[:2]
    assert len(mid) == 2 and len(top) == 2
    rest = [i for i, c in enumerate(cs) if c.n < 20][::9][:12]
    pick = mid + top + rest
    check([res[i] for i in pick], [cs[i] for i in pick])


@pytest.mark.parametrize("prec", [1, 3, 4])
def test_wide_circuits_as_tensor_core_plans(qsim, prec):
    """With a tensor-core precision, circuits of at least tc_min_n qubits run as fused tensor-core plans
    (their <Z> reduced on the device into the batch's outputs); the rest stay in the persistent launch."""
    widths = [10, 13, 14, 16, 17, 19, 15, 18]
    steps = [3, 2, 2, 3, 2, 2, 1, 2]
    cs = tfim_mix(widths, steps, seed=11)
    b = qsim.Batch(cs, max_fused=4, precision=prec, tc_min_n=16)
    assert b.info["tc_blocks"] > 0 and b.info["input_gates"] == sum(len(c) for c in cs)
    b.execute()
    r1 = b.results()
    check(r1, cs)
    b.execute(use_graph=True)
    b.execute(use_graph=True)  # replay: the tensor-core plans are captured with the persistent launch
    r2 = b.results()
    for (a1, b1), (a2, b2) in zip(r1, r2):
        assert np.array_equal(a1, a2) and np.array_equal(b1, b2)


def test_only_wide_circuits(qsim):
    cs = tfim_mix([16, 17], [2, 2], seed=12)
    b = qsim.Batch(cs, max_fused=4, precision=1, tc_min_n=13)
    b.execute(use_graph=True)
    check(b.results(), cs)


@pytest.mark.parametrize("prec", [1, 4])
def test_deep_wide_circuit_normalised(qsim, prec):
    """A 20-qubit chain with 32 Trotter steps (1248 gates) as a tensor-core plan inside a batch (3xTF32, or
    FP16X3 with 7-qubit blocks): its blocks' FP32 accumulation moves the norm by ~1e-5; the batch reports the
    normalised state's values, which stay within 1e-5 of the FP64 oracle."""
    cs = tfim_mix([20, 12], [32, 3], seed=13)
    b = qsim.Batch(cs, max_fused=4, precision=prec, tc_min_n=20)
    assert b.info["tc_blocks"] > 20
    b.execute()
    check(b.results(), cs)


def test_threshold_tuner_and_tuning_file(qsim, tmp_path):
    """The tensor-core threshold tuner times the whole batch per candidate and keeps the fastest; plans made
    with the default threshold then use it, and stay correct; the table survives a save and load."""
    cs = tfim_mix([12, 14, 16, 17, 18, 19, 20, 21, 15, 13], [2, 2, 2, 3, 2, 2, 2, 2, 3, 2], seed=21)
    best = qsim.batch_autotune_threshold(cs, precision=1)
    assert best in (14, 16, 18, 20, 22, 24, 27)
    b = qsim.Batch(cs, max_fused=0, precision=1)            # tc_min_n = 0: the tuned threshold
    wide = sum(1 for c in cs if c.n >= best)
    assert (b.info["tc_blocks"] > 0) == (wide > 0)
    b.execute(use_graph=True)
    check(b.results(), cs)
    path = tmp_path / "tune.json"
    qsim.batch_tune_save(str(path))
    qsim.batch_tune_load(str(path))
    import json
    assert json.loads(path.read_text())["tc_min_n"]["1"] == best


@pytest.mark.parametrize("prec", [0, 1, 4])
def test_one_shot_run_equals_plan_then_execute(qsim, prec):
    """qsim_batch_run (plan, run and read out in one call; the GPU starts on the planned circuits while the
    host plans the others) returns exactly what a plan executed afterwards returns, and matches the oracle."""
    widths = [10, 13, 14, 16, 17, 19, 15, 18, 20, 12]
    steps = [3, 2, 2, 3, 2, 2, 1, 2, 2, 3]
    cs = tfim_mix(widths, steps, seed=21)
    b = qsim.Batch(cs, max_fused=4, precision=prec, tc_min_n=16)
    b.execute()
    r1 = b.results()
    b.close()
    r2, info = qsim.batch_run(cs, max_fused=4, precision=prec, tc_min_n=16)
    assert info["input_gates"] == sum(len(c) for c in cs)
    assert (info["tc_blocks"] > 0) == (prec != 0)
    for (a1, b1), (a2, b2) in zip(r1, r2):
        assert np.array_equal(a1, a2) and np.array_equal(b1, b2)
    check(r2, cs)


def test_one_shot_run_small_only_and_full_size(qsim):
    """Circuits that all stay in shared memory (no workspace), and the benchmark's 256-chain batch with
    FP16X3 plans for the circuits of >= 20 qubits against plan-then-execute."""
    cs = tfim_mix([8, 10, 12, 13], [2, 3, 2, 1], seed=22)
    r, _ = qsim.batch_run(cs, max_fused=3)
    check(r, cs)
    cs = [c for c, _, _ in W.tfim_batch(256, seed=4, nmax=24)]
    b = qsim.Batch(cs, max_fused=0, precision=4, tc_min_n=20)
    b.execute()
    r1 = b.results()
    b.close()
    r2, _ = qsim.batch_run(cs, max_fused=0, precision=4, tc_min_n=20)
    for (a1, b1), (a2, b2) in zip(r1, r2):
        assert np.array_equal(a1, a2) and np.array_equal(b1, b2)
