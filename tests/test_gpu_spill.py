"""Out-of-core runs: a state held in host memory, streamed through device windows (Sec. 2.5: host memory
supplements GPU memory).

Small states against the FP64 oracle at the tolerances of the in-memory paths (complex64: max |error| <= 1e-5,
normalised infidelity <= 1e-9; complex128: 1e-12); sampling against the handle sampler; and, at 33 qubits
(64 GiB of host memory, windows of 2^28 amplitudes), the streamed run against the same circuit run in device
memory, followed by its inverse back to |0...0>.
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


def _host_basis(n, dtype, pinned=True):
    import torch
    t = torch.zeros(1 << n, dtype=torch.complex64 if dtype == 0 else torch.complex128, pin_memory=pinned)
    t[0] = 1.0
    return t


def _close(got, ref, n, dtype):
    g = np.ascontiguousarray(got.astype(np.complex128))
    err = float(np.max(np.abs(g - ref)))
    inf = oracle.infidelity(g, ref, n)
    at, it = (1e-5, 1e-9) if dtype == 0 else (1e-12, 1e-12)
    assert err <= at and inf <= it, (err, inf)


@pytest.mark.parametrize("dtype,kw", [
    (0, dict(mode=1, max_fused=6, precision=1)),      # fused 3xTF32 tensor-core blocks in every window
    (0, dict(mode=1, max_fused=6, precision=4)),      # FP16 split products
    (0, dict(mode=1, max_fused=7, precision=4)),      # FP16 split products, 7-qubit blocks where they pay
    (0, dict(mode=1, max_fused=4, precision=0)),      # CUDA-core fused blocks
    (1, dict(mode=0, max_fused=1, precision=0)),      # complex128, one pass per gate
])
def test_spill_small_against_oracle(qsim, dtype, kw):
    n = 20
    c = W.brickwork(n, 8, seed=41)
    rng = np.random.default_rng(2)
    for _ in range(30):
        c.append(W.random_gate(n, rng, kmax=2, cmax=1, diag_prob=0.3))
    host = _host_basis(n, dtype)
    info = qsim.spill_run(host, c, dtype, window_qubits=16, **kw)
    assert info["segments"] > 1 and info["windows"] == info["segments"] * 2 ** (n - 16)
    _close(host.numpy(), oracle.run(c), n, dtype)


def test_spill_pageable_memory_and_one_window(qsim):
    """Pageable host memory (numpy) works too; a window as large as the state gives one segment."""
    n = 18
    c = W.brickwork(n, 5, seed=3)
    host = np.zeros(1 << n, dtype=np.complex64)
    host[0] = 1
    info = qsim.spill_run(host, c, 0, window_qubits=15, global_slots=2, mode=1, max_fused=5, precision=1)
    assert info["global_slots"] == 2
    _close(host, oracle.run(c), n, 0)
    host[:] = 0
    host[0] = 1
    info = qsim.spill_run(host, c, 0, window_qubits=22, mode=1, max_fused=5, precision=1)
    assert info["segments"] == 1 and info["windows"] == 1
    _close(host, oracle.run(c), n, 0)


def test_spill_sampling_matches_handle_sampling(qsim):
    n = 20
    c = W.brickwork(n, 6, seed=8)
    host = _host_basis(n, 0)
    qsim.spill_run(host, c, 0, window_qubits=16, mode=1, max_fused=6, precision=1)
    st = qsim.State(n, qsim.C64)
    st.set_state(host.numpy())
    shots = 20000
    s_spill, nrm = qsim.spill_sample(host, n, 0, 16, 77, shots)
    s_dev = st.sample(77, shots)
    assert abs(nrm - st.norm()) <= 1e-9
    # the slice of each shot comes from FP64 prefix sums of slice totals and the uniform is rescaled inside
    # it, so an index may differ from the one-pass sampler only where rounding moves a CDF boundary
    assert np.mean(s_spill == s_dev) >= 0.999
    # and the samples follow |a_x|^2 (chi-square on the 6 lowest and the 4 highest qubits)
    from scipy.stats import chisquare
    for qs in ([0, 1, 2, 3, 4, 5], [16, 17, 18, 19]):
        p = st.probs(qs)
        key = np.zeros(shots, dtype=np.int64)
        for j, q in enumerate(qs):
            key |= ((s_spill.astype(np.int64) >> q) & 1) << j
        counts = np.bincount(key, minlength=1 << len(qs))
        assert chisquare(counts, p / p.sum() * shots).pvalue > 1e-4


def test_spill_33_qubits_against_device_run_and_back(qsim):
    """33 qubits (64 GiB host state, 9 top index bits streamed through windows of 2^28 amplitudes): the fused
    tensor-core run equals the same plan run in device memory on 8192 sampled amplitudes; the inverse
    circuit, streamed as well, returns |0...0> (norm, amplitude 0 and every sample)."""
    import torch
    n = 33
    c = W.brickwork(n, 3, seed=5)
    host = torch.empty(1 << n, dtype=torch.complex64, pin_memory=True)
    host.zero_()
    host[0] = 1.0
    kw = dict(mode=1, max_fused=6, precision=1)
    info = qsim.spill_run(host, c, 0, window_qubits=28, **kw)
    assert info["segments"] >= 2
    rng = np.random.default_rng(9)
    ys = np.sort(rng.choice(1 << n, size=8192, replace=False))
    got = host[torch.from_numpy(ys)].numpy().astype(np.complex128)
    st = qsim.State(n, qsim.C64)
    st.set_basis(0)
    st.run(c, **kw)
    ref = st.tensor[torch.from_numpy(ys).cuda()].cpu().numpy().astype(np.complex128)
    del st
    torch.cuda.empty_cache()
    assert float(np.max(np.abs(got - ref))) <= 1e-5 * 2.0 ** (-n / 2)
    qsim.spill_run(host, W.inverse(c), 0, window_qubits=28, **kw)
    assert abs(abs(complex(host[0])) - 1.0) <= 1e-4
    smp, nrm = qsim.spill_sample(host, n, 0, 28, 3, 2000)
    assert abs(nrm - 1.0) <= 1e-4 and np.all(smp == 0)
    assert info["host_bytes"] == 2 * info["segments"] * 8 * 2.0 ** n
