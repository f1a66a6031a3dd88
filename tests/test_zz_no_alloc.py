"""The allocation-free sampling entry point (qsim_sample_noalloc), called through the C ABI.

It serves callers that may not allocate device memory (a framework owning all GPU memory in its own pool,
or a latency-critical path): its scratch is a fixed array inside the library. Its samples must equal those
of the handle-based qsim_sample for the same state and seed -- integer indices, compared exactly -- on two
calls in a row, since every call reuses the same scratch. This file is collected last so that a failure
here, with -x, leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qsim(gpu_lib):
    from paper_2511_14664_gb300 import qsim as q
    return q


@pytest.mark.parametrize("dtype,n", [(0, 16), (1, 13), (0, 9)])
def test_noalloc_sampling_matches_handle_sampling(qsim, dtype, n):
    import torch
    st = qsim.State(n, dtype)
    st.set_basis(0)
    st.run(W.brickwork(n, 3, seed=21))
    shots = 3000
    out = torch.zeros(shots, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    L = qsim.lib()
    for seed in (11, 12):  # two calls in a row share (and overwrite) the static scratch
        rc = L.qsim_sample_noalloc(ctypes.c_void_p(st.tensor.data_ptr()), n, dtype, seed, shots,
                                   ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, L.qsim_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint64)
        ref = st.sample(seed, shots)
        assert np.array_equal(got, ref)


def _max_shots(n):
    """Largest request the 8 MiB scratch holds at n qubits: uniforms | segment sums | chunk sums, each region
    rounded up to 256 bytes."""
    up = lambda b: (b + 255) & ~255
    nseg = 1 << (n - min(n, 12))
    rest = up(8 * nseg) + up(8 * ((nseg + 1023) // 1024))
    return ((8 << 20) - rest) // 8 // 32 * 32   # a multiple of 32 uniforms fills its region exactly


def test_noalloc_at_the_scratch_limit(qsim):
    """The largest request that fits (every scratch region at its largest offset) equals the handle path
    exactly, twice in a row; one more shot is refused before any work."""
    import torch
    n = 22
    shots = _max_shots(n)
    st = qsim.State(n, 0)
    st.set_basis(0)
    st.run(W.brickwork(n, 2, seed=5))
    out = torch.zeros(shots + 1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    L = qsim.lib()
    for seed in (31, 32):
        rc = L.qsim_sample_noalloc(ctypes.c_void_p(st.tensor.data_ptr()), n, 0, seed, shots,
                                   ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, L.qsim_last_error()
        torch.cuda.synchronize()
        got = out[:shots].cpu().numpy().view(np.uint64)
        assert np.array_equal(got, st.sample(seed, shots))
    rc = L.qsim_sample_noalloc(ctypes.c_void_p(st.tensor.data_ptr()), n, 0, 33, shots + 32,
                               ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert rc == 1 and b"scratch" in L.qsim_last_error()


def test_noalloc_rejects_requests_beyond_the_scratch(qsim):
    import torch
    L = qsim.lib()
    st = qsim.State(10, 0)
    st.set_basis(3)
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    rc = L.qsim_sample_noalloc(ctypes.c_void_p(st.tensor.data_ptr()), 10, 0, 1, 2_000_000,
                               ctypes.c_void_p(out.data_ptr()), None)
    assert rc == 1
    assert b"scratch" in L.qsim_last_error()
    assert L.qsim_sample_noalloc(None, 10, 0, 1, 4, ctypes.c_void_p(out.data_ptr()), None) == 1
    # so many shots that 8 * shots would wrap around 64 bits: refused before any size arithmetic
    assert L.qsim_sample_noalloc(ctypes.c_void_p(st.tensor.data_ptr()), 10, 0, 1, 1 << 61,
                                 ctypes.c_void_p(out.data_ptr()), None) == 1
    # from 32 qubits on the segment sums alone fill the scratch (checked before the state is touched)
    assert L.qsim_sample_noalloc(ctypes.c_void_p(st.tensor.data_ptr()), 32, 0, 1, 1,
                                 ctypes.c_void_p(out.data_ptr()), None) == 1
    # a state that is not 256-byte aligned, an output that is not 8-byte aligned
    assert L.qsim_sample_noalloc(ctypes.c_void_p(st.tensor.data_ptr() + 8), 9, 0, 1, 4,
                                 ctypes.c_void_p(out.data_ptr()), None) == 1
    assert b"aligned" in L.qsim_last_error()
    assert L.qsim_sample_noalloc(ctypes.c_void_p(st.tensor.data_ptr()), 10, 0, 1, 2,
                                 ctypes.c_void_p(out.data_ptr() + 4), None) == 1
    torch.cuda.synchronize()
