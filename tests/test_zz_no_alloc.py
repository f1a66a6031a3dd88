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
