"""The device error word path, made to fail on the host (no kernel's wait is made to expire on the GPU).

Every bounded wait in the tensor-core kernels records an expiry in the handle's device error word and
returns; the host turns a set word into QSIM_ETIMEOUT at the next synchronising call and clears it. Here the
word is written from the host with qsim_inject_device_error, exactly as an expired wait would leave it, and
the test checks the status, the message and that the handle still simulates correctly afterwards.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qsim(gpu_lib):
    from paper_2511_14664_gb300 import qsim as q
    return q


def test_injected_error_word_becomes_etimeout_and_handle_recovers(qsim):
    L = qsim.lib()
    n = 14
    c = W.brickwork(n, 6, seed=17)
    st = qsim.State(n, qsim.C64)
    st.set_basis(0)
    st.run(c, mode=qsim.RUN_FUSED, max_fused=6, precision=qsim.PREC_TF32X3)
    assert L.qsim_synchronize(st.h) == 0
    assert L.qsim_inject_device_error(st.h, 1) == 0
    assert L.qsim_synchronize(st.h) == 4                     # QSIM_ETIMEOUT
    assert b"bounded wait" in L.qsim_last_error()
    assert L.qsim_synchronize(st.h) == 0                     # reported once, then cleared
    # a readout reports it too
    assert L.qsim_inject_device_error(st.h, 1) == 0
    out = ctypes.c_double()
    assert L.qsim_norm(st.h, ctypes.byref(out)) == 4
    assert L.qsim_inject_device_error(st.h, 0) == 1          # zero is not an error code
    # the handle still runs a circuit correctly (tensor-core plan and the per-gate path)
    ref = oracle.run(c)
    for kw in (dict(mode=qsim.RUN_FUSED, max_fused=6, precision=qsim.PREC_TF32X3), dict(mode=qsim.RUN_PLAIN)):
        st.set_basis(0)
        st.run(c, **kw)
        st.synchronize()
        psi = st.get_state().astype(np.complex128)
        assert float(np.max(np.abs(psi - ref))) <= 1e-5
        assert oracle.infidelity(np.ascontiguousarray(psi), ref, n) <= 1e-9
    assert L.qsim_inject_device_error(None, 1) == 1
