"""Host-side checks of the C ABI (no GPU): the library builds, loads, exports every declared entry point,
and its GPU-free entry points validate arguments."""
import ctypes
import os
import re

import pytest

from paper_2511_14664_gb300 import qsim

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "qsim.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(qsim_\w+)\s*\(", text, flags=re.M)))


def test_library_exports_every_declared_symbol():
    L = qsim.lib()
    names = declared_functions()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_covers_header():
    assert set(declared_functions()) <= set(qsim.SIGNATURES)


def test_abi_version():
    assert qsim.lib().qsim_abi_version() == 2


def test_state_bytes_matches_paper_memory_formula():
    # Sec. 1: at 32-bit floating point the state takes 2^(n-27) GiB (complex64 = 8 bytes per amplitude)
    from helpers import load_golden
    for n, gib in load_golden()["paper_facts"]["fp32_state_gib"]:
        assert qsim.state_bytes(n, qsim.C64) == gib * 2**30
    assert qsim.state_bytes(14, qsim.C128) == 16 * 2**14


def test_state_bytes_rejects_bad_arguments():
    for n, dt in [(0, 0), (37, 0), (10, 2)]:
        with pytest.raises(qsim.QsimError) as e:
            qsim.state_bytes(n, dt)
        assert e.value.code == 1
    assert qsim.lib().qsim_state_bytes(10, 0, None) == 1


def test_create_rejects_bad_arguments_without_touching_the_gpu():
    L = qsim.lib()
    h = ctypes.c_void_p()
    assert L.qsim_create(0, 0, None, 0, None, ctypes.byref(h)) == 1
    assert L.qsim_create(10, 7, None, 0, None, ctypes.byref(h)) == 1
    # caller buffer too small
    assert L.qsim_create(10, 0, ctypes.c_void_p(256), 100, None, ctypes.byref(h)) == 2
    # misaligned caller buffer
    assert L.qsim_create(4, 0, ctypes.c_void_p(8), 1 << 20, None, ctypes.byref(h)) == 1
    assert b"aligned" in L.qsim_last_error()
    assert L.qsim_create(4, 0, None, 0, None, None) == 1


def test_null_handles_are_rejected():
    L = qsim.lib()
    assert L.qsim_set_basis(None, 0) == 1
    assert L.qsim_norm(None, None) == 1
    assert L.qsim_destroy(None) == 0
    assert L.qsim_plan_destroy(None) == 0


def test_circuit_marshalling_matches_the_gate_struct():
    """The binding packs a gate list with array operations into records laid out as qsim_gate; every field
    and every matrix pointer must read back as the gate it came from (mixed widths, controls, diagonals)."""
    import ctypes
    import numpy as np
    import workloads as W
    from paper_2511_14664_gb300 import qsim
    assert qsim._GATE_NP.itemsize == ctypes.sizeof(qsim.Gate)
    rng = np.random.default_rng(3)
    c = W.Circuit(12)
    for _ in range(300):
        c.append(W.random_gate(12, rng, kmax=3, cmax=2, diag_prob=0.3))
    a = qsim.CircuitArgs(c)
    assert a.c.n == 12 and a.c.num_gates == len(c)
    for i, g in enumerate(c.gates):
        r = a.gates[i]
        assert r.k == len(g.targets) and r.nc == len(g.controls)
        assert list(r.targets[:r.k]) == list(g.targets) and list(r.controls[:r.nc]) == list(g.controls)
        m = np.ctypeslib.as_array(r.matrix, shape=(2 << (2 * r.k),)).view(np.complex128)
        assert np.array_equal(m.reshape(g.matrix.shape), g.matrix)
    empty = qsim.CircuitArgs(W.Circuit(5))
    assert empty.c.num_gates == 0
