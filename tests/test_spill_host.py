"""Out-of-core segmentation (host only, no GPU): the segments an out-of-core run streams the state through.

A state cut by its top index bits needs the pieces that differ in a global bit for any gate on it (Sec. 2.1);
the segmenter groups gates so that each segment touches at most `global_slots` of those bits. These tests
follow the segments on the oracle and check the invariants that make the streamed run equal to the circuit.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_2511_14664_gb300 import qsim


def _masks(c):
    return [sum(1 << q for q in tuple(g.targets) + tuple(g.controls)) for g in c.gates]


def _check_segments(c, window, slots):
    seg, used = qsim.spill_segments(c, window, slots)
    n = c.n
    h = slots or min(4, window - 12)
    L = n if window >= n else window - h
    top = ((1 << n) - 1) & ~((1 << L) - 1)
    m = _masks(c)
    assert len(seg) == len(c.gates) and (len(c.gates) == 0 or seg.max() == len(used) - 1)
    for i, gm in enumerate(m):
        assert gm & top & ~used[seg[i]] == 0          # every global qubit of a gate is in its segment's window
    for u in used:
        assert bin(u & top).count("1") <= (h if window < n else 0)
    for i in range(len(m)):                            # gates sharing a qubit keep their order
        for j in range(i + 1, len(m)):
            if m[i] & m[j]:
                assert seg[i] <= seg[j], (i, j)
    return seg, used


@pytest.mark.parametrize("n,window,slots", [(20, 16, 0), (20, 16, 2), (24, 18, 3), (22, 21, 2)])
def test_segments_brickwork(n, window, slots):
    c = W.brickwork(n, 6, seed=n)
    seg, used = _check_segments(c, window, slots)
    assert 1 < len(used) < len(c.gates)


def test_segments_follow_the_circuit_on_the_oracle():
    """Applying the gates segment by segment (input order inside a segment) gives the circuit's state."""
    n = 16
    rng = np.random.default_rng(3)
    c = W.Circuit(n)
    for _ in range(150):
        c.append(W.random_gate(n, rng, kmax=2, cmax=1, diag_prob=0.3))
    seg, used = _check_segments(c, 14, 2)
    order = sorted(range(len(c.gates)), key=lambda i: (seg[i], i))
    psi0 = oracle.basis(n, 0)
    ref = oracle.run(c, psi=psi0.copy())
    psi = psi0.copy()
    for i in order:
        g = c.gates[i]
        oracle.apply_gate(psi, n, g.targets, g.controls, g.matrix)
    assert np.max(np.abs(psi - ref)) <= 1e-12


def test_state_that_fits_one_window_is_one_segment():
    c = W.brickwork(14, 5, seed=1)
    seg, used = qsim.spill_segments(c, 20, 0)
    assert len(used) == 1 and np.all(seg == 0)


def test_gate_with_too_many_global_qubits_is_refused():
    c = W.Circuit(20)
    c.append(W.Gate((17, 18), (19,), np.eye(4), "wide"))   # three qubits among the top 6 index bits (L = 14)
    with pytest.raises(qsim.QsimError) as e:
        qsim.spill_segments(c, 16, 2)
    assert e.value.code == 5
    seg, used = qsim.spill_segments(c, 16, 3)
    assert len(used) == 1


def test_bad_geometry_is_refused():
    c = W.brickwork(20, 2, seed=1)
    for window, slots in [(13, 0), (16, 9), (16, 7)]:
        with pytest.raises(qsim.QsimError):
            qsim.spill_segments(c, window, slots)
