"""Checkpoint and resume through rfa_get_state / rfa_set_state: a run that is
saved, restored into a fresh grid and continued ends in the same state, bit
for bit, as the uninterrupted run (one step per launch and blocked), and a
blob from a grid of another shape or precision is refused."""
import numpy as np
import pytest

import paper_1907_05709_b300 as rfa
import phantoms as ph

pytestmark = pytest.mark.gpu


def _state(g):
    return [g.field(f) for f in (rfa.FIELD_THETA, rfa.FIELD_THETA_LO, rfa.FIELD_LATCH, rfa.FIELD_OMEGA)]


@pytest.mark.parametrize("sched", [None, (2, 0)])
def test_resume_equals_uninterrupted_run(sched):
    case = ph.random_small_case(31, 45, 38, 27, kind=ph.UMBRELLA, power=6.0)
    n1, n2 = 137, 260                                 # the second part crosses a damage fold
    a = rfa.Grid.from_case(case)
    if sched:
        a.set_schedule(*sched)
    a.step(n1)
    blob = rfa.rfa_get_state(a.handle)
    a.step(n2)
    want = _state(a)
    b = rfa.Grid.from_case(case)
    if sched:
        b.set_schedule(*sched)
    rfa.rfa_set_state(b.handle, blob)
    assert b.steps_done == n1
    b.step(n2)
    got = _state(b)
    for x, y in zip(want, got):
        assert np.array_equal(x, y)
    assert b.steps_done == n1 + n2
    a.close()
    b.close()


def test_blob_from_another_grid_is_refused():
    case = ph.random_small_case(32, 30, 20, 10)
    g = rfa.Grid.from_case(case)
    g.step(5)
    blob = rfa.rfa_get_state(g.handle)
    other = ph.random_small_case(32, 31, 20, 10)
    h = rfa.Grid.from_case(other)
    with pytest.raises(rfa.RfaError) as e:
        rfa.rfa_set_state(h.handle, blob)
    assert e.value.status == 1                         # RFA_E_INVALID
    f64 = rfa.Grid.from_case(case, state_prec=rfa.STATE_F64)
    with pytest.raises(rfa.RfaError):
        rfa.rfa_set_state(f64.handle, blob)
    for x in (g, h, f64):
        x.close()


def test_blob_with_counters_out_of_range_is_refused():
    """A blob whose step counters are corrupt (negative, or a damage-carry count
    at or beyond the fold interval) is refused: restoring it would postpone the
    FP64 fold of the FP32 damage carry without bound."""
    case = ph.random_small_case(33, 30, 20, 10)
    g = rfa.Grid.from_case(case)
    g.step(7)
    blob = bytearray(rfa.rfa_get_state(g.handle))
    steps, carry = np.frombuffer(bytes(blob[24:40]), np.int64)
    assert steps == 7 and 0 <= carry < 256
    for s_, c_ in ((7, 256), (7, 1 << 40), (7, -1), (-3, 0), (5, 6)):
        bad = bytearray(blob)
        bad[24:40] = np.array([s_, c_], np.int64).tobytes()
        with pytest.raises(rfa.RfaError) as e:
            rfa.rfa_set_state(g.handle, bytes(bad))
        assert e.value.status == 1
    rfa.rfa_set_state(g.handle, bytes(blob))          # the intact blob still restores
    assert g.steps_done == 7
    g.close()
