"""Failure detection without faulting the GPU: argument checks, the stability
check, non-finite states and bounded device-side waits all surface as status
codes, and the context stays usable afterwards."""
import numpy as np
import pytest

import paper_1907_05709_b300 as rfa
import phantoms as ph

pytestmark = pytest.mark.gpu


def _small():
    return ph.random_small_case(8, 24, 20, 18, power=4.0)


def test_unstable_time_step_rejected():
    case = _small()
    g = rfa.Grid(case.nx, case.ny, case.nz, case.h, 5.0)   # a = kappa dt / h^2 ~ 0.7 > 1/6
    with pytest.raises(rfa.RfaError) as e:
        g.set_tissue(case.labels, case.table)
    assert e.value.status == 4 and "reduce dt" in str(e.value)
    g.close()


def test_bad_label_and_order_errors():
    case = _small()
    g = rfa.Grid(case.nx, case.ny, case.nz, case.h, case.dt)
    with pytest.raises(rfa.RfaError) as e:
        g.place_needle(case.needle)            # before tissue
    assert e.value.status == 5
    lab = case.labels.copy()
    lab[3, 3, 3] = 9
    with pytest.raises(rfa.RfaError) as e:
        g.set_tissue(lab, case.table)
    assert e.value.status == 1
    g.set_tissue(case.labels, case.table)       # recovers
    g.place_needle(case.needle)
    g.step(5)
    g.synchronize()
    g.close()


def test_nonfinite_state_reported():
    case = _small()
    g = rfa.Grid.from_case(case)
    g.step(3)
    blob = bytearray(rfa.rfa_get_state(g.handle))
    # header is 40 bytes, then theta hi (float32, padded rows of 24 voxels)
    off = 40 + 4 * (5 * 20 * 24 + 7 * 24 + 9)
    blob[off:off + 4] = np.array([np.nan], np.float32).tobytes()
    rfa.rfa_set_state(g.handle, bytes(blob))
    g.step(2)
    with pytest.raises(rfa.RfaError) as e:
        g.synchronize()
    assert e.value.status == 6
    g.close()
    # a fresh grid on the same context works
    g2 = rfa.Grid.from_case(case)
    g2.step(4)
    g2.synchronize()
    g2.close()


def test_bounded_wait_times_out_and_context_survives():
    with pytest.raises(rfa.RfaError) as e:
        rfa.rfa_selftest_wait_timeout(2_000_000)   # ~1 ms of SM clocks
    assert e.value.status == 7
    case = _small()
    g = rfa.Grid.from_case(case)
    g.step(6)
    g.synchronize()
    assert np.all(np.isfinite(g.temperature()))
    g.close()


def _restore_limits():
    rfa.rfa_set_wait_limits(rfa.WAIT_LIMIT_DEFAULT, rfa.WAIT_LIMIT_DEFAULT)


def test_tma_wait_of_the_blocked_step_runs_out_and_the_grid_recovers():
    """The blocked step's own mbarrier waits with a 1-cycle limit: a wait that
    finds its TMA copy not yet landed gives up, its CTA waits (with the full
    limit) for its copies in flight and leaves, and the grid reports
    RFA_E_TIMEOUT.  The grid is large enough for a full wave of CTAs whose copies
    compete for L2 and HBM, over 20 launches, so some wait finds its copy in
    flight.  With the limits restored, set-up and stepping give the same bits
    as a grid that never timed out."""
    case = ph.random_small_case(9, 200, 160, 120, kind=ph.UMBRELLA, power=6.0)
    ref = rfa.Grid.from_case(case)
    ref.set_schedule(2, 0)
    ref.step(40)
    want = ref.temperature()
    ref.close()
    g = rfa.Grid.from_case(case)
    g.set_schedule(2, 0)
    try:
        rfa.rfa_set_wait_limits(1, rfa.WAIT_LIMIT_DEFAULT)
        g.step(40)
        with pytest.raises(rfa.RfaError) as e:
            g.synchronize()
        assert e.value.status == 7 and "mbarrier" in str(e.value)
    finally:
        _restore_limits()
    g.set_tissue(case.labels, case.table)   # clears the status, state from the labels
    g.step(40)
    g.synchronize()
    assert np.array_equal(g.temperature(), want)
    g.close()


def test_grid_barrier_of_the_batch_runs_out_and_the_batch_recovers():
    """The batch's grid barrier between time blocks with a 1-cycle limit: CTAs
    that arrive before the others give up, the launch reports RFA_E_TIMEOUT on
    the first member, naming the grid barrier.  With the limits restored the
    members, set up again, step to the same bits as stepped alone."""
    cases = [ph.random_small_case(40 + k, 64 + 8 * k, 48, 40, kind=ph.UMBRELLA, power=5.0) for k in range(6)]
    grids = [rfa.Grid.from_case(c) for c in cases]
    b = rfa.rfa_batch_create([g.handle for g in grids])
    try:
        rfa.rfa_set_wait_limits(rfa.WAIT_LIMIT_DEFAULT, 1)
        rfa.rfa_batch_step(b, 8)
        with pytest.raises(rfa.RfaError) as e:
            grids[0].synchronize()
        assert e.value.status == 7 and "grid barrier" in str(e.value)
    finally:
        _restore_limits()
    for g, c in zip(grids, cases):
        g.set_tissue(c.labels, c.table)
    rfa.rfa_batch_step(b, 8)
    grids[0].synchronize()
    got = [g.temperature() for g in grids]
    rfa.rfa_batch_destroy(b)
    for g, c, t in zip(grids, cases, got):
        alone = rfa.Grid.from_case(c)
        alone.set_schedule(2, 0)
        alone.step(8)
        assert np.array_equal(alone.temperature(), t)
        alone.close()
        g.close()


def test_wait_limits_are_checked():
    for bad in ((0, 1 << 32), (1, 0), ((1 << 32) + 1, 5)):
        with pytest.raises(rfa.RfaError) as e:
            rfa.rfa_set_wait_limits(*bad)
        assert e.value.status == 1
