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
