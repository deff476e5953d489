"""Temporally blocked step (several steps per launch, TMA-staged tiles):
bit-identical states to the one-step kernel, and parity with the oracle."""
import numpy as np
import pytest

import paper_1907_05709_b300 as rfa
import phantoms as ph
from tests.parity_util import compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

SCHEDULES = [(2, 0), (3, 0), (2, 1)]


@pytest.mark.parametrize("sched", SCHEDULES)
@pytest.mark.parametrize("dims", [(33, 17, 9), (130, 67, 41), (64, 64, 64), (200, 30, 70), (5, 200, 13)])
def test_blocked_equals_one_step(sched, dims):
    nx, ny, nz = dims
    case = ph.random_small_case(7 + nx, nx, ny, nz, kind=ph.UMBRELLA, power=5.0)
    n = 4 * sched[0] + 1                       # full blocks plus a one-step remainder
    a = run_gpu(case, rfa.STATE_F32C, rfa.PARAM_BF16, n)
    b = run_gpu(case, rfa.STATE_F32C, rfa.PARAM_BF16, n, schedule=sched)
    assert np.array_equal(a["theta"], b["theta"])
    assert np.array_equal(a["T"], b["T"])
    assert np.array_equal(a["latch"], b["latch"])
    # the blocked kernel sums a block's increments in FP32 before adding them to the
    # FP32 carry of the FP64 integral; both carries hold <= 256 steps (~256 * 2^-24)
    rel = np.abs(a["omega"] - b["omega"]) / np.maximum(a["omega"], 1e-300)
    assert rel.max() <= 2e-5


@pytest.mark.parametrize("sched", SCHEDULES)
def test_blocked_parity_with_oracle(sched):
    case = ph.random_small_case(21, 71, 45, 38, kind=ph.UMBRELLA, power=6.0)
    n = 301
    orc = run_oracle(case, rfa.PARAM_BF16, n)
    gpu = run_gpu(case, rfa.STATE_F32C, rfa.PARAM_BF16, n, schedule=sched)
    compare(case, gpu, orc, rfa.STATE_F32C)


def test_blocked_homogeneous_64_2000_steps():
    case = ph.homogeneous_case(damage=ph.Damage(enable=1))
    orc = run_oracle(case, rfa.PARAM_BF16, 2000)
    gpu = run_gpu(case, rfa.STATE_F32C, rfa.PARAM_BF16, 2000, schedule=(3, 0))
    res = compare(case, gpu, orc, rfa.STATE_F32C)
    assert res["err_T"] < 1e-4


def test_schedule_rejected_where_unsupported():
    case = ph.random_small_case(3, 20, 20, 20)
    g = rfa.Grid.from_case(case, state_prec=rfa.STATE_F64, param_prec=rfa.PARAM_BF16)
    with pytest.raises(rfa.RfaError) as e:
        g.set_schedule(2, 0)
    assert e.value.status == 8
    with pytest.raises(rfa.RfaError) as e:
        g.set_schedule(9, 0)
    assert e.value.status == 1
    g.close()
    # tile variant 1 runs depth 2 only; there is no variant 2
    g = rfa.Grid.from_case(case)
    for bad in ((3, 1), (2, 2)):
        with pytest.raises(rfa.RfaError) as e:
            g.set_schedule(*bad)
        assert e.value.status == 8
    g.close()
    # insulated faces: the blocked kernel needs Dirichlet faces (one step per launch)
    ins = ph.random_small_case(3, 20, 20, 20, face_bc=ph.INSULATED)
    g = rfa.Grid.from_case(ins)
    with pytest.raises(rfa.RfaError) as e:
        g.set_schedule(2, 0)
    assert e.value.status == 8
    rfa.rfa_autotune(g.handle, None)
    assert rfa.rfa_get_schedule(g.handle) == (1, 0)
    with pytest.raises(rfa.RfaError) as e:
        rfa.rfa_batch_create([g.handle])
    assert e.value.status == 8
    g.close()


def test_autotune_picks_a_schedule_and_keeps_state(tmp_path):
    case = ph.random_small_case(5, 96, 96, 96, kind=ph.UMBRELLA, power=5.0)
    g = rfa.Grid.from_case(case)
    g.step(7)
    before = g.field(rfa.FIELD_THETA)
    om_before = g.field(rfa.FIELD_OMEGA)
    cache = str(tmp_path / "tune.json")
    rfa.rfa_autotune(g.handle, cache)
    d, v = rfa.rfa_get_schedule(g.handle)
    assert d >= 1
    assert np.array_equal(g.field(rfa.FIELD_THETA), before)
    assert np.array_equal(g.field(rfa.FIELD_OMEGA), om_before)
    assert g.steps_done == 7
    g.close()
    # a second grid of the same shape reads the cached choice
    g2 = rfa.Grid.from_case(case)
    rfa.rfa_autotune(g2.handle, cache)
    assert rfa.rfa_get_schedule(g2.handle) == (d, v)
    g2.close()
