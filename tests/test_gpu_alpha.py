"""Perfusion weighted by the tissue state (rfa_set_perfusion_coupling,
alpha = 1/max(1, Omega)) on the GPU against the oracle, with either conduction
form; identical to the uncoupled blocked path while Omega stays below 1."""
import numpy as np
import pytest

import paper_1907_05709_b300 as rfa
import phantoms as ph
from tests.parity_util import compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cond", ["centre", "harmonic"])
@pytest.mark.parametrize("sp", [rfa.STATE_F64, rfa.STATE_F32C])
def test_coupled_perfusion_matches_oracle(cond, sp):
    case = ph.random_small_case(90, 33, 29, 27, kind=ph.UMBRELLA, power=10.0)
    case.perfusion = "tissue_state"
    case.conduction = cond
    n = 400
    orc = run_oracle(case, rfa.PARAM_BF16, n)
    assert orc["omega"].max() > 1.0               # the coupling is active
    gpu = run_gpu(case, sp, rfa.PARAM_BF16, n)
    compare(case, gpu, orc, sp)


def test_no_effect_while_omega_below_one():
    case = ph.random_small_case(91, 40, 31, 22, kind=ph.STRAIGHT, power=1.0)
    a = run_gpu(case, rfa.STATE_F32C, rfa.PARAM_BF16, 30)
    case.perfusion = "tissue_state"
    b = run_gpu(case, rfa.STATE_F32C, rfa.PARAM_BF16, 30)
    assert a["omega"].max() < 1.0
    assert np.array_equal(a["theta"], b["theta"])
