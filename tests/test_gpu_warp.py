"""Breathing-motion resampling (rfa_warp_temperature, Eq. breathing) on the GPU
against the FP64 oracle, on the same seeded case and motion field.

Tolerance: FP64 state 1e-9 K; compensated FP32 state 1e-3 K (the state's own
bound) + 2e-4 K for the FP32 interpolation of values up to a few hundred K."""
import numpy as np
import pytest

import oracle
import paper_1907_05709_b300 as rfa
import phantoms as ph
from tests.parity_util import run_oracle

pytestmark = pytest.mark.gpu


def _warp(g, case, u, as_f64=True):
    import torch
    ud = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    out = torch.empty((case.nz, case.ny, case.nx), dtype=torch.float64 if as_f64 else torch.float32,
                      device="cuda")
    rfa.rfa_warp_temperature(g.handle, ud, out, as_f64)
    g.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("sp,tol", [(rfa.STATE_F64, 1e-9), (rfa.STATE_F32C, 1.2e-3)])
def test_warp_matches_oracle(sp, tol):
    case = ph.random_small_case(50, 41, 34, 29, kind=ph.UMBRELLA, power=6.0)
    n = 150
    orc = run_oracle(case, rfa.PARAM_BF16, n)
    g = rfa.Grid.from_case(case, state_prec=sp)
    g.step(n)
    for t in (0.7, 2.0):
        u = ph.breathing_field(case, t, seed=3)
        expect = oracle.warp_temperature(orc["theta"], u, case.h, case.T_a_C)
        got = _warp(g, case, u)
        assert np.max(np.abs(got - expect)) <= tol
        got32 = _warp(g, case, u, as_f64=False)
        assert np.max(np.abs(got32 - expect)) <= tol + 1e-4
    g.close()


def test_zero_field_is_the_temperature_and_nan_is_clamped():
    case = ph.random_small_case(51, 33, 17, 9, kind=ph.STRAIGHT, power=4.0)
    g = rfa.Grid.from_case(case)
    g.step(40)
    T = g.temperature(as_f64=True)
    u = np.zeros((3, case.nz, case.ny, case.nx), np.float32)
    assert np.array_equal(_warp(g, case, u), T)
    u[:] = np.nan
    got = _warp(g, case, u)
    assert np.all(got == T[0, 0, 0])
    g.close()
