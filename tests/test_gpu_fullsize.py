"""Parity at the single-needle workload's full size and launch configuration
(256^3 umbrella phantom, autotuned blocked schedule, compensated FP32 state,
BF16 coefficients, Arrhenius damage):
  - every voxel against the FP64 oracle after the first 300 of its 12000 steps;
  - the whole 12000-step run, every voxel, against the FP64 oracle on the same
    coefficients (a few minutes of CPU work on the host cores) and against the
    FP64 GPU path.
The 512^3 workload is compared on a 128^3 crop and with the FP64 GPU path in
test_gpu_precision_study.py."""
import numpy as np
import pytest

import paper_1907_05709_b300 as rfa
import phantoms as ph
from tests.parity_util import compare, run_oracle

pytestmark = pytest.mark.gpu


def _gpu_run(case, sp, nsteps, tune):
    g = rfa.Grid.from_case(case, state_prec=sp, param_prec=rfa.PARAM_BF16)
    if tune:
        rfa.rfa_autotune(g.handle, None)
    g.step(nsteps)
    g.synchronize()
    out = dict(T=g.temperature(as_f64=True), theta=g.field(rfa.FIELD_THETA),
               omega=g.field(rfa.FIELD_OMEGA), latch=g.field(rfa.FIELD_LATCH),
               schedule=rfa.rfa_get_schedule(g.handle))
    mask, counts, vols, sv = g.necrosis()
    out.update(mask=mask, counts=counts, vols=vols, smooth=sv)
    g.close()
    return out


def test_umbrella256_first_300_steps_every_voxel():
    case = ph.umbrella_case_256(seed=0)
    orc = run_oracle(case, rfa.PARAM_BF16, 300)
    gpu = _gpu_run(case, rfa.STATE_F32C, 300, tune=True)
    assert gpu["schedule"][0] >= 1
    compare(case, gpu, orc, rfa.STATE_F32C)


def test_umbrella256_12000_steps_every_voxel_against_the_oracle():
    """Eq. CUDAbioheat3d stepped 12000 times with the 60 C latch and Eq.
    eq-tissState: T within 1e-3 K, Omega within the relative tolerance, masks
    equal outside the bands, counts and the smoothed volume as in every parity
    test."""
    case = ph.umbrella_case_256(seed=0)
    gpu = _gpu_run(case, rfa.STATE_F32C, case.nsteps, tune=True)
    orc = run_oracle(case, rfa.PARAM_BF16, case.nsteps)
    res = compare(case, gpu, orc, rfa.STATE_F32C)
    assert orc["counts"][0] > 1000 and orc["counts"][1] > 1000    # the case really ablates
    print(f"256^3 x 12000 vs oracle: max|dT| = {res['err_T']:.3e} K, "
          f"max rel dOmega = {res['err_omega_rel']:.3e}, band voxels {res['mask_band']}, "
          f"schedule {gpu['schedule']}")


def test_umbrella256_12000_steps_against_fp64_gpu():
    case = ph.umbrella_case_256(seed=0)
    a = _gpu_run(case, rfa.STATE_F32C, case.nsteps, tune=True)
    b = _gpu_run(case, rfa.STATE_F64, case.nsteps, tune=False)
    err = float(np.max(np.abs(a["T"] - b["T"])))
    assert err <= 1e-3, err
    band = np.abs(b["T"] - case.damage.T_thr_C) <= 1e-3
    assert not ((((a["mask"] & 1) != 0) != ((b["mask"] & 1) != 0)) & ~band).any()
    rel = np.abs(a["omega"] - b["omega"]) / np.maximum(b["omega"], 1e-300)
    assert rel.max() <= 0.35e-3 + 5e-5
    abad = (((a["mask"] & 2) != 0) != ((b["mask"] & 2) != 0)) & ~(np.abs(b["omega"] - 1) <= 1e-2)
    assert not abad.any()
    print(f"256^3 x 12000: max|dT| = {err:.3e} K, max rel dOmega = {rel.max():.3e}, "
          f"necrosis thermal {int(a['counts'][0])} arrhenius {int(a['counts'][1])}, "
          f"peak T {a['T'].max():.1f} C, schedule {a['schedule']}")
