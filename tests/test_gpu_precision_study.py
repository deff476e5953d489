"""Precision study on the large workload: 512^3, h = 0.25 mm, 8 vessels,
9-tine umbrella at 40 W, dt = 0.02 s, 5000 steps, Arrhenius damage.

  - arithmetic error: compensated FP32 state vs the FP64 GPU state on the same
    coefficients (BF16, then FP32), held to 1e-3 K;
  - model error of BF16 coefficient fields: FP64 state with BF16 vs FP32
    coefficients (reported, not a parity bound);
  - a 128^3 crop around the needle (Dirichlet crop faces) against the FP64
    oracle, every voxel.
Results are printed (run with -s)."""
import numpy as np
import pytest

import paper_1907_05709_b300 as rfa
import phantoms as ph
from tests.parity_util import compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def _run(case, sp, pp, tune=False):
    g = rfa.Grid.from_case(case, state_prec=sp, param_prec=pp)
    if tune:
        rfa.rfa_autotune(g.handle, None)
    g.step(case.nsteps)
    g.synchronize()
    T = g.temperature(as_f64=True)
    om = g.field(rfa.FIELD_OMEGA)
    _, counts, _, _ = g.necrosis(want_mask=False)
    g.close()
    return T, om, counts


def test_large512_precision_study():
    case = ph.large_case_512(seed=0)
    T32b, O32b, c32b = _run(case, rfa.STATE_F32C, rfa.PARAM_BF16, tune=True)
    T64b, O64b, c64b = _run(case, rfa.STATE_F64, rfa.PARAM_BF16)
    e_bf16 = float(np.max(np.abs(T32b - T64b)))
    del T32b
    T32f, _, c32f = _run(case, rfa.STATE_F32C, rfa.PARAM_F32)
    T64f, O64f, c64f = _run(case, rfa.STATE_F64, rfa.PARAM_F32)
    e_f32 = float(np.max(np.abs(T32f - T64f)))
    model = float(np.max(np.abs(T64b - T64f)))
    om_model = float(np.max(np.abs(O64b - O64f) / np.maximum(O64f, 1e-300)))
    print(f"\n512^3 x 5000: |FP32C-FP64| bf16 coeffs {e_bf16:.3e} K, fp32 coeffs {e_f32:.3e} K; "
          f"model error bf16 vs fp32 coefficients {model:.3e} K (Omega rel {om_model:.3e}); "
          f"necrosis thermal/Arrhenius bf16 {tuple(int(v) for v in c64b)} fp32 {tuple(int(v) for v in c64f)}; "
          f"peak T {T64f.max():.1f} C")
    assert e_bf16 <= 1e-3 and e_f32 <= 1e-3


def test_large512_crop128_against_oracle():
    full = ph.large_case_512(seed=0)
    c = [int(round(t / full.h)) for t in full.needle.tip]   # tip voxel (x, y, z)
    lo = [min(max(ci - 64, 0), 512 - 128) for ci in c]
    crop = ph.Case("crop128", 128, 128, 128, full.h, full.dt, full.nsteps,
                   np.ascontiguousarray(full.labels[lo[2]:lo[2] + 128, lo[1]:lo[1] + 128, lo[0]:lo[0] + 128]),
                   full.table, ph.Needle(**{**full.needle.__dict__,
                                            "tip": tuple(full.needle.tip[d] - lo[d] * full.h for d in range(3))}),
                   full.damage)
    orc = run_oracle(crop, rfa.PARAM_BF16, crop.nsteps)
    gpu = run_gpu(crop, rfa.STATE_F32C, rfa.PARAM_BF16, crop.nsteps, schedule=(2, 0))
    res = compare(crop, gpu, orc, rfa.STATE_F32C)
    print(f"\n128^3 crop x 5000 vs oracle: {res}")
