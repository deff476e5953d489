"""Helpers for GPU-vs-oracle parity tests: run one case through the C ABI and
through the FP64 oracle on the same seeded inputs, and compare.

Tolerances (floating point):
  - FP64 state: |T_gpu - T_oracle| <= 1e-9 K.
  - FP32 compensated state: <= 1e-3 K (the accuracy target of the path).
  - Damage integral: relative <= 0.35 * tol_T + 5e-5, from
    d ln(Omega) / dT = Ea / (R T_K^2) <= 0.33 / K at T_K >= 310 K plus the FP32
    evaluation of the exponent (log2(A dt) and Ea / (R ln 2) / T_K rounded to
    FP32, ~2e-5 relative).
  - Necrosis masks: identical except at voxels whose oracle temperature is
    within tol_T of the threshold (heating is monotone in time here, so the
    final temperature is the running maximum); Arrhenius bits identical except
    where |Omega_oracle - 1| <= 1e-2.
"""
import numpy as np

import oracle
import paper_1907_05709_b300 as rfa

PMODE = {rfa.PARAM_BF16: "bf16", rfa.PARAM_F32: "f32", rfa.PARAM_F64: "f64"}
TOL_T = {rfa.STATE_F64: 1e-9, rfa.STATE_F32C: 1e-3, rfa.STATE_F32: 1e-3}


def tol_omega(sp):
    return 1e-10 if sp == rfa.STATE_F64 else 0.35 * TOL_T[sp] + 5e-5


def run_gpu(case, sp, pp, nsteps, damage=True, schedule=None, chunks=None):
    g = rfa.Grid.from_case(case, state_prec=sp, param_prec=pp, damage=damage)
    if schedule is not None:
        g.set_schedule(*schedule)
    if chunks is None:
        chunks = [nsteps]
    for c in chunks:
        g.step(c)
    g.synchronize()
    out = dict(T=g.temperature(as_f64=True), theta=g.field(rfa.FIELD_THETA),
               latch=g.field(rfa.FIELD_LATCH), omega=g.field(rfa.FIELD_OMEGA),
               s=g.field(rfa.FIELD_S), a=g.field(rfa.FIELD_A), b=g.field(rfa.FIELD_B))
    mask, counts, vols, sv = g.necrosis()
    out.update(mask=mask, counts=counts, vols=vols, smooth=sv, steps=g.steps_done)
    g.close()
    return out


def run_oracle(case, pp, nsteps, damage=True):
    m = oracle.setup(case, PMODE[pp])
    st = oracle.initial_state(m)
    dmg = case.damage if damage else None
    if dmg is not None and not dmg.enable:
        dmg = None
    oracle.run(m, st, nsteps, damage=dmg, T_thr_C=case.damage.T_thr_C)
    mask, counts, vols, sv = oracle.necrosis(m, st, thr_C=case.damage.T_thr_C)
    return dict(model=m, T=st.theta + case.T_a_C, theta=st.theta, latch=st.latch,
                omega=st.omega, mask=mask, counts=counts, vols=vols, smooth=sv)


def compare(case, gpu, orc, sp, damage=True):
    """Assert parity; return a dict of the observed errors."""
    tol = TOL_T[sp]
    err_T = float(np.max(np.abs(gpu["T"] - orc["T"])))
    assert err_T <= tol, f"max |dT| = {err_T:.3e} K > {tol:.1e} K"
    thr = case.damage.T_thr_C
    band = np.abs(orc["T"] - thr) <= tol
    th_g = (gpu["mask"] & 1) != 0
    th_o = (orc["mask"] & 1) != 0
    diff = (th_g != th_o) & ~band
    assert not diff.any(), f"{int(diff.sum())} thermal-mask voxels differ outside the band"
    res = dict(err_T=err_T, mask_band=int(band.sum()))
    if damage and case.damage.enable:
        om_o, om_g = orc["omega"], gpu["omega"]
        rel = np.abs(om_g - om_o) / np.maximum(np.abs(om_o), 1e-300)
        err_om = float(np.max(rel))
        assert err_om <= tol_omega(sp), f"max rel dOmega = {err_om:.3e}"
        arr_band = np.abs(om_o - 1.0) <= 1e-2
        d2 = (((gpu["mask"] & 2) != 0) != ((orc["mask"] & 2) != 0)) & ~arr_band
        assert not d2.any(), f"{int(d2.sum())} Arrhenius-mask voxels differ outside the band"
        res["err_omega_rel"] = err_om
    # reductions: counts agree up to the band, smoothed volume to FP32 evaluation accuracy
    assert abs(int(gpu["counts"][0]) - int(orc["counts"][0])) <= int(band.sum())
    h3 = case.h ** 3
    assert abs(gpu["smooth"] - orc["smooth"]) <= 1e-5 * max(orc["smooth"], h3)
    return res
