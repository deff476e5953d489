"""Pins of the oracle's tissue-state perfusion coupling: the blood-perfusion
term of Eq. 2675-eq1_Linte weighted by alpha(t) (Eq. eq-tissState), read as
alpha = 1 / max(1, Omega) -- the inverse Arrhenius integral, capped at 1 where
the integral is below 1 (the paper's singularity near t = 0)."""
import math

import numpy as np

import oracle
import phantoms as ph


def test_uniform_field_follows_the_scalar_recurrence():
    """A uniform insulated box without source: every voxel follows
    theta' = theta (1 - b alpha), Omega' = Omega + dt A exp(-Ea / (R T'_K))."""
    t = ph.Tissue(w_b=2e-2)
    n = 4
    labels = np.zeros((n, n, n), np.uint8)
    dmg = ph.Damage(enable=1)
    case = ph.Case("uniform", n, n, n, 1e-3, 0.5, 0, labels, [t], ph.Needle(power=0.0), dmg,
                   face_bc=ph.INSULATED, perfusion="tissue_state")
    m = oracle.setup(case, "f64")
    st = oracle.initial_state(m)
    th0 = 45.0
    st.theta[:] = th0
    N = 400
    oracle.run(m, st, N, damage=dmg)
    b = t.w_b * t.rho_b * t.c_b / (t.rho * t.c) * case.dt
    th, om = th0, 0.0
    for _ in range(N):
        th = th + (-(b / max(1.0, om)) * th)
        om = om + case.dt * dmg.A * math.exp(-dmg.Ea / (dmg.R * (th + 37.0 + 273.15)))
    assert om > 1.0                               # the coupling is active at the end
    assert np.allclose(st.theta, th, rtol=1e-12, atol=0)
    assert np.allclose(st.omega, om, rtol=1e-12, atol=0)


def test_no_effect_below_the_damage_threshold_and_hotter_above():
    case = ph.random_small_case(30, 21, 18, 17, power=1.0)
    base = oracle.setup(case, "f64")
    case.perfusion = "tissue_state"
    cpl = oracle.setup(case, "f64")
    a, b = oracle.initial_state(base), oracle.initial_state(cpl)
    oracle.run(base, a, 40, damage=case.damage)
    oracle.run(cpl, b, 40, damage=case.damage)
    assert a.omega.max() < 1.0
    assert np.array_equal(a.theta, b.theta)
    # a hot needle: where Omega > 1 perfusion weakens, so the field is never cooler
    case2 = ph.random_small_case(31, 21, 18, 17, power=12.0)
    base2 = oracle.setup(case2, "f64")
    case2.perfusion = "tissue_state"
    cpl2 = oracle.setup(case2, "f64")
    a, b = oracle.initial_state(base2), oracle.initial_state(cpl2)
    oracle.run(base2, a, 400, damage=case2.damage)
    oracle.run(cpl2, b, 400, damage=case2.damage)
    assert b.omega.max() > 1.0
    assert np.all(b.theta >= a.theta - 1e-12)
    assert np.max(b.theta - a.theta) > 1e-3
