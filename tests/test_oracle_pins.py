"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the exact
discrete decay of a sine mode, the perfusion decay, energy balance, the
steady perfused point source and the 1D erfc solution of a held boundary
(both with refinement), the paper's monotonicity property, the constant-
temperature Arrhenius integral, the paper's printed liver constants, and a
dense brute-force step matrix.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.fft

import oracle
import phantoms as ph
from tests import brute

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _case(nx, ny, nz, table, needle, face_bc=ph.DIRICHLET, h=1e-3, dt=0.05, labels=None,
          damage=None):
    lab = np.zeros((nz, ny, nx), np.uint8) if labels is None else labels
    return ph.Case("t", nx, ny, nz, h, dt, 0, lab, table, needle,
                   damage if damage is not None else ph.Damage(enable=0), face_bc=face_bc)


def _no_source():
    return ph.Needle(kind=ph.STRAIGHT, power=0.0)


# ------------------------------------------------------------------ rounding
def test_bf16_rounding_definition():
    # ties go to the even 8-bit significand
    assert oracle.round_bf16(1.0 + 2.0 ** -8) == 1.0
    assert oracle.round_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert oracle.round_bf16(1.0 + 2.0 ** -8 + 2.0 ** -30) == 1.0 + 2.0 ** -7
    rng = np.random.default_rng(1)
    for x in rng.uniform(1e-6, 1.0, 500) * rng.choice([-1, 1], 500):
        r = oracle.round_bf16(float(x))
        e = math.frexp(r)[1]
        # 8 significant bits and within half an ulp of x
        assert float(r) * 2.0 ** (8 - e) == round(float(r) * 2.0 ** (8 - e))
        assert abs(r - x) <= 2.0 ** (math.frexp(x)[1] - 9) * (1 + 1e-12)


# ------------------------------------------------------------------ stencil
def test_sine_mode_exact_discrete_decay():
    nx, ny, nz = 17, 13, 11
    mx, my, mz = 2, 1, 3
    t = ph.liver()
    case = _case(nx, ny, nz, [t], _no_source(), face_bc=ph.DIRICHLET)
    m = oracle.setup(case, "f64")
    st = oracle.initial_state(m)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    th0 = (np.sin(np.pi * mx * x / (nx - 1)) * np.sin(np.pi * my * y / (ny - 1))
           * np.sin(np.pi * mz * z / (nz - 1)))
    st.theta[...] = 100.0 * th0
    # exact eigenvalue of one step: g = 1 - 4 a sum_d sin^2(pi m_d / (2 (N_d - 1))) - b
    a = t.k / (t.rho * t.c) * case.dt / case.h ** 2
    b = t.w_b * t.rho_b * t.c_b / (t.rho * t.c) * case.dt
    g = 1.0 - 4 * a * sum(math.sin(math.pi * md / (2 * (nd - 1))) ** 2
                          for md, nd in ((mx, nx), (my, ny), (mz, nz))) - b
    n = 300
    oracle.run(m, st, n)
    ref = 100.0 * th0 * g ** n
    assert np.max(np.abs(st.theta - ref)) <= 1e-12 * 100.0


def test_uniform_perfusion_decay_insulated():
    t = ph.tumor()
    case = _case(7, 6, 5, [t], _no_source(), face_bc=ph.INSULATED)
    m = oracle.setup(case, "f64")
    st = oracle.initial_state(m)
    st.theta[...] = 7.5
    b = t.w_b * t.rho_b * t.c_b / (t.rho * t.c) * case.dt
    oracle.run(m, st, 1000)
    assert np.allclose(st.theta, 7.5 * (1 - b) ** 1000, rtol=1e-12, atol=0)


def test_paper_metabolic_steady_state():
    """With the paper's printed liver constants and no source, a uniform
    insulated block approaches theta_ss = Q_m / (w_b c_b) as
    theta^n = theta_ss (1 - (1 - b)^n)."""
    g = json.load(open(os.path.join(GOLD, "paper_liver_constants.json")))
    t = ph.paper_liver()
    assert (t.Q_m, t.rho, t.c, t.k, t.w_b, t.c_b) == (
        g["Q_m_W_per_m3"], g["rho_kg_per_m3"], g["c_p_J_per_kg_K"], g["K_W_per_m_K"],
        g["w_b_kg_per_m3_s"], g["c_b_J_per_kg_K"])
    case = _case(5, 5, 5, [t], _no_source(), face_bc=ph.INSULATED, dt=0.1)
    m = oracle.setup(case, "f64")
    st = oracle.initial_state(m)
    n = 20000
    oracle.run(m, st, n)
    th_ss = g["Q_m_W_per_m3"] / (g["w_b_kg_per_m3_s"] * g["c_b_J_per_kg_K"])
    b = g["w_b_kg_per_m3_s"] * g["c_b_J_per_kg_K"] / (g["rho_kg_per_m3"] * g["c_p_J_per_kg_K"]) * 0.1
    assert np.allclose(st.theta, th_ss * (1 - (1 - b) ** n), rtol=1e-10)
    assert abs(th_ss - 0.1775) < 1e-3


@pytest.mark.parametrize("kind", [ph.STRAIGHT, ph.UMBRELLA])
def test_energy_balance_insulated_no_perfusion(kind):
    t = ph.Tissue(w_b=0.0)
    n = 20
    h = 1e-3
    c = ph.centre(n, h)
    nd = ph.Needle(kind=kind, tip=(c, c, c + 2e-3), active_len=6e-3, tine_len=5e-3,
                   n_tines=8, tine_axial=1, power=12.0)
    case = _case(n, n, n, [t], nd, face_bc=ph.INSULATED, h=h, dt=0.1)
    m = oracle.setup(case, "f64")
    st = oracle.initial_state(m)
    N = 400
    oracle.run(m, st, N)
    energy = float(np.sum(m.rhoc * h ** 3 * st.theta))
    assert abs(energy - N * 0.1 * 12.0) <= 1e-11 * N * 0.1 * 12.0


def test_source_shape_hand_picked():
    h = 1e-3
    t = ph.liver()
    tip = (3 * h, 3 * h, 5 * h)
    nd = ph.Needle(kind=ph.STRAIGHT, tip=tip, active_len=3 * h, power=5.0, r_clamp=h)
    case = _case(8, 8, 8, [t], nd, face_bc=ph.INSULATED, h=h)
    m = oracle.setup(case, "f64")
    d = m.dist
    assert d[6, 3, 3] == pytest.approx(h, rel=1e-14)          # on the axis beyond the tip
    assert d[2, 3, 3] == pytest.approx(0.0, abs=1e-18)         # proximal end of the active part
    assert d[4, 3, 4] == pytest.approx(h, rel=1e-14)           # beside the shaft
    assert d[7, 5, 5] == pytest.approx(math.sqrt(12) * h, rel=1e-14)  # nearest point = tip
    s = m.s
    # inside the clamp radius every weight is max(d, r0)^-4 = r0^-4
    assert s[3, 3, 3] == pytest.approx(s[4, 3, 4], rel=1e-14) == pytest.approx(s[6, 3, 3], rel=1e-14)
    assert s[7, 5, 5] / s[3, 3, 3] == pytest.approx(1.0 / 144.0, rel=1e-13)
    # normalisation: sum_i q_i h^3 = P
    assert float(np.sum(s * m.rhoc / case.dt) * h ** 3) == pytest.approx(5.0, rel=1e-13)

    # umbrella: tine 0 at azimuth 0 lies in the xz-plane at 60 deg off +z
    L = 4 * h
    nd = ph.Needle(kind=ph.UMBRELLA, tip=tip, tine_len=L, n_tines=4, tine_axial=1, power=5.0,
                   r_clamp=0.1 * h)
    case = _case(10, 8, 10, [t], nd, face_bc=ph.INSULATED, h=h)
    d = oracle.setup(case, "f64").dist
    assert d[7, 3, 7] == pytest.approx((4 - 2 * math.sqrt(3)) * h, rel=1e-12)  # past the tine end
    assert d[7, 3, 3] == pytest.approx(0.0, abs=1e-18)                         # on the axial tine
    # 4 ring tines without the axial one: 4-fold symmetry about the axis through
    # the tip, (x, y) -> (-y, x) around (3, 3), but no 8-fold symmetry
    nd = ph.Needle(kind=ph.UMBRELLA, tip=tip, tine_len=L, n_tines=4, tine_axial=0, power=5.0,
                   r_clamp=0.1 * h)
    case = _case(7, 7, 10, [t], nd, face_bc=ph.INSULATED, h=h)
    d = oracle.setup(case, "f64").dist
    rot = d[:, ::-1, :].transpose(0, 2, 1)          # rot[z, y, x] = d[z, 6 - x, y]
    assert np.allclose(d, rot, rtol=1e-12, atol=1e-18)
    assert d[7, 3, 6] < 0.6 * h and d[7, 6, 6] > 1.5 * h


def _dst_steady(n_int, h, t, q_centre):
    """Discrete steady state of the scheme on a Dirichlet box with a single
    source voxel, by the DST-I diagonalisation of the 7-point operator."""
    K, beta = t.k, t.w_b * t.rho_b * t.c_b
    q = np.zeros((n_int,) * 3)
    c = n_int // 2
    q[c, c, c] = q_centre
    qh = scipy.fft.dstn(q, type=1)
    k = np.arange(1, n_int + 1)
    lam1 = 4 * np.sin(np.pi * k / (2 * (n_int + 1))) ** 2 / h ** 2
    den = beta + K * (lam1[:, None, None] + lam1[None, :, None] + lam1[None, None, :])
    return scipy.fft.idstn(qh / den, type=1)


def test_steady_point_source_fixed_point_and_refinement():
    t = ph.liver()
    P = 1.0
    Lb = math.sqrt(t.k / (t.w_b * t.rho_b * t.c_b))
    half = 24e-3
    errs = []
    for h in (1e-3, 0.5e-3, 0.25e-3):
        n = int(round(2 * half / h)) + 1
        th = _dst_steady(n - 2, h, t, P / h ** 3)
        c = (n - 2) // 2
        rs = np.array([2e-3, 3e-3, 4e-3, 6e-3])
        num = np.array([th[c, c, c + int(round(r / h))] for r in rs])
        ana = P / (4 * math.pi * t.k * rs) * np.exp(-rs / Lb)
        errs.append(float(np.max(np.abs(num - ana) / ana)))
        if h == 1e-3:
            # the oracle's step keeps this discrete steady state fixed
            dt = 0.25
            case = _case(n, n, n, [t], _no_source(), face_bc=ph.DIRICHLET, h=h, dt=dt)
            m = oracle.setup(case, "f64")
            m.s[c + 1, c + 1, c + 1] = P / h ** 3 * dt / m.rhoc[c + 1, c + 1, c + 1]
            st = oracle.initial_state(m)
            st.theta[1:-1, 1:-1, 1:-1] = th
            before = st.theta.copy()
            oracle.run(m, st, 1)
            assert np.max(np.abs(st.theta - before)) <= 1e-10 * np.max(th)
            # and time stepping from T_a reaches it (8 perfusion time constants)
            st = oracle.initial_state(m)
            tau = t.rho * t.c / (t.w_b * t.rho_b * t.c_b)
            oracle.run(m, st, int(math.ceil(8 * tau / dt)))
            assert np.max(np.abs(st.theta[1:-1, 1:-1, 1:-1] - th)) <= 1e-3 * np.max(th)
    # the error against P/(4 pi k r) exp(-r/L) decreases monotonically under refinement
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.02


def test_erfc_held_boundary_refinement():
    """1D half space with x = 0 held at theta0 and no perfusion: theta0 erfc(x / 2 sqrt(kappa t));
    the time integral printed in Sec. 'General Formal Framework' is read as this solution."""
    t_ins = ph.Tissue(w_b=0.0)
    hot = ph.Tissue(fixed=1, T_fixed_C=37.0 + 53.0)
    kappa = t_ins.k / (t_ins.rho * t_ins.c)
    T_end = 30.0
    errs = []
    for h in (0.2e-3, 0.1e-3, 0.05e-3):
        nx = int(round(20e-3 / h))
        dt = 0.25 * h * h / kappa
        N = int(round(T_end / dt))
        lab = np.zeros((1, 1, nx), np.uint8)
        lab[0, 0, 0] = 1
        case = _case(nx, 1, 1, [t_ins, hot], _no_source(), face_bc=ph.INSULATED, h=h, dt=dt,
                     labels=lab)
        m = oracle.setup(case, "f64")
        st = oracle.initial_state(m)
        oracle.run(m, st, N)
        x = np.arange(nx) * h
        ana = 53.0 * np.array([math.erfc(xx / (2 * math.sqrt(kappa * N * dt))) for xx in x])
        sel = x <= 8e-3
        errs.append(float(np.max(np.abs(st.theta[0, 0, sel] - ana[sel]))))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.05


def test_monotone_heating_in_time_and_distance():
    """Sec. 'Results': the simulated heating is monotone in time and distance."""
    n = 21
    h = 1e-3
    c = ph.centre(n, h)
    nd = ph.Needle(kind=ph.STRAIGHT, tip=(c, c, c + 3e-3), active_len=6e-3, power=10.0)
    case = _case(n, n, n, [ph.liver()], nd, face_bc=ph.DIRICHLET, h=h, dt=0.2)
    m = oracle.setup(case, "f64")
    st = oracle.initial_state(m)
    prev = st.theta.copy()
    for _ in range(60):
        oracle.run(m, st, 1)
        assert np.all(st.theta >= prev)
        line = st.theta[n // 2, n // 2, n // 2:]
        assert np.all(np.diff(line) <= 0)
        prev = st.theta.copy()


def test_random_phantom_monotone_in_time():
    case = ph.random_small_case(3, 12, 10, 9, nsteps=0)
    m = oracle.setup(case, "f64")
    st = oracle.initial_state(m)
    prev = st.theta.copy()
    for _ in range(40):
        oracle.run(m, st, 1)
        assert np.all(st.theta >= prev)
        prev = st.theta.copy()


# ------------------------------------------------------------------ damage
def test_arrhenius_constant_temperature_kahan():
    TC = 70.0
    hot = ph.Tissue(fixed=1, T_fixed_C=TC)
    dmg = ph.Damage(enable=1)
    case = _case(4, 3, 2, [hot], _no_source(), face_bc=ph.INSULATED, dt=0.05, damage=dmg)
    m = oracle.setup(case, "f64")
    st = oracle.initial_state(m)
    N = 12000
    oracle.run(m, st, N, damage=dmg)
    inc = 0.05 * dmg.A * math.exp(-dmg.Ea / (dmg.R * (TC + 273.15)))
    exact = math.fsum([inc] * N)
    assert np.all(np.abs(st.omega - exact) <= math.ulp(exact))
    assert np.all(st.latch == 1)


# ------------------------------------------------------------------ brute force
@pytest.mark.parametrize("face_bc", [ph.DIRICHLET, ph.INSULATED])
def test_dense_brute_force_8cube(face_bc):
    case = ph.random_small_case(7, 8, 8, 8, face_bc=face_bc, nsteps=0, power=3.0)
    case.labels[2, 2, 2] = ph.VESSEL
    m = oracle.setup(case, "bf16")
    A, c = brute.step_matrix(m.a, m.b, m.s + m.qm, m.isfixed)
    N = 700
    ref = brute.evolve(A, c, m.theta0.ravel(), N)
    st = oracle.initial_state(m)
    oracle.run(m, st, N)
    assert np.max(np.abs(st.theta.ravel() - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_dense_brute_force_latch_and_damage():
    dmg = ph.Damage(enable=1, T_thr_C=45.0)
    case = ph.random_small_case(11, 6, 7, 5, nsteps=0, power=2.0, damage=dmg)
    m = oracle.setup(case, "f64")
    A, c = brute.step_matrix(m.a, m.b, m.s + m.qm, m.isfixed)
    N = 150
    th = m.theta0.ravel().copy()
    incs = [[] for _ in range(th.size)]
    latch = np.zeros(th.size, bool)
    for _ in range(N):
        th = A @ th + c
        TK = th + 37.0 + 273.15
        latch |= th + 37.0 >= 45.0
        for i in range(th.size):
            incs[i].append(0.05 * dmg.A * math.exp(-dmg.Ea / (dmg.R * TK[i])))
    st = oracle.initial_state(m)
    oracle.run(m, st, N, damage=dmg)
    om = np.array([math.fsum(v) for v in incs])
    assert np.array_equal(st.latch.ravel() != 0, latch)
    assert np.allclose(st.omega.ravel(), om, rtol=1e-12, atol=0)


def test_latch_after_each_step_tests_the_new_temperature():
    """The latch after n steps is max_{k=1..n} T^k >= T_thr (the step's new
    temperature, not the one it started from): checked against brute force at
    every step where the brute-force latch set grows, and the step before."""
    case = ph.random_small_case(11, 6, 7, 5, nsteps=0, power=2.0, damage=ph.Damage(enable=0, T_thr_C=45.0))
    m = oracle.setup(case, "f64")
    A, c = brute.step_matrix(m.a, m.b, m.s + m.qm, m.isfixed)
    th = m.theta0.ravel().copy()
    latch = np.zeros(th.size, bool)
    sets = [latch.copy()]
    for _ in range(150):
        th = A @ th + c
        latch |= th + case.T_a_C >= 45.0
        sets.append(latch.copy())
    grow = [n for n in range(1, len(sets)) if sets[n].sum() > sets[n - 1].sum()]
    assert len(grow) >= 3
    for n in sorted(set(grow) | {g - 1 for g in grow if g > 1}):
        st = oracle.initial_state(m)
        oracle.run(m, st, n, T_thr_C=45.0)
        assert np.array_equal(st.latch.ravel() != 0, sets[n]), n


# ------------------------------------------------------------------ paper set-up
def test_paper_fixed_tip_experiment_properties():
    """Sec. 'Evaluation Methods' / 'Simulation of Heat Propagation': a 5x5x3-voxel
    hemispherical tip at 0.5 mm held at 90 C, dt = 0.1 s.  The simulated heating is
    monotone at both probes, nearer is hotter, and the 5 mm probe stays below the
    42.5 C tissue-death threshold after one minute (as the paper reports)."""
    case = ph.paper_tip_case(90.0, nsteps=1200)
    m = oracle.setup(case, "f64")
    st = oracle.initial_state(m)
    pr = ph.paper_tip_probes()
    prev = None
    for k in range(12):
        oracle.run(m, st, 100)
        t25, t50 = (st.theta[pr["2.5mm"]] + 37.0, st.theta[pr["5mm"]] + 37.0)
        assert t25 > t50 > 37.0
        if prev is not None:
            assert t25 > prev[0] and t50 > prev[1]
        prev = (t25, t50)
        if k == 5:      # t = 60 s
            assert t50 < 42.5


# ------------------------------------------------------------------ necrosis read-out
def _necrosis_model(nx=6, ny=5, nz=4, h=2e-3):
    case = _case(nx, ny, nz, [ph.liver()], _no_source(), h=h)
    return oracle.setup(case, "f64")


def test_necrosis_counts_volumes_and_smoothed_volume_closed_forms():
    """The necrosis read-out (the 60 C criterion of Sec. "Introduction" and the
    Arrhenius criterion Omega >= 1 of Eq. eq-tissState), against values the
    definitions fix exactly:
      - sigma(0) = 1/2, so a field uniformly at the threshold has the smoothed
        volume h^3 N / 2;
      - sigma(ln 3) = 3/4 and sigma(-ln 3) = 1/4, at any width w when the field
        sits at thr +- w ln 3 (a width applied as a product, a flipped exponent
        or a missing h^3 changes these);
      - counts of a hand-set latch and Omega pattern (Omega exactly 1 counts,
        the double just below it does not), volumes h^3 * count."""
    h = 2e-3
    m = _necrosis_model(h=h)
    st = oracle.initial_state(m)
    N = st.theta.size
    h3 = h ** 3
    Ta = m.T_a

    # uniform at the threshold: sigma(0) = 1/2 everywhere
    st.theta[...] = 60.0 - Ta
    _, counts, vols, vs = oracle.necrosis(m, st)
    assert counts == (0, 0) and vols == (0.0, 0.0)
    assert math.isclose(vs, h3 * N / 2, rel_tol=1e-14)

    # thr + w ln 3 (sigma = 3/4) and thr - w ln 3 (sigma = 1/4), several widths and thresholds
    for w, thr in ((1.0, 60.0), (2.0, 60.0), (0.25, 42.5), (3.0, 50.0)):
        st.theta[...] = thr + w * math.log(3.0) - Ta
        vs_hi = oracle.necrosis(m, st, width_K=w, thr_C=thr)[3]
        assert math.isclose(vs_hi, 0.75 * h3 * N, rel_tol=1e-12), (w, thr)
        st.theta[...] = thr - w * math.log(3.0) - Ta
        vs_lo = oracle.necrosis(m, st, width_K=w, thr_C=thr)[3]
        assert math.isclose(vs_lo, 0.25 * h3 * N, rel_tol=1e-12), (w, thr)
    # half the voxels each way: 3/4 + 1/4 per pair
    flat = st.theta.reshape(-1)
    flat[0::2] = 60.0 + math.log(3.0) - Ta
    flat[1::2] = 60.0 - math.log(3.0) - Ta
    assert math.isclose(oracle.necrosis(m, st)[3], h3 * N / 2, rel_tol=1e-12)
    # far above and far below: sigma -> 1 and 0
    st.theta[...] = 60.0 + 200.0 - Ta
    assert math.isclose(oracle.necrosis(m, st)[3], h3 * N, rel_tol=1e-14)
    st.theta[...] = 60.0 - 200.0 - Ta
    assert oracle.necrosis(m, st)[3] < h3 * N * 1e-80

    # hand-set latch and Omega: counts, bits and volumes
    rng = np.random.default_rng(5)
    latch = (rng.random(st.latch.shape) < 0.3).astype(np.uint8)
    om = np.zeros(st.omega.shape)
    sel = rng.random(om.shape)
    om[sel < 0.2] = 1.0                               # exactly at the criterion: dead
    om[(sel >= 0.2) & (sel < 0.4)] = np.nextafter(1.0, 0.0)  # just below: alive
    om[(sel >= 0.4) & (sel < 0.5)] = 7.5              # well above: dead
    st.latch[...] = latch
    st.omega[...] = om
    mask, counts, vols, _ = oracle.necrosis(m, st)
    n_th = int(latch.sum())
    n_ar = int(np.count_nonzero(sel < 0.2) + np.count_nonzero((sel >= 0.4) & (sel < 0.5)))
    assert counts == (n_th, n_ar)
    assert vols == (h3 * n_th, h3 * n_ar)
    assert np.array_equal(mask & 1, latch)
    assert np.array_equal((mask >> 1) & 1, ((sel < 0.2) | ((sel >= 0.4) & (sel < 0.5))).astype(np.uint8))
    assert not (mask & ~np.uint8(3)).any()
