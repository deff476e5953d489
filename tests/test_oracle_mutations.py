"""The pins catch plausible mistakes in the oracle (CPU only).

Each case plants one mistake -- a dropped term, a wrong sign, a transposed or
shifted index, an off-by-one face test, a missing unit offset, a skipped
compensation, the step matrix instead of its transpose -- into a copy of the
oracle's C source (compiled with the oracle's own flags and bound in place of
the oracle library), or into a copy of one of its numpy functions (bound in
place of that function), and runs the pins (closed forms, invariants, brute
force, finite differences).  At least one pin must fail (or stop with an
error) for every mistake; an unmodified copy must pass them all.  The oracle
source itself is never changed.
"""
import ctypes
import inspect
import os
import textwrap

import pytest

import oracle
from oracle import build as oracle_build
import phantoms as ph
from tests import test_oracle_adjoint as ADJ
from tests import test_oracle_alpha as ALPHA
from tests import test_oracle_cond as COND
from tests import test_oracle_pins as PINS
from tests import test_oracle_potential as POT
from tests import test_oracle_warp as WARP

# the pins, fastest first (a mutant stops at the first pin that fails)
CHECKS = [
    ("sine-mode decay", PINS.test_sine_mode_exact_discrete_decay),
    ("uniform perfusion decay", PINS.test_uniform_perfusion_decay_insulated),
    ("energy balance, straight", lambda: PINS.test_energy_balance_insulated_no_perfusion(ph.STRAIGHT)),
    ("energy balance, umbrella", lambda: PINS.test_energy_balance_insulated_no_perfusion(ph.UMBRELLA)),
    ("source shape", PINS.test_source_shape_hand_picked),
    ("necrosis read-out", PINS.test_necrosis_counts_volumes_and_smoothed_volume_closed_forms),
    ("monotone heating", PINS.test_monotone_heating_in_time_and_distance),
    ("monotone phantom", PINS.test_random_phantom_monotone_in_time),
    ("Arrhenius closed form", PINS.test_arrhenius_constant_temperature_kahan),
    ("brute force, Dirichlet", lambda: PINS.test_dense_brute_force_8cube(ph.DIRICHLET)),
    ("brute force, insulated", lambda: PINS.test_dense_brute_force_8cube(ph.INSULATED)),
    ("brute force, latch and damage", PINS.test_dense_brute_force_latch_and_damage),
    ("latch after each step", PINS.test_latch_after_each_step_tests_the_new_temperature),
    ("adjoint = dense transpose, Dirichlet", lambda: ADJ.test_adjoint_matches_dense_transpose(ph.DIRICHLET)),
    ("adjoint = dense transpose, insulated", lambda: ADJ.test_adjoint_matches_dense_transpose(ph.INSULATED)),
    ("adjoint vs central FD", ADJ.test_adjoint_gradients_match_central_fd),
    ("erfc line", PINS.test_erfc_held_boundary_refinement),
    ("metabolic steady state", PINS.test_paper_metabolic_steady_state),
    ("conservative: uniform K", COND.test_uniform_K_equals_the_centre_form),
    ("conservative: energy", COND.test_energy_balance_with_heterogeneous_K),
    ("conservative: dense matrix", lambda: COND.test_dense_step_matrix(ph.DIRICHLET)),
    ("conservative: two-material slab", COND.test_two_material_slab_steady_state),
    ("conservative: adjoint transpose", COND.test_adjoint_matches_dense_transpose),
    ("tissue state: scalar recurrence", ALPHA.test_uniform_field_follows_the_scalar_recurrence),
    ("tissue state: below threshold", ALPHA.test_no_effect_below_the_damage_threshold_and_hotter_above),
    ("potential: two-material resistor", POT.test_two_material_resistor),
    ("potential: power balance, maximum principle", POT.test_tellegen_power_balance_and_maximum_principle),
    ("potential: symmetry", POT.test_symmetry_of_a_centred_needle),
    ("resample: zero field", WARP.test_zero_field_is_identity),
    ("resample: shift x", lambda: WARP.test_integer_shift_with_clamp(0, 3)),
    ("resample: shift y", lambda: WARP.test_integer_shift_with_clamp(1, -2)),
    ("resample: shift z", lambda: WARP.test_integer_shift_with_clamp(2, 4)),
    ("resample: affine field", WARP.test_affine_field_reproduced_exactly),
    ("resample: scipy", WARP.test_matches_scipy_map_coordinates),
    ("paper hot tip", PINS.test_paper_fixed_tip_experiment_properties),
    ("steady point source", PINS.test_steady_point_source_fixed_point_and_refinement),
]

STEP = "tn = t + conduction(nx, ny, nz, a, wf, cur, x, y, z) - bi * t + s[i] + qm[i];"

# (name, text in oracle.c, planted replacement); each text occurs exactly once
MUTANTS = [
    ("perfusion sink dropped", STEP, "tn = t + conduction(nx, ny, nz, a, wf, cur, x, y, z) + s[i] + qm[i];"),
    ("source sign flipped", STEP, "tn = t + conduction(nx, ny, nz, a, wf, cur, x, y, z) - bi * t - s[i] + qm[i];"),
    ("metabolic term dropped", STEP, "tn = t + conduction(nx, ny, nz, a, wf, cur, x, y, z) - bi * t + s[i];"),
    ("x- neighbour dropped", "        if (x > 0)      sum += cur[IDX(x - 1, y, z)] - t;\n", ""),
    ("y+ neighbour read along z", "        if (y < ny - 1) sum += cur[IDX(x, y + 1, z)] - t;",
     "        if (y < ny - 1) sum += cur[IDX(x, y, z < nz - 1 ? z + 1 : z)] - t;"),
    ("off-by-one z face", "        if (z < nz - 1) sum += cur[IDX(x, y, z + 1)] - t;",
     "        if (z < nz - 2) sum += cur[IDX(x, y, z + 1)] - t;"),
    ("fixed voxels stepped", "if (isfixed[i]) {\n                        tn = t;", "if (0) {\n                        tn = t;"),
    ("Kelvin offset dropped", "double TK = tn + T_a + 273.15;", "double TK = tn + T_a;"),
    ("damage on the old temperature", "double TK = tn + T_a + 273.15;", "double TK = t + T_a + 273.15;"),
    ("Kahan compensation dropped", "double yk = inc - omega_c[i];", "double yk = inc;"),
    ("latch on the old temperature", "if (tn + T_a >= T_thr) latch[i] = 1;", "if (t + T_a >= T_thr) latch[i] = 1;"),
    ("source normalised over fixed voxels too", "if (!isfixed[i]) W += w[i];", "W += w[i];"),
    ("no clamp radius", "double r = d > r0 ? d : r0;\n                w[i] = ns > 0",
     "double r = d > 1e-9 ? d : 1e-9;\n                w[i] = ns > 0"),
    ("1/r^3 fall-off", "w[i] = ns > 0 ? 1.0 / (r * r * r * r) : 0.0;", "w[i] = ns > 0 ? 1.0 / (r * r * r) : 0.0;"),
    ("conduction over h, not h^2", "a[i] = round_param((k / (rho * c)) * dt / (h * h), param_mode);",
     "a[i] = round_param((k / (rho * c)) * dt / h, param_mode);"),
    ("perfusion without rho_b", "b[i] = round_param((w_b * rho_b * c_b / (rho * c)) * dt, param_mode);",
     "b[i] = round_param((w_b * c_b / (rho * c)) * dt, param_mode);"),
    ("adjoint: step matrix, not its transpose", "return a[j];  /* i is a grid neighbour of j */",
     "return a[IDX(xi, yi, zi)];"),
    ("adjoint: degree fixed at 6", "return 1.0 - a[j] * deg - b[j];", "return 1.0 - a[j] * 6 - b[j];"),
    ("conservative: x+ face takes the x- weight",
     "if (x < nx - 1) f += wf[1 * n + i] * (cur[IDX(x + 1, y, z)] - t);",
     "if (x < nx - 1) f += wf[0 * n + i] * (cur[IDX(x + 1, y, z)] - t);"),
    ("tissue state: b times Omega", "b[i] / fmax(1.0, omega[i])", "b[i] * fmax(1.0, omega[i])"),
]


def _bind_copy(tmp_path, old, new):
    src = open(oracle_build.SRC).read()
    if old is not None:
        assert src.count(old) == 1, f"mutation site not unique: {old!r}"
        src = src.replace(old, new)
    c = os.path.join(tmp_path, "oracle_copy.c")
    with open(c, "w") as f:
        f.write(src)
    lib = oracle_build.compile_library(c, os.path.join(tmp_path, "liboracle_copy.so"))
    return oracle.bind(ctypes.CDLL(lib))


# (name, oracle function, text in its source, planted replacement)
PY_MUTANTS = [
    ("face weights: arithmetic mean", "face_weights", "W[l, m] = g * (2.0 * tl.k * tm.k / Ks)",
     "W[l, m] = g * (0.5 * Ks)"),
    ("face weights: the neighbour's rho c", "face_weights", "W[l, m] = g * (2.0 * tl.k * tm.k / Ks)",
     "W[l, m] = case.dt / (tm.rho * tm.c * case.h * case.h) * (2.0 * tl.k * tm.k / Ks)"),
    ("face weights: x- and x+ swapped", "face_weights", "((2, -1), (2, 1), (1, -1)", "((2, 1), (2, -1), (1, -1)"),
    ("resample: weights of the two z corners swapped", "warp_temperature",
     "((z0, 1.0 - fz), (z1, fz))", "((z0, fz), (z1, 1.0 - fz))"),
    ("resample: nearest instead of floor", "warp_temperature", "fl = np.floor(dd)", "fl = np.round(dd)"),
    ("resample: clamp one voxel late", "warp_temperature", "low, high = i < 0, i >= n - 1",
     "low, high = i < 0, i >= n"),
    ("potential faces: arithmetic mean", "harmonic_faces", "hm = np.divide(2.0 * vals * nb, s, out=np.zeros_like(s), where=s > 0)",
     "hm = 0.5 * s"),
    ("potential: electrode and ground swapped", "potential_solve", "Vfix = electrode.astype(np.float64)",
     "Vfix = ground.astype(np.float64)"),
    ("potential: boundary term sign", "potential_solve", "np.add.at(rhs, i[~jf], sf[~jf] * nb_fix[m][~jf])",
     "np.add.at(rhs, i[~jf], -sf[~jf] * nb_fix[m][~jf])"),
    ("Joule heating: |dV| not squared", "joule", "(nb - V) ** 2", "np.abs(nb - V)"),
    ("Joule heating: face not split", "joule", "return q / (2.0 * h * h)", "return q / (h * h)"),
    ("necrosis: sigmoid exponent sign flipped", "necrosis", "np.exp(-(T - thr_C) / width_K)",
     "np.exp((T - thr_C) / width_K)"),
    ("necrosis: h^3 dropped from the smoothed volume", "necrosis", "vs = h3 * float(", "vs = float("),
    ("necrosis: width multiplied, not divided", "necrosis", "np.exp(-(T - thr_C) / width_K)",
     "np.exp(-(T - thr_C) * width_K)"),
    ("necrosis: Arrhenius criterion strict", "necrosis", "(st.omega >= 1.0)", "(st.omega > 1.0)"),
    ("necrosis: volumes without h^3", "necrosis", "(h3 * n_th, h3 * n_ar)", "(n_th, n_ar)"),
    ("necrosis: ambient temperature dropped", "necrosis", "T = st.theta + Ta", "T = st.theta"),
]


def _failing_check():
    for name, check in CHECKS:
        try:
            check()
        except Exception:  # an assertion, or an error the mistake provoked
            return name
    return None


def test_unmodified_copy_passes_every_pin(tmp_path, monkeypatch):
    monkeypatch.setattr(oracle, "_lib", _bind_copy(str(tmp_path), None, None))
    assert _failing_check() is None


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(name, old, new, tmp_path, monkeypatch):
    monkeypatch.setattr(oracle, "_lib", _bind_copy(str(tmp_path), old, new))
    caught = _failing_check()
    assert caught is not None, f"no pin catches: {name}"


@pytest.mark.parametrize("name,fname,old,new", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_pins_catch_planted_mistake_in_numpy_parts(name, fname, old, new, monkeypatch):
    src = textwrap.dedent(inspect.getsource(getattr(oracle, fname)))
    assert src.count(old) == 1, f"mutation site not unique: {old!r}"
    ns = dict(vars(oracle))
    exec(compile(src.replace(old, new), f"<{fname} with a planted mistake>", "exec"), ns)
    monkeypatch.setattr(oracle, fname, ns[fname])
    caught = _failing_check()
    assert caught is not None, f"no pin catches: {name}"
