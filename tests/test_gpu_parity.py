"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs, element by element."""
import numpy as np
import pytest

import oracle
import paper_1907_05709_b300 as rfa
import phantoms as ph
from tests.parity_util import compare, run_gpu, run_oracle, PMODE

pytestmark = pytest.mark.gpu


def test_setup_and_source_fields_match_oracle():
    case = ph.random_small_case(2, 33, 17, 9, kind=ph.UMBRELLA)
    for sp, pp in [(rfa.STATE_F32C, rfa.PARAM_BF16), (rfa.STATE_F64, rfa.PARAM_F64),
                   (rfa.STATE_F32, rfa.PARAM_F32)]:
        gpu = run_gpu(case, sp, pp, 0)
        m = oracle.setup(case, PMODE[pp])
        # coefficients: identical after the same rounding
        assert np.array_equal(gpu["a"], m.a)
        assert np.array_equal(gpu["b"], m.b)
        s_ref = m.s + m.qm
        tol = 1e-12 if sp == rfa.STATE_F64 else 2 ** -23
        assert np.max(np.abs(gpu["s"] - s_ref) / np.maximum(s_ref, 1e-300)) <= tol
        assert np.array_equal(gpu["theta"], m.theta0)


def test_source_field_nine_tines_larger_grid():
    """The source weights on a 72 x 64 x 56 grid at h = 0.5 mm around a 9-tine
    umbrella (many voxels nearly equidistant from two tines): every voxel to
    1e-12 of the oracle's FP64 source."""
    case = ph.random_small_case(3, 72, 64, 56, h=0.5e-3, kind=ph.UMBRELLA)
    assert case.needle.n_tines == 8 and case.needle.tine_axial == 1
    gpu = run_gpu(case, rfa.STATE_F64, rfa.PARAM_F64, 0)
    m = oracle.setup(case, "f64")
    s_ref = m.s + m.qm
    assert np.max(np.abs(gpu["s"] - s_ref) / np.maximum(s_ref, 1e-300)) <= 1e-12


def test_homogeneous_64_fp64_2000_steps():
    """64^3, h = 1 mm, homogeneous liver, straight 15 mm needle at 15 W,
    dt = 0.05 s, 2000 steps, FP64 state: <= 1e-9 K."""
    case = ph.homogeneous_case()
    orc = run_oracle(case, rfa.PARAM_BF16, 2000)
    gpu = run_gpu(case, rfa.STATE_F64, rfa.PARAM_BF16, 2000)
    compare(case, gpu, orc, rfa.STATE_F64)
    assert orc["counts"][0] > 1000  # the case really ablates


def test_homogeneous_64_fp32c_2000_steps():
    case = ph.homogeneous_case()
    orc = run_oracle(case, rfa.PARAM_BF16, 2000)
    gpu = run_gpu(case, rfa.STATE_F32C, rfa.PARAM_BF16, 2000)
    res = compare(case, gpu, orc, rfa.STATE_F32C)
    assert res["err_T"] < 1e-4


@pytest.mark.parametrize("dims", [(33, 17, 9), (130, 67, 41), (1, 1, 50), (7, 1, 1), (5, 6, 200)])
@pytest.mark.parametrize("sp", [rfa.STATE_F32C, rfa.STATE_F64])
def test_ragged_phantoms_with_damage(dims, sp):
    nx, ny, nz = dims
    case = ph.random_small_case(sum(dims), nx, ny, nz, kind=ph.UMBRELLA, power=4.0,
                                face_bc=ph.INSULATED if min(dims) == 1 else ph.DIRICHLET)
    n = 150
    orc = run_oracle(case, rfa.PARAM_BF16, n)
    gpu = run_gpu(case, sp, rfa.PARAM_BF16, n)
    compare(case, gpu, orc, sp)


@pytest.mark.parametrize("pp", [rfa.PARAM_BF16, rfa.PARAM_F32, rfa.PARAM_F64])
def test_param_precisions(pp):
    case = ph.random_small_case(5, 40, 21, 19, kind=ph.STRAIGHT, power=6.0)
    n = 200
    orc = run_oracle(case, pp, n)
    gpu = run_gpu(case, rfa.STATE_F32C, pp, n)
    compare(case, gpu, orc, rfa.STATE_F32C)


def test_point_source_at_tile_corner():
    """A near-point source (r0 tiny) on the corner voxel of a 128 x 8 tile."""
    case = ph.random_small_case(9, 200, 20, 12, power=1.0)
    h = case.h
    case.needle = ph.Needle(kind=ph.STRAIGHT, tip=(127 * h, 7 * h, 6 * h), active_len=0.0,
                            power=1.0, r_clamp=1e-3 * h)
    case.labels[:] = ph.LIVER
    orc = run_oracle(case, rfa.PARAM_BF16, 120)
    gpu = run_gpu(case, rfa.STATE_F32C, rfa.PARAM_BF16, 120)
    compare(case, gpu, orc, rfa.STATE_F32C)
    assert np.argmax(gpu["T"]) == np.argmax(orc["T"])


def test_zero_steps_and_chunking():
    case = ph.random_small_case(4, 20, 20, 20, power=5.0)
    g0 = run_gpu(case, rfa.STATE_F32C, rfa.PARAM_BF16, 0)
    assert np.all(g0["T"] == 37.0 + g0["theta"])
    a = run_gpu(case, rfa.STATE_F32C, rfa.PARAM_BF16, 90)
    b = run_gpu(case, rfa.STATE_F32C, rfa.PARAM_BF16, 90, chunks=[1, 0, 44, 45])
    assert np.array_equal(a["T"], b["T"]) and np.array_equal(a["omega"], b["omega"])


def test_erfc_line_on_gpu():
    """1D insulated line held at 90 C at x = 0 (Sec. 'General Formal Framework' BC problem)."""
    t_ins = ph.Tissue(w_b=0.0)
    hot = ph.Tissue(fixed=1, T_fixed_C=90.0)
    nx = 300
    h = 0.1e-3
    kappa = t_ins.k / (t_ins.rho * t_ins.c)
    dt = 0.25 * h * h / kappa
    lab = np.zeros((1, 1, nx), np.uint8)
    lab[0, 0, 0] = 1
    case = ph.Case("erfc", nx, 1, 1, h, dt, 0, lab, [t_ins, hot],
                   ph.Needle(kind=ph.STRAIGHT, power=0.0), ph.Damage(enable=0),
                   face_bc=ph.INSULATED)
    orc = run_oracle(case, rfa.PARAM_F64, 800)
    gpu = run_gpu(case, rfa.STATE_F64, rfa.PARAM_F64, 800)
    compare(case, gpu, orc, rfa.STATE_F64)


@pytest.mark.parametrize("T_tip", [90.0, 60.0])
def test_paper_fixed_tip_setup(T_tip):
    """The paper's hemispherical 90 C / 60 C tip at 0.5 mm, dt = 0.1 s, 120 s."""
    case = ph.paper_tip_case(T_tip, nsteps=1200)
    orc = run_oracle(case, rfa.PARAM_BF16, 1200, damage=False)
    gpu = run_gpu(case, rfa.STATE_F32C, rfa.PARAM_BF16, 1200, damage=False)
    compare(case, gpu, orc, rfa.STATE_F32C, damage=False)
    gpu64 = run_gpu(case, rfa.STATE_F64, rfa.PARAM_BF16, 1200, damage=False)
    compare(case, gpu64, orc, rfa.STATE_F64, damage=False)


@pytest.mark.parametrize("T_tip", [90.0, 60.0])
def test_paper_fixed_tip_through_place_needle(T_tip):
    """The same set-up through rfa_place_needle with a FIXED_TIP needle (all
    voxels liver, no painted label): the library builds the hemisphere itself
    and must match the oracle run on the painted-label case, with the blocked
    kernel too (bit-identical to one step per launch)."""
    case = ph.paper_tip_case(T_tip, nsteps=1200)
    orc = run_oracle(case, rfa.PARAM_BF16, 1200, damage=False)
    lib_case = ph.paper_tip_needle_case(T_tip, nsteps=1200)
    for sp in (rfa.STATE_F32C, rfa.STATE_F64):
        gpu = run_gpu(lib_case, sp, rfa.PARAM_BF16, 1200, damage=False)
        compare(case, gpu, orc, sp, damage=False)
        tip = ph.paper_tip_case(T_tip, nsteps=0).labels == 1
        assert np.all(gpu["T"][tip] == T_tip) and np.all(gpu["a"][tip] == 0) and np.all(gpu["s"][tip] == 0)
    blk = run_gpu(lib_case, rfa.STATE_F32C, rfa.PARAM_BF16, 1200, damage=False, schedule=(2, 0))
    one = run_gpu(lib_case, rfa.STATE_F32C, rfa.PARAM_BF16, 1200, damage=False)
    assert np.array_equal(blk["T"], one["T"])


def test_fixed_tip_moves_and_is_removed():
    """Placing another needle gives the old hemisphere's voxels back their label's
    coefficients (free voxels keep their temperature); a moved tip paints the new
    place only; rfa_set_tissue starts over and paints the placed tip again."""
    lib_case = ph.paper_tip_needle_case(90.0, n=32, nsteps=0)
    g = rfa.Grid.from_case(lib_case, rfa.STATE_F32C, rfa.PARAM_BF16, damage=False)
    a_free = g.field(rfa.FIELD_A)[5, 5, 5]
    old = ph.paper_tip_case(90.0, n=32, nsteps=0).labels == 1
    assert np.all(g.field(rfa.FIELD_A)[old] == 0) and np.all(g.temperature()[old] == 90.0)
    g.step(50)
    T50 = g.temperature()
    nd = lib_case.needle
    moved = ph.Needle(kind=ph.FIXED_TIP, tip=(nd.tip[0] + 4 * lib_case.h, nd.tip[1], nd.tip[2]),
                      axis=(-1.0, 0.0, 0.0), power=0.0, T_tip_C=60.0)
    g.place_needle(moved)
    a = g.field(rfa.FIELD_A)
    T = g.temperature()
    c = 16
    new = np.zeros_like(old)
    for w in range(3):
        for u in range(-2, 3):
            for v in range(-2, 3):
                if 36 * u * u + 36 * v * v + 25 * w * w <= 225:
                    new[c + v, c + u, c + 4 - w] = True    # (z, y, x): dome toward -x
    assert np.all(a[new] == 0) and np.all(T[new] == 60.0)
    freed = old & ~new
    assert freed.any() and np.all(a[freed] == a_free) and np.array_equal(T[freed], T50[freed])
    with pytest.raises(rfa.RfaError) as e:
        rfa.rfa_set_conduction(g.handle, rfa.COND_HARMONIC)
    assert e.value.status == 8
    g.set_tissue(lib_case.labels, lib_case.table)        # starts over, the moved tip painted again
    T = g.temperature()
    assert np.all(T[new] == 60.0) and np.all(T[~new] == lib_case.T_a_C)
    g.close()
