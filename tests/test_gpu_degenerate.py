"""Degenerate cases of the path on the GPU, against the FP64 oracle: a grid
with one interior voxel, one-voxel-thin slabs and lines, a grid of fixed
voxels only, a needle of zero power, metabolic heat alone, and the blocked
kernel on grids smaller than one tile."""
import numpy as np
import pytest

import paper_1907_05709_b300 as rfa
import phantoms as ph
from tests.parity_util import compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def _case(nx, ny, nz, table, needle, labels=None, face_bc=ph.DIRICHLET, h=1e-3, dt=0.05, damage=None):
    lab = np.zeros((nz, ny, nx), np.uint8) if labels is None else labels
    return ph.Case("degenerate", nx, ny, nz, h, dt, 0, lab, table, needle,
                   damage if damage is not None else ph.Damage(enable=1), face_bc=face_bc)


def _straight(nx, ny, nz, h=1e-3, power=3.0):
    c = ((nx - 1) * h / 2, (ny - 1) * h / 2, (nz - 1) * h / 2)
    return ph.Needle(kind=ph.STRAIGHT, tip=c, active_len=max(nz - 1, 1) * h * 0.5, power=power)


@pytest.mark.parametrize("sp", [rfa.STATE_F64, rfa.STATE_F32C])
def test_one_interior_voxel(sp):
    # Dirichlet faces leave one free voxel: it takes the whole power
    case = _case(3, 3, 3, [ph.liver()], _straight(3, 3, 3, power=0.05))
    orc = run_oracle(case, rfa.PARAM_BF16, 200)
    gpu = run_gpu(case, sp, rfa.PARAM_BF16, 200)
    compare(case, gpu, orc, sp)
    assert gpu["T"][1, 1, 1] > case.T_a_C and np.all(np.delete(gpu["T"].ravel(), 13) == case.T_a_C)


@pytest.mark.parametrize("dims", [(1, 9, 7), (11, 1, 1), (1, 1, 6), (6, 5, 1)])
def test_thin_slabs_and_lines_insulated(dims):
    nx, ny, nz = dims
    case = _case(nx, ny, nz, [ph.liver()], _straight(nx, ny, nz, power=0.5), face_bc=ph.INSULATED)
    orc = run_oracle(case, rfa.PARAM_F64, 150)
    gpu = run_gpu(case, rfa.STATE_F64, rfa.PARAM_F64, 150)
    compare(case, gpu, orc, rfa.STATE_F64)


def test_fixed_voxels_only():
    lab = np.full((6, 7, 8), ph.VESSEL, np.uint8)
    case = _case(8, 7, 6, [ph.liver(), ph.tumor(), ph.vessel()], _straight(8, 7, 6), labels=lab)
    gpu = run_gpu(case, rfa.STATE_F32C, rfa.PARAM_BF16, 50)
    assert np.all(gpu["T"] == ph.vessel().T_fixed_C)
    assert np.all(gpu["s"] == 0.0)
    assert int(gpu["counts"][0]) == 0


def test_zero_power_and_no_metabolic_heat_keep_the_ambient_temperature():
    case = _case(20, 18, 16, [ph.liver()], _straight(20, 18, 16, power=0.0))
    gpu = run_gpu(case, rfa.STATE_F32C, rfa.PARAM_BF16, 100)
    assert np.all(gpu["T"] == case.T_a_C)
    assert np.all(gpu["s"] == 0.0) and int(gpu["counts"][0]) == 0


def test_metabolic_heat_alone():
    t = ph.liver()
    t.Q_m = 10714.0                      # the paper's metabolic heat rate
    case = _case(20, 18, 16, [t], _straight(20, 18, 16, power=0.0))
    orc = run_oracle(case, rfa.PARAM_BF16, 300)
    for sp in (rfa.STATE_F64, rfa.STATE_F32C):
        gpu = run_gpu(case, sp, rfa.PARAM_BF16, 300)
        compare(case, gpu, orc, sp)
        assert gpu["T"][8, 9, 10] > case.T_a_C


@pytest.mark.parametrize("dims", [(6, 5, 4), (40, 7, 9), (3, 3, 3)])
def test_blocked_kernel_on_grids_smaller_than_a_tile(dims):
    nx, ny, nz = dims
    case = _case(nx, ny, nz, [ph.liver(), ph.tumor()], _straight(nx, ny, nz, power=0.3))
    a = run_gpu(case, rfa.STATE_F32C, rfa.PARAM_BF16, 9)
    b = run_gpu(case, rfa.STATE_F32C, rfa.PARAM_BF16, 9, schedule=(2, 0))
    assert np.array_equal(a["theta"], b["theta"]) and np.array_equal(a["latch"], b["latch"])
