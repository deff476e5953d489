"""Conservative conduction (rfa_set_conduction(RFA_COND_HARMONIC)): GPU one-step
kernel and its adjoint against the FP64 oracle on the same seeded inputs and the
same FP32-rounded label-pair weights.  Tolerances as in the other parity tests
(FP64 state 1e-9 K, compensated FP32 1e-3 K, gradients 1e-3 relative)."""
import numpy as np
import pytest

import oracle
import paper_1907_05709_b300 as rfa
import phantoms as ph
from tests.parity_util import compare, run_gpu, run_oracle
from tests.test_gpu_adjoint import _compare_grads, c3_loss_seed

pytestmark = pytest.mark.gpu


def _case(seed, dims, face_bc=ph.DIRICHLET, kind=ph.UMBRELLA, power=6.0):
    c = ph.random_small_case(seed, *dims, kind=kind, power=power, face_bc=face_bc)
    c.table[ph.TUMOR].k = 1.6
    c.table[ph.VESSEL].k = 0.3
    c.conduction = "harmonic"
    return c


@pytest.mark.parametrize("sp", [rfa.STATE_F64, rfa.STATE_F32C])
@pytest.mark.parametrize("dims,face", [((41, 34, 29), ph.DIRICHLET), ((33, 17, 9), ph.INSULATED)])
def test_conservative_step_matches_oracle(sp, dims, face):
    case = _case(70, dims, face_bc=face)
    n = 201
    orc = run_oracle(case, rfa.PARAM_BF16, n)
    gpu = run_gpu(case, sp, rfa.PARAM_BF16, n)
    compare(case, gpu, orc, sp)


def test_conservative_fp64_coefficients():
    case = _case(71, (30, 26, 22))
    orc = run_oracle(case, rfa.PARAM_F64, 120)
    gpu = run_gpu(case, rfa.STATE_F64, rfa.PARAM_F64, 120)
    compare(case, gpu, orc, rfa.STATE_F64)


@pytest.mark.parametrize("face", [ph.DIRICHLET, ph.INSULATED])
def test_conservative_adjoint_matches_oracle(face):
    import torch
    # insulated faces: face voxels are updated too, so their adjoint rows differ
    case = _case(72, (37, 30, 33), face_bc=face, kind=ph.STRAIGHT, power=5.0)
    nsteps = 130
    m = oracle.setup(case, "bf16")
    st = oracle.initial_state(m)
    oracle.run(m, st, nsteps)
    rng = np.random.default_rng(0)
    sel = rng.random(m.a.shape) < 0.1
    target = st.theta + case.T_a_C + rng.normal(0, 2.0, size=m.a.shape)
    seed = c3_loss_seed(st.theta, case.T_a_C, target, sel)
    _, _, gk, gw, gP, gtip = oracle.adjoint(m, nsteps, seed)
    g_orc = np.concatenate([[gP], gtip, gk, gw])
    g = rfa.Grid.from_case(case, damage=False)
    g.step(nsteps, record=True)
    g_gpu = g.backward(torch.from_numpy(seed.astype(np.float32)).cuda())
    g.close()
    _compare_grads(g_gpu, g_orc, len(case.table))
    assert g_gpu[4 + ph.VESSEL] != 0.0          # the vessel's K sets its face conductances


def test_conservative_mode_refusals():
    case = _case(73, (20, 20, 20))
    g = rfa.Grid.from_case(case)
    with pytest.raises(rfa.RfaError) as e:
        g.set_schedule(2, 0)                     # no blocked kernel for this form
    assert e.value.status == 8
    with pytest.raises(rfa.RfaError) as e:
        rfa.rfa_batch_create([g.handle])
    assert e.value.status == 8
    with pytest.raises(rfa.RfaError) as e:
        rfa.rfa_set_conduction(g.handle, 5)
    assert e.value.status == 1
    g.close()
    # an unstable time step for the harmonic weights is refused at set-up
    bad = _case(74, (16, 16, 16))
    bad.table[ph.TUMOR].k = 60.0
    g = rfa.Grid(bad.nx, bad.ny, bad.nz, bad.h, bad.dt)
    rfa.rfa_set_conduction(g.handle, rfa.COND_HARMONIC)
    with pytest.raises(rfa.RfaError) as e:
        g.set_tissue(bad.labels, bad.table)
    assert e.value.status == 4
    g.close()


@pytest.mark.parametrize("cond,perf", [("harmonic", "constant"), ("centre", "tissue_state"),
                                       ("harmonic", "tissue_state")])
@pytest.mark.parametrize("face", [ph.DIRICHLET, ph.INSULATED])
def test_model_step_rows_across_thread_blocks(cond, perf, face):
    """Rows of 150 voxels span two blocks of 32 quads, the second one ragged: the
    x neighbours are read across the block edge (lane 31 of the first block, lane
    0 of the second), and the lanes past the row's end read a clamped quad and
    store nothing."""
    case = _case(73, (150, 22, 16), face_bc=face, power=8.0)
    case.conduction, case.perfusion = cond, perf
    n = 160
    orc = run_oracle(case, rfa.PARAM_BF16, n)
    gpu = run_gpu(case, rfa.STATE_F32C, rfa.PARAM_BF16, n)
    compare(case, gpu, orc, rfa.STATE_F32C)


def test_conservative_adjoint_rows_across_thread_blocks():
    import torch
    case = _case(74, (150, 24, 20), kind=ph.STRAIGHT, power=5.0)
    nsteps = 90
    m = oracle.setup(case, "bf16")
    st = oracle.initial_state(m)
    oracle.run(m, st, nsteps)
    rng = np.random.default_rng(1)
    sel = rng.random(m.a.shape) < 0.1
    target = st.theta + case.T_a_C + rng.normal(0, 2.0, size=m.a.shape)
    seed = c3_loss_seed(st.theta, case.T_a_C, target, sel)
    _, _, gk, gw, gP, gtip = oracle.adjoint(m, nsteps, seed)
    g_orc = np.concatenate([[gP], gtip, gk, gw])
    g = rfa.Grid.from_case(case, damage=False)
    g.step(nsteps, record=True)
    g_gpu = g.backward(torch.from_numpy(seed.astype(np.float32)).cuda())
    g.close()
    _compare_grads(g_gpu, g_orc, len(case.table))
