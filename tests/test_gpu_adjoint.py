"""GPU adjoint (rfa_backward) against the FP64 oracle's discrete adjoint on the
same rounded coefficients, and the torch.autograd wrapper.

Tolerance: 1e-3 relative per gradient component (the accuracy target of the
path), with an absolute floor of 1e-3 of the largest component of its kind for
components near zero."""
import numpy as np
import pytest

import oracle
import paper_1907_05709_b300 as rfa
import phantoms as ph

pytestmark = pytest.mark.gpu


def c3_loss_seed(theta, T_a, target, sel, width=1.0, thr=60.0):
    """Seed dL/dT of L = mean_S (T - T*)^2 + mean sigmoid((T - 60)/1 K)."""
    T = theta + T_a
    d = T[sel] - target[sel]
    sig = 1.0 / (1.0 + np.exp(-(T - thr) / width))
    g = np.zeros_like(theta)
    g[sel] = 2.0 * d / d.size
    g += sig * (1 - sig) / width / theta.size
    return g


def _compare_grads(g_gpu, g_orc, nl):
    rel = 1e-3
    kinds = [slice(0, 1), slice(1, 4), slice(4, 4 + nl), slice(4 + nl, 4 + 2 * nl)]
    for k in kinds:
        a, b = g_gpu[k], g_orc[k]
        floor = 1e-3 * np.max(np.abs(b)) if np.any(b != 0) else 1e-300
        assert np.all(np.abs(a - b) <= rel * np.abs(b) + floor), (k, a, b)


def _adjoint_case(case, nsteps, seed_rng=0, chunks=None, schedule=None):
    m = oracle.setup(case, "bf16")
    st = oracle.initial_state(m)
    oracle.run(m, st, nsteps)
    rng = np.random.default_rng(seed_rng)
    sel = rng.random(m.a.shape) < 0.1
    target = st.theta + case.T_a_C + rng.normal(0, 2.0, size=m.a.shape)
    seed = c3_loss_seed(st.theta, case.T_a_C, target, sel)
    _, _, gk, gw, gP, gtip = oracle.adjoint(m, nsteps, seed)
    g_orc = np.concatenate([[gP], gtip, gk, gw])

    import torch
    g = rfa.Grid.from_case(case, damage=False)
    if schedule is not None:
        g.set_schedule(*schedule)
    for c in (chunks or [nsteps]):
        g.step(c, record=True)
    seed_dev = torch.from_numpy(seed.astype(np.float32)).cuda()
    g_gpu = g.backward(seed_dev)
    g.close()
    return g_gpu, g_orc


@pytest.mark.parametrize("kind", [ph.STRAIGHT, ph.UMBRELLA])
def test_adjoint_matches_oracle_small(kind):
    case = ph.random_small_case(31, 41, 34, 29, kind=kind, power=6.0)
    g_gpu, g_orc = _adjoint_case(case, 150)
    _compare_grads(g_gpu, g_orc, len(case.table))
    assert g_gpu[4 + ph.VESSEL] == 0.0 and g_gpu[4 + 3 + ph.VESSEL] == 0.0


@pytest.mark.parametrize("sched", [(2, 0), (2, 1)])
def test_adjoint_recorded_in_chunks_and_blocked_forward(sched):
    case = ph.random_small_case(32, 37, 30, 33, kind=ph.UMBRELLA, power=5.0)
    # forward by the 2-step blocked kernel; the recomputation replays the checkpoint
    # segments with the blocked kernel too (two steps per launch, Dirichlet faces)
    g_gpu, g_orc = _adjoint_case(case, 123, chunks=[50, 1, 72], schedule=sched)
    _compare_grads(g_gpu, g_orc, len(case.table))


def test_adjoint_128_cube_2000_steps():
    """128^3, h = 0.75 mm, tumour/vessel phantom, straight needle at 20 W,
    2000 steps: every gradient against the FP64 oracle adjoint."""
    case = ph.adjoint_case_128()
    g_gpu, g_orc = _adjoint_case(case, 2000)
    _compare_grads(g_gpu, g_orc, len(case.table))


def test_adjoint_256_cube_bounded_steps():
    """The HBM-bound size the bench times (256^3, h = 0.5 mm, straight needle at
    20 W), recorded with the autotuned blocked schedule; the oracle's FP64
    discrete adjoint is run for the first 150 of the bench's 2000 steps (about
    ten seconds of CPU work) and every gradient compared."""
    case = ph.adjoint_case_256(nsteps=150)
    g_gpu, g_orc = _adjoint_case(case, 150, schedule=(2, 0))
    _compare_grads(g_gpu, g_orc, len(case.table))


def test_backward_needs_recorded_steps():
    import torch
    case = ph.random_small_case(3, 20, 20, 20)
    g = rfa.Grid.from_case(case, damage=False)
    g.step(10)
    seed = torch.zeros(case.labels.shape, dtype=torch.float32, device="cuda")
    with pytest.raises(rfa.RfaError) as e:
        g.backward(seed)
    assert e.value.status == 5
    g.step(5, record=True)          # earlier unrecorded steps still block it
    with pytest.raises(rfa.RfaError):
        g.backward(seed)
    g.close()


def test_autograd_function_matches_rfa_backward():
    import torch
    from paper_1907_05709_b300.autograd import pack_params, simulate
    case = ph.random_small_case(33, 30, 28, 26, kind=ph.STRAIGHT, power=5.0)
    g = rfa.Grid.from_case(case, damage=False)
    params = pack_params(case.needle, case.table).requires_grad_(True)
    T = simulate(g, case.labels, case.table, case.needle, params, 80)
    target = T.detach() + 0.5
    loss = ((T - target) ** 2).mean() + torch.sigmoid((T - 60.0) / 1.0).mean()
    loss.backward()
    seed = (2.0 * (T.detach() - target) / T.numel()
            + torch.sigmoid((T.detach() - 60.0)) * (1 - torch.sigmoid((T.detach() - 60.0))) / T.numel())
    direct = g.backward(seed.contiguous())
    assert np.allclose(params.grad.numpy(), direct, rtol=1e-5, atol=0)
    assert params.grad[0].item() != 0.0
    g.close()


def test_adjoint_rows_across_thread_blocks():
    """Rows of 150 voxels span two blocks of 32 quads, the second ragged: the
    reverse step's x neighbours across the block edge and the clamped lanes past
    the row's end."""
    case = ph.random_small_case(33, 150, 24, 20, kind=ph.UMBRELLA, power=6.0)
    g_gpu, g_orc = _adjoint_case(case, 80)
    _compare_grads(g_gpu, g_orc, len(case.table))
