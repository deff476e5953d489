"""Batched stepping (rfa_batch_*): several needle configurations on grids of
uneven size in one persistent launch must give the states of stepping every
member alone (bit-identical temperatures), and match the oracle."""
import numpy as np
import pytest

import paper_1907_05709_b300 as rfa
import phantoms as ph
from tests.parity_util import compare, run_oracle

pytestmark = pytest.mark.gpu

SIZES = [(40, 36, 30), (33, 17, 29), (64, 64, 64), (20, 50, 41), (71, 45, 38)]


def _members(damage, seed0=40):
    cases = [ph.random_small_case(seed0 + k, *dims, kind=ph.UMBRELLA if k % 2 else ph.STRAIGHT,
                                  power=4.0 + k) for k, dims in enumerate(SIZES)]
    grids = [rfa.Grid.from_case(c, damage=damage) for c in cases]
    return cases, grids


def _state(g):
    return g.field(rfa.FIELD_THETA), g.field(rfa.FIELD_LATCH), g.field(rfa.FIELD_OMEGA)


@pytest.mark.parametrize("damage", [False, True])
@pytest.mark.parametrize("sched", [None, (2, 0), (3, 0), (2, 1)])
def test_batch_equals_members_stepped_alone(damage, sched):
    cases, alone = _members(damage)
    _, grids = _members(damage)
    n1, n2 = 37, 64                                # remainders and a second call
    for g in alone:
        g.step(n1)
        g.step(n2)
    b = rfa.rfa_batch_create([g.handle for g in grids])
    if sched is not None:
        # the batch keeps its own schedule; set it through the tuner's cache
        import json, tempfile, os
        vox = sum(c.nvox for c in cases)
        path = os.path.join(tempfile.mkdtemp(), "tune.txt")
        with open(path, "w") as f:
            f.write(json.dumps({f"batch/{len(cases)}/{vox}/d{int(damage)}": list(sched)}) + "\n")
        rfa.rfa_batch_autotune(b, path)
        assert rfa.rfa_batch_get_schedule(b)[:2] == sched
    rfa.rfa_batch_step(b, n1)
    rfa.rfa_batch_step(b, n2)
    for g in grids:
        g.synchronize()
    for a, g in zip(alone, grids):
        ta, la, oa = _state(a)
        tg, lg, og = _state(g)
        assert np.array_equal(ta, tg)
        assert np.array_equal(la, lg)
        # the FP32 damage carry holds up to 256 steps before it is folded into FP64:
        # runs that fold at different steps differ by <= ~256 * 2^-24 relative
        assert np.allclose(oa, og, rtol=3e-5, atol=0)
        assert g.steps_done == n1 + n2
    rfa.rfa_batch_destroy(b)
    for g in alone + grids:
        g.close()


def test_batch_member_matches_oracle():
    cases, grids = _members(True, seed0=60)
    b = rfa.rfa_batch_create([g.handle for g in grids])
    n = 201
    rfa.rfa_batch_step(b, n)
    k = 4
    grids[0].synchronize()
    g = grids[k]
    gpu = dict(T=g.temperature(as_f64=True), theta=g.field(rfa.FIELD_THETA),
               omega=g.field(rfa.FIELD_OMEGA))
    mask, counts, vols, sv = g.necrosis()
    gpu.update(mask=mask, counts=counts, vols=vols, smooth=sv)
    orc = run_oracle(cases[k], rfa.PARAM_BF16, n)
    compare(cases[k], gpu, orc, rfa.STATE_F32C)
    rfa.rfa_batch_destroy(b)
    for g in grids:
        g.close()


def test_batch_autotune_restores_states(tmp_path):
    cases, grids = _members(True, seed0=80)
    for g in grids:
        g.step(5)
    before = [_state(g) for g in grids]
    b = rfa.rfa_batch_create([g.handle for g in grids])
    rfa.rfa_batch_autotune(b, str(tmp_path / "t.txt"))
    d, v, graphs = rfa.rfa_batch_get_schedule(b)
    assert (d, v) in [(2, 0), (3, 0), (2, 1)]
    for g, st in zip(grids, before):
        now = _state(g)
        assert all(np.array_equal(x, y) for x, y in zip(st, now))
        assert g.steps_done == 5
    rfa.rfa_batch_destroy(b)
    for g in grids:
        g.close()


def test_batch_rejects_unsupported_members():
    case = ph.random_small_case(3, 20, 20, 20)
    g64 = rfa.Grid.from_case(case, state_prec=rfa.STATE_F64)
    with pytest.raises(rfa.RfaError) as e:
        rfa.rfa_batch_create([g64.handle])
    assert e.value.status == 8
    g = rfa.Grid.from_case(case)
    with pytest.raises(rfa.RfaError):
        rfa.rfa_batch_create([g.handle, g.handle])
    g.close()
    g64.close()


def _oracle_sample(cases):
    """Eight members for the oracle comparison: the first of each grid size, the
    smallest 9-tine umbrella, 4-tine umbrella and straight needle not yet picked,
    then the smallest remaining ones."""
    pick = []
    for n in (96, 128, 160, 192):
        pick += [k for k, c in enumerate(cases) if c.nx == n][:1]
    by_size = sorted(range(len(cases)), key=lambda k: (cases[k].nvox, k))
    for pred in (lambda c: c.needle.kind == ph.UMBRELLA and c.needle.tine_axial == 1,
                 lambda c: c.needle.kind == ph.UMBRELLA and c.needle.tine_axial == 0,
                 lambda c: c.needle.kind == ph.STRAIGHT):
        pick += [k for k in by_size if pred(cases[k]) and k not in pick][:1]
    rest = sorted((c.nvox, k) for k, c in enumerate(cases) if k not in pick)
    pick += [k for _, k in rest[:8 - len(pick)]]
    return pick


def test_batch64_full_configuration():
    """The benchmark's batch as bench.py times it: 64 members on 96^3 .. 192^3
    grids, 4000 steps, the autotuned schedule in one graph-replayed persistent
    launch.  Sampled members (the smallest, the largest, a 9-tine umbrella)
    equal the same member stepped alone, bit for bit; eight members -- one of
    each grid size, each needle kind, the rest the smallest -- match the FP64
    oracle after all 4000 steps, every voxel (Eq. CUDAbioheat3d)."""
    cases = ph.batch_members(0, 64, 4000)
    grids = [rfa.Grid.from_case(c, damage=False) for c in cases]
    b = rfa.rfa_batch_create([g.handle for g in grids])
    rfa.rfa_batch_autotune(b, None)
    rfa.rfa_batch_step(b, 4000)
    for g in grids:
        g.synchronize()
    nvox = [c.nvox for c in cases]
    nine = [k for k, c in enumerate(cases) if c.needle.kind == ph.UMBRELLA and c.needle.tine_axial == 1]
    sample = sorted({int(np.argmin(nvox)), int(np.argmax(nvox)), nine[0]})
    for k in sample:
        alone = rfa.Grid.from_case(cases[k], damage=False)
        alone.step(4000)
        ta, la, _ = _state(alone)
        tb, lb, _ = _state(grids[k])
        assert np.array_equal(ta, tb) and np.array_equal(la, lb), k
        alone.close()
    pick = _oracle_sample(cases)
    assert len(pick) == 8 and {cases[k].nx for k in pick} == {96, 128, 160, 192}
    for k in pick:
        g = grids[k]
        gpu = dict(T=g.temperature(as_f64=True), theta=g.field(rfa.FIELD_THETA), omega=g.field(rfa.FIELD_OMEGA))
        mask, counts, vols, sv = g.necrosis()
        gpu.update(mask=mask, counts=counts, vols=vols, smooth=sv)
        orc = run_oracle(cases[k], rfa.PARAM_BF16, 4000, damage=False)
        res = compare(cases[k], gpu, orc, rfa.STATE_F32C, damage=False)
        print(f"member {k} ({cases[k].nx}^3, needle kind {cases[k].needle.kind}): max|dT| = {res['err_T']:.2e} K")
    rfa.rfa_batch_destroy(b)
    for g in grids:
        g.close()
