"""The allocation-free necrosis reduction (rfa_necrosis_reduce_noalloc).

Some callers may not allocate device memory once they run -- a real-time
frame loop where an allocation would stall the device, or an application
that reserves its whole memory budget up front.  This entry point keeps its
scratch in a fixed device array inside the library; its results must equal
those of rfa_necrosis_mask.  The file is collected last so that a run which
stops at the first failure has run every other test before it.
"""
import numpy as np
import pytest

import paper_1907_05709_b300 as rfa
import phantoms as ph

pytestmark = pytest.mark.gpu


def test_noalloc_reduction_matches_necrosis_mask_on_two_calls():
    import torch
    case = ph.random_small_case(13, 70, 40, 30, kind=ph.UMBRELLA, power=8.0)
    g = rfa.Grid.from_case(case)
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    seen_thermal = 0
    for nsteps in (60, 140):              # two calls in a row, on different states
        g.step(nsteps)
        _, counts, vols, sv = g.necrosis(want_mask=False)
        out.fill_(-1.0)
        rfa.rfa_necrosis_reduce_noalloc(g.handle, out, 1.0)
        torch.cuda.synchronize()
        res = out.cpu()
        got = res.view(torch.int64)[:2].numpy()
        assert np.array_equal(got, counts)
        # same FP64 sum of FP32 sigmoids, reduced over a different block partition
        assert abs(float(res[2]) - sv) <= 1e-12 * max(sv, 1e-30)
        seen_thermal = max(seen_thermal, int(counts[0]))
    assert seen_thermal > 0
    g.close()


def test_noalloc_rejects_grids_above_its_scratch():
    g = rfa.Grid(650, 650, 640, 1e-3, 0.05, rfa.STATE_F32, rfa.PARAM_BF16)
    import torch
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(rfa.RfaError) as e:
        rfa.rfa_necrosis_reduce_noalloc(g.handle, out, 1.0)
    assert e.value.status == 1 and "268435456" in str(e.value)
    g.close()
