"""The allocation-free necrosis reduction (rfa_necrosis_reduce_noalloc).

Some callers may not allocate device memory once they run -- a real-time
frame loop where an allocation would stall the device, or an application
that reserves its whole memory budget up front.  This entry point keeps its
scratch in a fixed device array inside the library; its results must equal
those of rfa_necrosis_mask, and agree with the FP64 oracle's necrosis
read-out on the same seeded case.  The file is collected last so that a run
which stops at the first failure has run every other test before it.
"""
import numpy as np
import pytest

import oracle
import paper_1907_05709_b300 as rfa
import phantoms as ph

pytestmark = pytest.mark.gpu


def test_noalloc_reduction_matches_necrosis_mask_and_oracle_on_two_calls():
    import torch
    case = ph.random_small_case(13, 70, 40, 30, kind=ph.UMBRELLA, power=8.0)
    g = rfa.Grid.from_case(case)
    m = oracle.setup(case, "bf16")
    st = oracle.initial_state(m)
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
        assert float(res[3]) == 0.0
        seen_thermal = max(seen_thermal, int(counts[0]))

        # the FP64 oracle on the same inputs (Eq. CUDAbioheat3d, the 60 C latch and
        # Eq. eq-tissState): counts equal up to the voxels within the temperature
        # tolerance of the threshold (or |Omega - 1| <= 1e-2), smoothed volume to the
        # FP32 evaluation of the sigmoids
        oracle.run(m, st, nsteps, damage=case.damage)
        _, oc, _, osv = oracle.necrosis(m, st, thr_C=case.damage.T_thr_C)
        T_o = st.theta + case.T_a_C
        band_th = int(np.count_nonzero(np.abs(T_o - case.damage.T_thr_C) <= 1e-3))
        band_ar = int(np.count_nonzero(np.abs(st.omega - 1.0) <= 1e-2))
        assert abs(int(got[0]) - oc[0]) <= band_th
        assert abs(int(got[1]) - oc[1]) <= band_ar
        assert abs(float(res[2]) - osv) <= 1e-5 * max(osv, case.h ** 3)
    assert seen_thermal > 0
    g.close()


def test_noalloc_rejects_a_misaligned_result_buffer_before_any_launch():
    import torch
    case = ph.random_small_case(13, 20, 12, 9, kind=ph.UMBRELLA, power=4.0)
    g = rfa.Grid.from_case(case)
    buf = torch.full((64,), 0xAB, dtype=torch.uint8, device="cuda")
    with pytest.raises(rfa.RfaError) as e:
        rfa.rfa_necrosis_reduce_noalloc(g.handle, buf[4:36], 1.0)
    assert e.value.status == 1 and "aligned" in str(e.value)
    torch.cuda.synchronize()
    assert bool((buf.cpu() == 0xAB).all())   # nothing was written
    g.close()


def test_noalloc_rejects_grids_above_its_scratch():
    g = rfa.Grid(650, 650, 640, 1e-3, 0.05, rfa.STATE_F32, rfa.PARAM_BF16)
    import torch
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(rfa.RfaError) as e:
        rfa.rfa_necrosis_reduce_noalloc(g.handle, out, 1.0)
    assert e.value.status == 1 and "268435456" in str(e.value)
    g.close()


def test_noalloc_reduction_captures_in_a_cuda_graph():
    """After its first call on a device the entry point neither allocates nor
    synchronises: a second call is captured into a CUDA graph on the grid's
    stream (an allocating or synchronising call would end the capture with an
    error), and replays of the graph read the state at replay time and give the
    results of rfa_necrosis_mask."""
    import torch
    case = ph.random_small_case(17, 48, 40, 32, kind=ph.UMBRELLA, power=8.0)
    s = torch.cuda.Stream()
    g = rfa.Grid.from_case(case, cuda_stream=s.cuda_stream)
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(s):
        g.step(40)
        rfa.rfa_necrosis_reduce_noalloc(g.handle, out, 1.0)   # the first call looks up the scratch
    s.synchronize()
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg, stream=s):
        rfa.rfa_necrosis_reduce_noalloc(g.handle, out, 1.0)
    seen = 0
    for nsteps in (60, 120):
        with torch.cuda.stream(s):
            g.step(nsteps)
            out.fill_(-1.0)
            cg.replay()
        s.synchronize()
        res = out.cpu()
        _, counts, _, sv = g.necrosis(want_mask=False)
        assert np.array_equal(res.view(torch.int64)[:2].numpy(), counts)
        assert abs(float(res[2]) - sv) <= 1e-12 * max(sv, 1e-30)
        seen = max(seen, int(counts[0]))
    assert seen > 0
    del cg
    g.close()
