#!/usr/bin/env python3
"""Throughput benchmark of the RFA bioheat hot path on B300.

One bench "step" is one pass of the whole hot path over one synthetic
phantom: tissue set-up (labels -> coefficients), needle placement (RF
source), N explicit time steps fused with the 60 C latch and the FP64
Arrhenius integral, and the necrosis reduction.  Default workload (large512):
512^3 voxels, h = 0.25 mm, 1-3 tumours and 8 vessels, 9-tine umbrella at
40 W, dt = 0.02 s, 5000 steps, BF16 coefficient fields, compensated FP32
state.  The 256^3 single-needle workload (4-tine umbrella at 30 W, 12000
steps) is timed beside it, with the one-step kernel too, as are the adjoint,
the batch and the model options.

The metric is voxel-steps per second (GVox-steps/s); ``value`` times the
device-resident path (labels already in HBM), ``e2e`` the same work through
the C ABI from host buffers including the host<->device copies.  Multi-GPU
runs (torchrun) simulate independent phantoms per rank (weak scaling, no
collective on the data path).

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the
same workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import phantoms as ph  # noqa: E402

METRIC = "bioheat GVox-steps/s and % HBM roofline; batched+adjoint vs plain @1e-3 K"
NOMINAL_HBM_GBS = 7700.0
UNIT = "GVox-steps/s"


def workload(name: str, seed: int, sim_steps):
    if name == "umbrella256":
        c = ph.umbrella_case_256(seed=seed)
    elif name == "homogeneous64":
        c = ph.homogeneous_case()
    elif name == "adjoint128":
        c = ph.adjoint_case_128(seed=seed)
    elif name == "adjoint256":
        c = ph.adjoint_case_256(seed=seed)
    elif name == "large512":
        c = ph.large_case_512(seed=seed)
    else:
        raise SystemExit(f"unknown workload {name}")
    if sim_steps:
        c.nsteps = int(sim_steps)
    return c


def workload_config(c, name, oracle_arm: bool = False):
    """The workload of a bench line; ``oracle_arm`` describes the FP64 oracle's
    arithmetic (the reference arm) instead of the GPU path's."""
    gb = 46.0 * c.nvox / 1e9
    return {"workload": name, "grid": [c.nx, c.ny, c.nz], "h_mm": c.h * 1e3, "dt_s": c.dt,
            "time_steps": c.nsteps, "needle": {0: "straight", 1: "umbrella", 2: "fixed tip"}[c.needle.kind],
            # every tine: the ring's and the axial one (the 9-tine umbrella: 8 + 1)
            "n_tines": c.needle.n_tines + c.needle.tine_axial if c.needle.kind == 1 else 0,
            "axial_tine": bool(c.needle.tine_axial) if c.needle.kind == 1 else False,
            "power_W": c.needle.power, "arrhenius": bool(c.damage.enable),
            "state": "fp64 (oracle)" if oracle_arm else "fp32 hi+lo compensated",
            "coefficients": "bf16 (rounded, fed to the FP64 oracle)" if oracle_arm else "bf16",
            "l2": f"inputs larger than L2 (working set ~46 B/voxel, {gb:.1f} GB)"}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    Q = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.lines = []
        self.proc = None

    def start(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.uuid:
                cmd[1:1] = ["-i", self.uuid]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 10:
                continue
            try:
                sm.append(float(p[2]))
                smax.append(float(p[3]))
                power.append(float(p[4]))
            except ValueError:
                continue
            for nm, v in zip(names, p[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ roofline
def algorithmic_bytes_per_voxel(arrhenius: bool, depth: int) -> float:
    """Compulsory HBM bytes per voxel for one launch of the step kernel
    (compensated FP32 state, BF16 coefficients): theta hi+lo read and written
    (16), packed a/b (4), source (4), latch read+write (2); with the damage
    integral its FP32 carry read and written (8) and the FP64 value read and
    written (16) on the launches that fold the carry (every 256 steps)."""
    fold = 16.0 * depth / 256.0
    return 16 + 4 + 4 + 2 + ((8 + fold) if arrhenius else 0)


KERNEL_SOURCES = {
    "k_step_tb": ["kernels_tb.cu", "rfa_update.cuh", "rfa_internal.cuh"],
    "k_step_plain": ["kernels_step.cu", "rfa_update.cuh", "rfa_internal.cuh"],
}


def kernel_source_sha(kernel: str):
    """Hash of the source files that define ``kernel``."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1907_05709_b300", "csrc")
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def load_traffic(kernel: str, nvox: int):
    """DRAM bytes per launch from the committed ncu summary (profiles/traffic.json),
    if it was taken on the current sources of that kernel (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(p))
    except Exception:
        return None
    e = d.get(kernel)
    if not e or e.get("source_sha") != kernel_source_sha(kernel):
        return None
    return e["bytes_per_voxel_per_launch"] * nvox


def measured_peak_hbm():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


# ------------------------------------------------------------------ CPU oracle
def oracle_sample(case, target_s=15.0, min_steps=2, max_steps=2000, nthreads=0, model=None):
    """Time the FP64 oracle on the full grid for a bounded number of steps
    (nthreads 0: all cores)."""
    import oracle
    t0 = time.perf_counter()
    m = model if model is not None else oracle.setup(case, "bf16")
    t_setup = time.perf_counter() - t0
    st = oracle.initial_state(m)
    dmg = case.damage if case.damage.enable else None
    t0 = time.perf_counter()
    oracle.run(m, st, min_steps, damage=dmg, nthreads=nthreads)
    t_cal = (time.perf_counter() - t0) / min_steps
    n = int(max(min_steps, min(max_steps, target_s / max(t_cal, 1e-9))))
    t0 = time.perf_counter()
    oracle.run(m, st, n, damage=dmg, nthreads=nthreads)
    t = time.perf_counter() - t0
    return n, t, t_setup, m


def cpu_baseline(case, target_s=15.0):
    """The oracle on all host cores, and on one thread beside it (a shorter
    sample): the per-step cost is fixed, so a few steps give the rate."""
    n, t, _, m = oracle_sample(case, target_s)
    n1, t1, _, _ = oracle_sample(case, max(2.0, target_s / 5), min_steps=1, nthreads=1, model=m)
    # the 64^3 homogeneous case run entirely (2000 steps), all cores
    import oracle
    c0 = ph.homogeneous_case()
    m0 = oracle.setup(c0, "bf16")
    st0 = oracle.initial_state(m0)
    t0 = time.perf_counter()
    oracle.run(m0, st0, c0.nsteps)
    t_c0 = time.perf_counter() - t0
    return {"value": case.nvox * n / t / 1e9, "unit": UNIT, "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"FP64 oracle (C, OpenMP over z, {os.cpu_count()} threads), full "
                      f"{case.nx}x{case.ny}x{case.nz} phantom, {n} of {case.nsteps} time steps"
                      f"{' with Arrhenius' if case.damage.enable else ''}, set-up excluded",
            "single_thread": {"value": case.nvox * n1 / t1 / 1e9, "unit": UNIT, "cores": 1,
                              "sample": f"the same, 1 thread, {n1} time steps"},
            "homogeneous64_full": {"value": c0.nvox * c0.nsteps / t_c0 / 1e9, "unit": UNIT,
                                   "cores": os.cpu_count(),
                                   "sample": f"64^3 homogeneous liver, all {c0.nsteps} steps"}}


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    case = workload(args.workload, 0, args.sim_steps)
    import oracle
    # The oracle's set-up (S1, S2) runs once and is charged to every step pro rata:
    # one bench step of the GPU runs the set-up and all case.nsteps time steps, one
    # step here a bounded sample of n time steps on the full grid plus the necrosis
    # read-out, with n / case.nsteps of the set-up time added.
    n, t_cal, t_setup, m = oracle_sample(case, target_s=3.0, min_steps=2)
    per_step_target = float(os.environ.get("RFA_REFERENCE_STEP_S", "5.0"))
    n = max(2, int(n * per_step_target / 3.0))
    dmg = case.damage if case.damage.enable else None
    st = oracle.initial_state(m)
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.run(m, st, n, damage=dmg)
        oracle.necrosis(m, st)
        dt = time.perf_counter() - t0 + t_setup * n / case.nsteps
        if k >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = case.nvox * n * len(times) / tot / 1e9
    sample = (f"FP64 oracle (C, OpenMP over z, {os.cpu_count()} threads) on the full "
              f"{case.nx}x{case.ny}x{case.nz} phantom: {n} of {case.nsteps} time steps"
              f"{' with Arrhenius' if case.damage.enable else ''} + necrosis per step, plus "
              f"{n}/{case.nsteps} of the set-up's {t_setup:.1f} s")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(case, args.workload, oracle_arm=True),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ secondary
def _ms_between(torch, stream, fn):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def measure_adjoint(rfa, stream, conduction="centre", cpu_baseline_on: bool = False, name="adjoint128"):
    """adjoint128: 128^3, h = 0.75 mm, straight 20 W needle, 2000 steps (its
    fields sit in L2); adjoint256: the same at 256^3, h = 0.5 mm (~0.8 GB of
    fields, HBM-bound).  Recorded forward (sqrt(N) checkpoints) vs rfa_backward
    (recompute + adjoint + contractions), seed = a uniform dL/dT.
    conduction="harmonic" runs the conservative form (its own forward and
    adjoint kernels)."""
    import torch
    case = workload(name, 0, None)
    case.conduction = conduction
    g = rfa.Grid.from_case(case, damage=False, cuda_stream=stream.cuda_stream)
    rfa.rfa_autotune(g.handle, None)      # the forward runs with the tuned schedule
    seed = torch.full(case.labels.shape, 1e-6, dtype=torch.float32, device="cuda")
    fwd = lambda: g.step(case.nsteps, record=True)
    out = {}

    def reset():
        g.set_tissue(case.labels, case.table)

    reset()
    fwd()
    g.backward(seed)          # warm-up
    reset()
    t_f = _ms_between(torch, stream, fwd)
    t_b = _ms_between(torch, stream, lambda: out.setdefault("g", g.backward(seed)))
    reset()
    sched = rfa.rfa_get_schedule(g.handle)
    t_plain = _ms_between(torch, stream, lambda: g.step(case.nsteps))
    g.close()
    res = {"workload": name, "grid": [case.nx, case.ny, case.nz], "time_steps": case.nsteps,
           "forward_recorded_ms": t_f, "backward_ms": t_b, "forward_unrecorded_ms": t_plain,
           "backward_over_forward": t_b / t_f, "schedule": sched}
    if cpu_baseline_on:
        # the oracle's discrete adjoint beside it: 20 reverse steps of the same case
        import oracle
        mo = oracle.setup(case, "f64")
        seed_np = np.full((case.nz, case.ny, case.nx), 1e-6)
        t0 = time.perf_counter()
        oracle.adjoint(mo, 20, seed_np)
        t = time.perf_counter() - t0
        res["cpu_baseline"] = {"value": case.nvox * 20 / t / 1e9, "unit": "GVox-steps/s (backward)",
                               "cores": os.cpu_count(), "kind": "oracle",
                               "sample": f"{case.nx}^3, 20 steps of the FP64 oracle's adjoint (recompute and reverse)"}
    return res


def measure_single_grid(rfa, stream, name="umbrella256", schedule="auto", nsteps=None):
    """One grid of ``name`` stepped alone with the given schedule ("auto": the
    autotuner's pick, "plain": one step per launch): GVox-steps/s and the step
    kernel's fraction of HBM on its algorithmic bytes (per launch, averaged over
    the run, CUDA events on the launching stream).  Set-up outside the timing."""
    import torch
    case = workload(name, 0, nsteps)
    g = rfa.Grid.from_case(case, cuda_stream=stream.cuda_stream)
    if schedule == "auto":
        rfa.rfa_autotune(g.handle, os.environ.get("RFA_AUTOTUNE_CACHE") or None)
    elif schedule == "plain":
        g.set_schedule(1, 0)
    depth, variant = rfa.rfa_get_schedule(g.handle)
    g.step(min(case.nsteps, 200))                 # warm-up
    g.set_tissue(case.labels, case.table)
    ms = _ms_between(torch, stream, lambda: g.step(case.nsteps))
    g.close()
    launches = case.nsteps // depth + case.nsteps % depth
    peak, _ = measured_peak_hbm()
    nbytes = algorithmic_bytes_per_voxel(bool(case.damage.enable), depth) * case.nvox
    achieved = nbytes * launches / (ms * 1e-3) / 1e9
    return {"workload": name, "grid": [case.nx, case.ny, case.nz], "time_steps": case.nsteps,
            "schedule": {"tb_depth": depth, "tile_variant": variant},
            "kernel": "k_step_tb" if depth > 1 else "k_step_plain",
            "gvox_steps_s": case.nvox * case.nsteps / (ms * 1e-3) / 1e9, "ms": ms,
            "avg_launch_us": 1e3 * ms / launches, "bytes_per_voxel_per_launch": nbytes / case.nvox,
            "achieved_GBs": achieved, "peak_GBs": peak, "frac": achieved / peak}


def measure_next_rows(rfa, stream, case, g, cpu_baseline_on: bool):
    """The model options, each against its compulsory bytes (HBM roofline), and
    -- the CPU-baseline leg, unless disabled -- the FP64 oracle timed on a
    bounded sample beside it: breathing resample (Eq. breathing) of the bench
    grid; conservative conduction step, step with tissue-state perfusion and
    potential-solve source (CG iterations) on the 256^3 single-needle phantom."""
    import torch
    peak, _ = measured_peak_hbm()
    out = {}
    n = case.nvox
    cores = os.cpu_count()

    def roof(nbytes, ms, nvox=None):
        gbs = nbytes / (ms * 1e-3) / 1e9
        return {"achieved_GBs": gbs, "peak_GBs": peak, "frac": gbs / peak,
                "bytes_per_voxel": nbytes / (nvox or n)}

    def cpu(value, unit, sample):
        return {"value": value, "unit": unit, "cores": cores, "kind": "oracle", "sample": sample}

    # breathing resample of the bench grid's current state to an FP32 field: u 12 B,
    # theta hi 4 B (a float output reads hi alone), T 4 B
    u = torch.from_numpy(ph.breathing_field(case, 1.0)).cuda()
    dst = torch.empty((case.nz, case.ny, case.nx), dtype=torch.float32, device="cuda")
    rfa.rfa_warp_temperature(g.handle, u, dst, False)
    ms = _ms_between(torch, stream, lambda: [rfa.rfa_warp_temperature(g.handle, u, dst, False)
                                             for _ in range(5)]) / 5
    out["breathing_warp"] = dict(roof(20.0 * n, ms), ms=ms, gvox_s=n / (ms * 1e-3) / 1e9)
    del u, dst
    if cpu_baseline_on:
        import oracle
        sm = ph.single_needle_case(seed=1, n=96, nsteps=1)
        mo = oracle.setup(sm, "bf16")
        uo = ph.breathing_field(sm, 1.0)
        t0 = time.perf_counter()
        oracle.warp_temperature(mo.theta0, uo, sm.h, sm.T_a_C)
        out["breathing_warp"]["cpu_baseline"] = cpu(sm.nvox / (time.perf_counter() - t0) / 1e9, "GVox/s",
                                                    "96^3 resample, numpy FP64")
    # conservative conduction / tissue-state perfusion, 20 steps on a second grid;
    # bytes per voxel-step: theta hi+lo 16, a/b 4, s 4, label 1, latch 2, carry 8 (+ Omega 8)
    for name, cond, perf, bpv in (("conservative_step", "harmonic", "constant", 35.0),
                                  ("tissue_state_step", "centre", "tissue_state", 43.0)):
        c2 = ph.umbrella_case_256(seed=0, nsteps=20)
        c2.conduction, c2.perfusion = cond, perf
        g2 = rfa.Grid.from_case(c2, cuda_stream=stream.cuda_stream)
        g2.step(4)
        ms = _ms_between(torch, stream, lambda: g2.step(20)) / 20
        g2.close()
        n2 = c2.nvox
        out[name] = dict(roof(bpv * n2, ms, n2), workload="umbrella256", ms_per_step=ms,
                         gvox_steps_s=n2 / (ms * 1e-3) / 1e9)
        if cpu_baseline_on:
            import oracle
            sm = ph.single_needle_case(seed=1, n=96, nsteps=4)
            sm.conduction, sm.perfusion = cond, perf
            mo = oracle.setup(sm, "bf16")
            st = oracle.initial_state(mo)
            t0 = time.perf_counter()
            oracle.run(mo, st, 4, damage=sm.damage)
            out[name]["cpu_baseline"] = cpu(sm.nvox * 4 / (time.perf_counter() - t0) / 1e9, "GVox-steps/s",
                                            "96^3, 4 steps, FP64 oracle (C, OpenMP)")
    # potential-solve source: FP32 CG iterations inside an FP64 defect correction, with the
    # multigrid preconditioner (default) and, beside it, Jacobi.  Fine-grid bytes per voxel
    # and iteration -- Jacobi 54: direction + spmv (cls, label, D, z, previous p read, p and
    # Ap written: 22), update (1/D, e, r, p, Ap read, e, r, z written: 32).  Multigrid 164:
    # direction + spmv 22, update (e, r, p, Ap read, e, r written) 24, r.z 8, and the
    # V-cycle's fine passes 110 (first sweep b, 1/D read, x written 12; three sweeps and the
    # residual, each x, b, D, 1/D or the residual, cls, label ~21 / 17.5; restriction 4.5;
    # prolongation 12.5).  Coarse levels (about 1/7 more), the set-up and the FP64
    # correction passes are not counted: the figures are floors.
    c3 = ph.umbrella_case_256(seed=0, nsteps=1)
    g3 = rfa.Grid(c3.nx, c3.ny, c3.nz, c3.h, c3.dt, rfa.STATE_F32C, rfa.PARAM_BF16, c3.face_bc, c3.T_a_C,
                  stream.cuda_stream)
    g3.set_tissue(c3.labels, c3.table)
    sig = [t.sigma for t in c3.table]
    rfa.rfa_place_needle_potential(g3.handle, c3.needle, sig, 40, 1e-30)      # warm-up
    res = {}
    ms = _ms_between(torch, stream, lambda: res.setdefault(
        "r", rfa.rfa_place_needle_potential(g3.handle, c3.needle, sig, 20000, 1e-10)))
    rfa.rfa_set_potential_preconditioner(g3.handle, rfa.PRECOND_JACOBI)
    ms_j = _ms_between(torch, stream, lambda: res.setdefault(
        "j", rfa.rfa_place_needle_potential(g3.handle, c3.needle, sig, 20000, 1e-10)))
    g3.close()
    it, rel = res["r"]
    it_j, rel_j = res["j"]
    keys = ("workload", "grid", "time_steps", "forward_recorded_ms", "backward_ms", "backward_over_forward")
    adj = measure_adjoint(rfa, stream, conduction="harmonic")
    out["conservative_adjoint"] = {k: adj[k] for k in keys}
    adj = measure_adjoint(rfa, stream, conduction="harmonic", name="adjoint256")   # fields beyond L2
    out["conservative_adjoint256"] = {k: adj[k] for k in keys}
    n3 = c3.nvox
    out["potential_source"] = dict(roof(164.0 * n3 * it, ms, n3), workload="umbrella256", ms=ms,
                                   preconditioner="multigrid", cg_iterations=it,
                                   rel_residual=rel, ms_per_iteration=ms / max(it, 1),
                                   jacobi={"ms": ms_j, "cg_iterations": it_j, "rel_residual": rel_j,
                                           "frac": roof(54.0 * n3 * it_j, ms_j, n3)["frac"]},
                                   multigrid_over_jacobi=ms_j / ms)
    if cpu_baseline_on:
        import oracle
        sm = ph.single_needle_case(seed=1, n=32, nsteps=1)
        sm.source = "potential"
        t0 = time.perf_counter()
        oracle.setup(sm, "bf16")
        out["potential_source"]["cpu_baseline"] = cpu(time.perf_counter() - t0, "s",
                                                      "32^3 set-up with a direct sparse solve (scipy)")
    return out


def measure_path_rows(rfa, stream, case, g, labels_dev, cpu_baseline_on: bool = True):
    """The path's steps outside the time loop at the bench's size, on the bench
    grid after its timed steps: S6, the necrosis counts and smoothed volume
    (the allocation-free entry point: device result, no host copy), against its
    bytes (latch 1, Omega 8, carry 4, theta hi+lo 8 = 21 B/voxel); S1 + S2,
    rfa_set_tissue (coefficients, start state, and the needle placed again),
    and S2 alone, rfa_place_needle (FP64 distances to the needle's segments,
    FP64 sum of the weights: bound by B300's FP64 pipe, once per placement)."""
    import torch
    peak, _ = measured_peak_hbm()
    n = case.nvox
    out = {}
    res = torch.zeros(4, dtype=torch.float64, device="cuda")
    rfa.rfa_necrosis_reduce_noalloc(g.handle, res, 1.0)
    ms = _ms_between(torch, stream, lambda: [rfa.rfa_necrosis_reduce_noalloc(g.handle, res, 1.0)
                                             for _ in range(10)]) / 10
    gbs = 21.0 * n / (ms * 1e-3) / 1e9
    out["necrosis_reduce"] = {"ms": ms, "bytes_per_voxel": 21.0, "achieved_GBs": gbs, "peak_GBs": peak,
                              "frac": gbs / peak, "gvox_s": n / (ms * 1e-3) / 1e9}
    ms = _ms_between(torch, stream, lambda: [g.set_tissue(labels_dev, case.table) for _ in range(3)]) / 3
    out["tissue_setup_and_source"] = {"ms": ms, "gvox_s": n / (ms * 1e-3) / 1e9}
    ms = _ms_between(torch, stream, lambda: [g.place_needle(case.needle) for _ in range(3)]) / 3
    out["source_place"] = {"ms": ms, "gvox_s": n / (ms * 1e-3) / 1e9}
    if cpu_baseline_on:
        # the oracle beside them, on a 96^3 sample of the same phantom generator
        import oracle
        cores = os.cpu_count()
        sm = ph.single_needle_case(seed=1, n=96, nsteps=4)
        t0 = time.perf_counter()
        mo = oracle.setup(sm, "bf16")
        t_setup = time.perf_counter() - t0
        st = oracle.initial_state(mo)
        oracle.run(mo, st, 4, damage=sm.damage)
        t0 = time.perf_counter()
        oracle.necrosis(mo, st)
        t_nec = time.perf_counter() - t0
        for key, t, what in (("tissue_setup_and_source", t_setup, "set-up and 1/r^4 source"),
                             ("necrosis_reduce", t_nec, "necrosis mask, counts and smoothed volume")):
            out[key]["cpu_baseline"] = {"value": sm.nvox / t / 1e9, "unit": "GVox/s", "cores": cores,
                                        "kind": "oracle", "sample": f"96^3, {what}, FP64 oracle"}
    return out


def measure_batched(rfa, stream, args):
    """64 needle configurations on {96,128,160,192}^3 grids, 4000 steps (or
    --batch-steps), with the latch and the Arrhenius integral as in the headline:
    one batched persistent launch per call vs the per-needle loop of one-step
    launches, and vs the per-needle loop with the tuned schedule."""
    import torch
    cases = ph.batch_members(0, 64, args.batch_steps)
    grids = [rfa.Grid.from_case(c, damage=True, cuda_stream=stream.cuda_stream) for c in cases]
    vox = sum(c.nvox for c in cases)
    n = args.batch_steps
    b = rfa.rfa_batch_create([g.handle for g in grids])
    rfa.rfa_batch_autotune(b, None)
    rfa.rfa_batch_step(b, 24)             # warm-up (graph capture)
    t_batch = _ms_between(torch, stream, lambda: rfa.rfa_batch_step(b, n))
    d, v, graph = rfa.rfa_batch_get_schedule(b)
    rfa.rfa_batch_destroy(b)

    def loop(depth, variant):
        for g in grids:
            g.set_schedule(depth, variant)
        for g in grids:
            g.step(n)

    t_plain = _ms_between(torch, stream, lambda: loop(1, 0))
    t_tuned = _ms_between(torch, stream, lambda: loop(d, v))
    for g in grids:
        g.close()
    return {"workload": "batch64", "members": len(cases), "voxels": vox, "time_steps": n, "arrhenius": True,
            "batched_ms": t_batch, "batched_gvox_steps_s": vox * n / t_batch / 1e6,
            "plain_loop_ms": t_plain, "plain_loop_gvox_steps_s": vox * n / t_plain / 1e6,
            "tuned_loop_ms": t_tuned, "batched_over_plain_loop": t_plain / t_batch,
            "batched_over_tuned_loop": t_tuned / t_batch,
            "schedule": {"tb_depth": d, "tile_variant": v, "cuda_graph": graph}}


# ------------------------------------------------------------------ our arm
# ------------------------------------------------------------------ ranks
def reduce_max(x: float, dist, device) -> float:
    """Max over ranks (identity on one process); every rank gets the result."""
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(nvox: int, nsteps: int, bench_steps: int, world: int, ms_max: float) -> float:
    """Whole-job GVox-steps/s: every rank advances its own replica (weak scaling),
    divided by the slowest rank's time."""
    return nvox * nsteps * bench_steps * world / (ms_max * 1e-3) / 1e9


def run_ours(args):
    import torch
    import paper_1907_05709_b300 as rfa

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    case = workload(args.workload, rank, args.sim_steps)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(case, target_s=args.cpu_seconds)

    stream = torch.cuda.current_stream()
    g = rfa.Grid(case.nx, case.ny, case.nz, case.h, case.dt, rfa.STATE_F32C, rfa.PARAM_BF16,
                 case.face_bc, case.T_a_C, stream.cuda_stream)
    labels_dev = torch.from_numpy(np.ascontiguousarray(case.labels)).to(dev)
    labels_pin = torch.from_numpy(np.ascontiguousarray(case.labels)).pin_memory()
    T_host = torch.empty(case.nvox, dtype=torch.float32).pin_memory()
    d = case.damage
    g.set_tissue(labels_dev, case.table)
    g.place_needle(case.needle)
    g.set_damage(int(d.enable), d.A, d.Ea, d.R, d.T_thr_C)
    depth, variant = 1, 0
    if args.schedule == "auto":
        try:
            # RFA_AUTOTUNE_CACHE: optional JSON file the autotuner reads and updates
            rfa.rfa_autotune(g.handle, os.environ.get("RFA_AUTOTUNE_CACHE") or None)
        except rfa.RfaError:
            pass
    elif args.schedule.startswith("tb"):        # tbN or tbNvV: depth N, tile variant V
        dv = args.schedule[2:].split("v")
        g.set_schedule(int(dv[0]), int(dv[1]) if len(dv) > 1 else 0)
    depth, variant = rfa.rfa_get_schedule(g.handle)

    step_ms = []
    whole_ms = []

    def one_step(host: bool):
        lab = labels_pin if host else labels_dev
        w0 = torch.cuda.Event(enable_timing=True)
        w1 = torch.cuda.Event(enable_timing=True)
        w0.record(stream)
        g.set_tissue(lab, case.table)       # S1, and S2 (the placed needle is placed again)
        g.set_damage(int(d.enable), d.A, d.Ea, d.R, d.T_thr_C)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.step(case.nsteps)
        e1.record(stream)
        _, counts, vols, sv = g.necrosis(want_mask=False)
        if host:
            rfa.rfa_get_temperature(g.handle, T_host, False, False)
        w1.record(stream)
        step_ms.append((e0, e1))
        whole_ms.append((w0, w1))
        return counts

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        one_step(False)
    barrier()
    step_ms.clear()
    whole_ms.clear()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clk = ClockSampler(uuid)
    clk.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(args.steps):
        counts = one_step(False)
    t_end.record(stream)
    barrier()
    clocks = clk.stop()
    ms = t_start.elapsed_time(t_end)
    kern_ms = sum(a.elapsed_time(b) for a, b in step_ms)
    per_step = sorted(case.nvox * case.nsteps / (a.elapsed_time(b) * 1e-3) / 1e9 for a, b in whole_ms)
    step_stats = {"best": per_step[-1], "median": statistics.median(per_step), "worst": per_step[0],
                  "n": len(per_step), "unit": UNIT}
    ms_max = reduce_max(ms, dist, dev)
    vox_steps = case.nvox * case.nsteps * args.steps * world
    value = job_throughput(case.nvox, case.nsteps, args.steps, world, ms_max)

    # end to end from host buffers (labels in, temperature field out)
    e2e = None
    if not args.no_e2e:
        # at most 5 bench steps (each is a whole simulation), wall clock around them
        n_e2e = max(2, min(args.steps, 5))
        one_step(True)
        barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            one_step(True)
        barrier()
        wall = time.perf_counter() - t0
        e2e = {"value": case.nvox * case.nsteps * n_e2e * world / reduce_max(wall, dist, dev) / 1e9,
               "unit": UNIT, "steps": n_e2e,
               "h2d_bytes_per_step": int(case.nvox + 256 * 9 * 8 + 104),
               "d2h_bytes_per_step": int(case.nvox * 4 + 32 + 4)}

    # roofline of the dominant kernel (the step kernel)
    launches_per_step = (case.nsteps // depth + case.nsteps % depth) if depth > 1 else case.nsteps
    avg_launch_ms = kern_ms / (args.steps * launches_per_step)
    nbytes = algorithmic_bytes_per_voxel(bool(d.enable), depth) * case.nvox
    peak, peak_kind = measured_peak_hbm()
    achieved = nbytes / (avg_launch_ms * 1e-3) / 1e9
    kname = "k_step_tb" if depth > 1 else "k_step_plain"
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": load_traffic(kname, case.nvox),
            "kernel": kname, "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)",
            "algorithmic_bytes_per_launch": nbytes, "avg_launch_us": avg_launch_ms * 1e3,
            "steps_per_launch": depth,
            "nominal": {"peak": NOMINAL_HBM_GBS, "frac": achieved / NOMINAL_HBM_GBS,
                        "note": "B300 HBM3e nominal 7.7 TB/s; the frac above is of measured"}}
    kernels_per_step = 2 + 3 + launches_per_step + 2   # setup (2), source (3), steps, necrosis (2)
    secondary = None
    if rank == 0 and not args.no_secondary:
        secondary = {}
        if args.workload != "umbrella256":
            secondary["umbrella256"] = measure_single_grid(rfa, stream, "umbrella256", "auto")
        secondary["umbrella256_plain"] = measure_single_grid(rfa, stream, "umbrella256", "plain", 2000)
        secondary["adjoint"] = measure_adjoint(rfa, stream, cpu_baseline_on=not args.no_cpu_baseline)
        secondary["adjoint256"] = measure_adjoint(rfa, stream, name="adjoint256")
        secondary["batched"] = measure_batched(rfa, stream, args)
        secondary["next_rows"] = measure_next_rows(rfa, stream, case, g, not args.no_cpu_baseline)
        secondary["path_rows"] = measure_path_rows(rfa, stream, case, g, labels_dev, not args.no_cpu_baseline)
        # the ratios the targets name, last in the line (a log tail keeps them)
        summ = {"headline_frac": roof["frac"]}
        if "umbrella256" in secondary:
            summ["umbrella256_gvox_steps_s"] = secondary["umbrella256"]["gvox_steps_s"]
            summ["umbrella256_frac"] = secondary["umbrella256"]["frac"]
        summ["plain_step_frac_256"] = secondary["umbrella256_plain"]["frac"]
        summ["adjoint128_backward_over_forward"] = secondary["adjoint"]["backward_over_forward"]
        summ["adjoint256_backward_over_forward"] = secondary["adjoint256"]["backward_over_forward"]
        summ["conservative_adjoint128_backward_over_forward"] = \
            secondary["next_rows"]["conservative_adjoint"]["backward_over_forward"]
        summ["conservative_adjoint256_backward_over_forward"] = \
            secondary["next_rows"]["conservative_adjoint256"]["backward_over_forward"]
        summ["batched_over_plain_loop"] = secondary["batched"]["batched_over_plain_loop"]
        summ["batched_over_tuned_loop"] = secondary["batched"]["batched_over_tuned_loop"]
        summ["batched_gvox_steps_s"] = secondary["batched"]["batched_gvox_steps_s"]
        secondary["summary"] = summ
    if dist is not None:
        dist.barrier()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic (seeded tumour/vessel phantom per rank)",
                "config": dict(workload_config(case, args.workload),
                               parallelism=f"replicas x{world}" if world > 1 else "single GPU",
                               schedule={"tb_depth": depth, "tile_variant": variant}),
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "per_step": step_stats,
                "gpu_launches": kernels_per_step * args.steps,
                "necrosis_voxels": [int(counts[0]), int(counts[1])],
                "secondary": secondary}
        print(json.dumps(line), flush=True)
    g.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def profile_case(name):
    """Short fixed cases for ncu captures of the secondary kernels (no JSON line)."""
    import torch
    import paper_1907_05709_b300 as rfa
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    if name == "batch16":
        cases = ph.batch_members(0, 16, 100, sizes=(96, 128, 160))
        grids = [rfa.Grid.from_case(c, damage=False, cuda_stream=stream.cuda_stream) for c in cases]
        b = rfa.rfa_batch_create([g.handle for g in grids])
        for _ in range(3):
            rfa.rfa_batch_step(b, 8)
        rfa.rfa_batch_destroy(b)
    elif name == "adjoint128":
        case = ph.adjoint_case_128(nsteps=200)
        g = rfa.Grid.from_case(case, damage=False, cuda_stream=stream.cuda_stream)
        g.set_schedule(2, 0)
        g.step(case.nsteps, record=True)
        seed = torch.full(case.labels.shape, 1e-6, dtype=torch.float32, device="cuda")
        for _ in range(2):
            g.backward(seed)
    elif name in ("adjoint256", "adjoint256h"):
        # the same at 256^3 (fields beyond L2): 200 recorded steps, two backward passes;
        # adjoint256h with the conservative (harmonic-mean face) conduction
        case = ph.adjoint_case_256(nsteps=200)
        if name == "adjoint256h":
            case.conduction = "harmonic"
        g = rfa.Grid.from_case(case, damage=False, cuda_stream=stream.cuda_stream)
        if name == "adjoint256":
            g.set_schedule(2, 0)
        g.step(case.nsteps, record=True)
        seed = torch.full(case.labels.shape, 1e-6, dtype=torch.float32, device="cuda")
        for _ in range(2):
            g.backward(seed)
    elif name == "model256":
        # the model options at 256^3: breathing resample, necrosis reduction,
        # conservative step, tissue-state step, 40 iterations of the potential solve
        case = ph.umbrella_case_256(seed=0, nsteps=8)
        g = rfa.Grid.from_case(case, cuda_stream=stream.cuda_stream)
        g.step(8)
        u = torch.from_numpy(ph.breathing_field(case, 1.0)).cuda()
        dst = torch.empty((case.nz, case.ny, case.nx), dtype=torch.float32, device="cuda")
        for _ in range(3):
            rfa.rfa_warp_temperature(g.handle, u, dst, False)
        res = torch.zeros(4, dtype=torch.float64, device="cuda")
        for _ in range(3):
            rfa.rfa_necrosis_reduce_noalloc(g.handle, res, 1.0)
        g.close()
        for cond, perf in (("harmonic", "constant"), ("centre", "tissue_state")):
            c2 = ph.umbrella_case_256(seed=0, nsteps=8)
            c2.conduction, c2.perfusion = cond, perf
            g2 = rfa.Grid.from_case(c2, cuda_stream=stream.cuda_stream)
            g2.step(8)
            g2.close()
        g3 = rfa.Grid(case.nx, case.ny, case.nz, case.h, case.dt, rfa.STATE_F32C, rfa.PARAM_BF16, case.face_bc,
                      case.T_a_C, stream.cuda_stream)
        g3.set_tissue(case.labels, case.table)
        rfa.rfa_place_needle_potential(g3.handle, case.needle, [t.sigma for t in case.table], 40, 1e-30)
        g3.close()
    elif name == "potential256":
        # the potential-solve source at 256^3 with the multigrid preconditioner, to 1e-10
        case = ph.umbrella_case_256(seed=0, nsteps=1)
        g3 = rfa.Grid(case.nx, case.ny, case.nz, case.h, case.dt, rfa.STATE_F32C, rfa.PARAM_BF16, case.face_bc,
                      case.T_a_C, stream.cuda_stream)
        g3.set_tissue(case.labels, case.table)
        rfa.rfa_place_needle_potential(g3.handle, case.needle, [t.sigma for t in case.table], 20000, 1e-10)
        g3.close()
    else:
        raise SystemExit(f"unknown profile case {name}")
    torch.cuda.synchronize()
    return 0


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large512")
    ap.add_argument("--sim-steps", type=int, default=None, help="override time steps per bench step")
    ap.add_argument("--schedule", default="auto", help="auto | plain | tbN | tbNvV")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-secondary", action="store_true", help="skip the adjoint and batched measurements")
    ap.add_argument("--batch-steps", type=int, default=4000)
    ap.add_argument("--profile-case", default=None, help="batch16 | adjoint128 | adjoint256 | adjoint256h | model256 | potential256: short case for ncu")
    args = ap.parse_args(argv)
    if args.schedule == "plain":
        args.schedule = "tb1"
    return args


def main():
    args = parse_args()
    if args.profile_case:
        return profile_case(args.profile_case)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
