"""Benchmark: whole transcranial plans on a synthetic skull (240 x 240 x 200,
dx 0.5 mm, 500 kHz, 1500 FDTD steps, 64 mm / 63 mm focused bowl).

One bench step = one plan = every step of the hot path: property table ->
coefficients, Rayleigh-Sommerfeld source plane, FDTD through the skull with
peak map and 10-cycle FP64 amplitude capture, the water-only FDTD, E_L, and the
BHTE (40 s on at 30 % duty cycle, 80 s off) with T_max and CEM43.  The metric
counts FDTD voxel-steps of both runs per second of whole-plan time.

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun each rank runs its own plans (its own seeded skull and bowl
placement); no data crosses ranks ("weak" scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FDTD Gvoxel-steps/s"
UNIT = "Gvoxel-steps/s"
WORKLOAD = ("synthetic skull {nx}x{ny}x{nz} dx0.5mm 500kHz {steps} steps, bowl 64/63 mm, water run, "
            "BHTE 40s/30%/80s")


def workload(case):
    return WORKLOAD.format(nx=case.nx, ny=case.ny, nz=case.nz, steps=case.n_steps)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="bvf", choices=["bvf", "reference"])
    ap.add_argument("--fdtd-steps", type=int, default=1500)
    ap.add_argument("--grid", default="240,240,200")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--storage", default="f32", choices=["f32", "f16"],
                    help="acoustic state storage of the headline measurement")
    ap.add_argument("--sweep", action="store_true",
                    help="batched planning sweep (64 uneven domains) instead of the plan bench")
    ap.add_argument("--sweep-domains", type=int, default=64)
    ap.add_argument("--sweep-steps", type=int, default=200)
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the scaled-FP16-storage leg reported under mixed_precision")
    ap.add_argument("--no-surrogate", action="store_true",
                    help="skip the surrogate (Fourier neural operator) inference leg")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the 64-domain batched sweep leg")
    ap.add_argument("--no-config3", action="store_true",
                    help="skip the 250 / 700 kHz mixed-precision leg (config3)")
    ap.add_argument("--surrogate", action="store_true",
                    help="run only the surrogate inference on --grid and print its line")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(ms, pg, device="cpu"):
    """Slowest rank's time (ms): the job is as fast as its last rank."""
    if pg is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, steps, units_per_step, ms):
    """Units all ranks processed per second, in billions (each rank runs its
    own plans: weak scaling)."""
    return world * steps * units_per_step / (ms / 1e3) / 1e9


def bench_config(case, storage):
    """The workload as both arms name it (descriptors only, no results)."""
    es = 4 if storage == "f32" else 2
    return {"workload": workload(case), "grid": [case.nx, case.ny, case.nz],
            "fdtd_steps": case.n_steps, "runs_per_step": 2, "n_sls": case.n_sls,
            "n_pml": case.n_pml, "dft_cycles": case.dft_cycles, "storage": storage,
            "l2": "inputs larger than L2 (state %.0f MB per run)"
                  % (case.voxels * es * (9 + 6 * case.n_sls) / 1e6)}


def make_case(args, rank):
    from paper_2301_12727_gb300 import synth
    nx, ny, nz = (int(v) for v in args.grid.split(","))
    return synth.skull_case(nx, ny, nz, dx=0.5e-3, f0=5e5, n_steps=args.fdtd_steps,
                            seed=1234 + rank, dft_cycles=10)


# --------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.flush()
        rows = []
        with open(self.out.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.out.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


KERNEL_SOURCES = ("bvf_acoustic_tma.cu", "bvf_stencil.cuh", "bvf_tma.cuh")
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "fdtd_stress_velocity_skull160.md")


def kernel_source_sha():
    """Hash of every source the TMA FDTD kernels compile from."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2301_12727_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def stress_traffic_per_voxel(window_fraction):
    """Measured DRAM bytes per voxel of the stress kernel, averaged over launches
    inside and outside the DFT window like the algorithmic bytes, from the
    committed ncu summary; None unless that summary was taken on the current
    kernel sources and holds both figures."""
    try:
        text = open(PROFILE_SUMMARY).read()
    except OSError:
        return None
    sha = kernel_source_sha()
    vals = {}
    for line in text.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256_16") != sha:
        return None
    try:
        win = float(vals["dram_bytes_per_voxel_dft_window"])
        out = float(vals["dram_bytes_per_voxel_outside_window"])
    except (KeyError, ValueError):
        return None
    return window_fraction * win + (1.0 - window_fraction) * out


# --------------------------------------------------------------------------
def cpu_baseline_oracle(case, budget_s=15.0, max_steps=200):
    """The FP64 oracle as it stands, on this host's cores, over a bounded
    sample of the same workload (the first FDTD steps of the skull run)."""
    import numpy as np
    import oracle
    oracle.build()
    b = case.bowl
    plane = oracle.rs_plane(b["aperture"], b["roc"], b["apex"], b["dir"], case.nx, case.ny,
                            case.dx, case.k_src * case.dx, case.f0, case.c0, b["p0"])
    A = oracle.Acoustic(case.nx, case.ny, case.nz, case.dx, case.dt, case.index, case.materials,
                        case.f0, qc=case.qc, n_sls=case.n_sls, n_pml=case.n_pml, pml_R=case.pml_R)
    A.set_source(plane, case.k_src, case.c0, oracle.ENV_RAMP_CW)
    # two probes separate the per-call copy overhead from the per-step cost
    t0 = time.perf_counter()
    assert A.run(1, peak_from=0) == 0
    t1 = time.perf_counter()
    assert A.run(3, peak_from=0) == 0
    t2 = time.perf_counter()
    per_step = max((t2 - t1) - (t1 - t0), 1e-3) / 2.0
    overhead = max((t1 - t0) - per_step, 0.0)
    n = max(2, min(max_steps, int((budget_s - overhead) / per_step)))
    t0 = time.perf_counter()
    assert A.run(n, peak_from=0) == 0
    t = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": case.voxels * n / t / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d FDTD steps (of %d) of the skull run on the full %dx%dx%d grid, "
                      "FP64, %.1f s" % (n, case.n_steps, case.nx, case.ny, case.nz, t),
            "seconds": t, "steps": n}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    case = make_case(args, 0)
    times = []
    base = None
    for it in range(args.warmup + args.steps):
        r = cpu_baseline_oracle(case, budget_s=8.0, max_steps=100)
        if it >= args.warmup:
            times.append(r)
        base = r
    vox = sum(r["steps"] for r in times) * case.voxels
    sec = sum(r["seconds"] for r in times)
    value = vox / sec / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sec / max(len(times), 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(case, args.storage),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": base["cores"],
                             "kind": "oracle", "sample": base["sample"] +
                             "; each bench step: %d FDTD steps on the full grid"
                             % times[-1]["steps"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# Surrogate network: 4 Fourier layers, width 32, 12 modes, projection width
# 128, run on the plan's grid.
FNO_DIMS = dict(c_in=8, width=32, modes=12, n_layers=4, hidden=128, c_out=2)


def run_surrogate(args):
    """The surrogate leg alone (one GPU): inference time on --grid."""
    import torch
    import __graft_entry__
    torch.cuda.set_device(0)
    __graft_entry__.build()
    case = make_case(args, 0)
    leg = surrogate_leg(case, args.steps, args.warmup, None, None,
                        cpu_baseline=not args.no_cpu_baseline)
    print(json.dumps({"metric": "surrogate inference ms", "value": leg["ms_per_inference"],
                      "unit": "ms", "higher_is_better": False, "surrogate": leg}), flush=True)
    return 0


def graph_ms(fn, reps):
    """Milliseconds per replay of fn recorded once in a CUDA graph (fn's
    launches on torch's current stream; one warm call on a side stream first)."""
    import torch
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fn()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def surrogate_leg(case, steps, warmup, ms_plan, ms_fdtd, cpu_baseline=True):
    """Inference time of the surrogate on the plan's feature volume (seeded
    untrained weights: the time does not depend on their values), its stage
    split and its HBM roofline, for the TF32 path (call by call and replayed
    from a CUDA graph) and the BF16 path (bvf_fno_bf16_forward, from a graph);
    with cpu_baseline, the FP64 oracle timed on a 48^3 sample as the
    surrogate's CPU baseline."""
    import time
    import numpy as np
    import torch
    from paper_2301_12727_gb300 import bvf, fno, synth
    nx, ny, nz = case.nx, case.ny, case.nz
    net = fno.Surrogate(FNO_DIMS, synth.fno_weights(FNO_DIMS, 2301))
    idx = torch.from_numpy(case.index).cuda()
    src = bvf.rs_plane(dict(case.bowl), nx, ny, case.dx, case.k_src * case.dx, case.f0)
    feats = torch.empty((8, nz, ny, nx), dtype=torch.float32, device="cuda")
    out = torch.empty((FNO_DIMS["c_out"], nz, ny, nx), dtype=torch.float32, device="cuda")
    water = synth.water_row(case.f0)

    def one():
        fno.bvf_fno_features(idx, case.materials, water, case.f0, case.k_src, src,
                             case.bowl["p0"], feats)
        net(feats, out)

    for _ in range(max(3, warmup)):
        one()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k = max(5, steps)
    e0.record()
    for _ in range(k):
        one()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / k
    net.timing(True)
    one()
    torch.cuda.synchronize()
    stages = net.stage_times()
    net.timing(False)
    k = max(5, steps)
    ms_graph = graph_ms(one, k)
    net.close()
    bf = fno.Bf16Net(FNO_DIMS, synth.fno_weights(FNO_DIMS, 2301), (nx, ny, nz), max_batch=1)
    fb, ob = feats[None], out[None]

    def one_bf16():
        fno.bvf_fno_features(idx, case.materials, water, case.f0, case.k_src, src,
                             case.bowl["p0"], feats)
        bf.forward(fb, ob)

    ms_bf16 = graph_ms(one_bf16, k)
    bf.close()
    N = case.voxels
    d = FNO_DIMS
    # algorithmic bytes per inference: the features read by the lift, every
    # activation volume written once and read once (lift, then each layer;
    # the forward x transform is fused into the pass that writes a volume),
    # the output written once; spectra and weights are below 2 %
    act = 4.0 * d["width"] * N
    bytes_inf = 4.0 * N * (d["c_in"] + d["c_out"]) + act * (2 * d["n_layers"] + 2)
    peak, peak_kind = measured_peak_hbm()
    base = None
    if cpu_baseline:
        # the CPU baseline: the FP64 oracle on a 48^3 sample of the same network
        from oracle import fno as ofno
        rng = np.random.default_rng(7)
        a_small = rng.standard_normal((8, 48, 48, 48))
        w = synth.fno_weights(FNO_DIMS, 2301).astype(np.float64)
        t0 = time.perf_counter()
        ofno.forward(a_small, w, **FNO_DIMS)
        t_or = time.perf_counter() - t0
        base = {"value": 48 ** 3 / t_or, "unit": "voxels/s", "kind": "oracle", "cores": 1,
                "sample": "one 48^3 inference, FP64 numpy"}
    return {"model": "Fourier neural operator, 4 layers, width 32, 12 modes, projection 128",
            "weights": "seeded, untrained (inference time does not depend on the values)",
            "grid": [nx, ny, nz], "ms_per_inference": ms, "voxels_per_s": N / (ms / 1e3),
            "speedup_vs_plan": ms_plan / ms if ms_plan else None,
            "speedup_vs_plan_fdtd": ms_fdtd / ms if ms_fdtd else None,
            "graph": {"ms_per_inference": ms_graph,
                      "speedup_vs_plan": ms_plan / ms_graph if ms_plan else None},
            "bf16": {"path": "bvf_fno_bf16_forward: every contraction a tcgen05 kind::f16 BF16 "
                             "product with FP32 accumulation, replayed from a CUDA graph",
                     "ms_per_inference": ms_bf16,
                     "speedup_vs_plan": ms_plan / ms_bf16 if ms_plan else None,
                     "speedup_vs_plan_fdtd": ms_fdtd / ms_bf16 if ms_fdtd else None},
            "stages_ms": stages,
            "tensor_core": "layer output (k_row_tc), forward x transform (k_dftx_tc) and "
                           "projection (k_project_tc): tcgen05.mma kind::tf32 into TMEM, "
                           "all with the three-product FP32 split",
            "roofline": {"bound": "hbm", "achieved": bytes_inf / (ms / 1e3) / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": bytes_inf / (ms / 1e3) / 1e9 / peak,
                         "peak_kind": peak_kind, "algorithmic_bytes": bytes_inf},
            "cpu_baseline": base}


def _config3_case(f0):
    from paper_2301_12727_gb300 import synth
    return synth.config3_case(f0, *synth.CONFIG3_GRIDS[f0])


def config3_leg(cases):
    """Mixed-precision workload family (9 points per wavelength, 250 kHz on
    128 x 128 x 108 and 700 kHz on 360 x 360 x 300, transit + 10 cycles, then
    the BHTE): one warm-up and one timed plan per storage; plan throughput,
    FDTD kernel time, the FP16-over-FP32 speed-ups, and every output's
    difference from the FP64 oracle's stored results (planes through the
    focus, tests/golden/config3_*.npz, written by the oracle alone)."""
    import torch
    from paper_2301_12727_gb300 import plan as planmod, synth
    from tests.golden import config3 as ref3
    out = {}
    for f0 in sorted(cases):
        c = cases[f0]
        reg = synth.thermal_regime(c.dx, c.materials)
        regime = planmod.ThermalRegime(dt=reg["dt"], duty=reg["duty"])
        idx = torch.from_numpy(c.index).cuda()
        try:
            meta, ref = ref3.load(f0)
        except OSError:
            meta = ref = None          # the oracle's result file is not there
        vs = 2 * c.n_steps * c.voxels
        rec = {"grid": [c.nx, c.ny, c.nz], "dx_mm": c.dx * 1e3, "fdtd_steps": c.n_steps,
               "dft_cycles": c.dft_cycles, "thermal_dt_s": reg["dt"],
               "voxel_steps_per_plan": vs}
        for storage in ("f32", "f16"):
            pl = planmod.Planner(c, storage=storage)
            pl.run(idx, c.materials, c.bowl, regime)
            torch.cuda.synchronize()
            pl.kernel_timing(True)
            stream = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = pl.run(idx, c.materials, c.bowl, regime)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            kt = pl.kernel_times()
            pl.kernel_timing(False)
            amp, ph = pl.skull.amp_phase()
            maps = dict(p=pl.skull.pressure(), peak=r.peak, amp=amp, phase=ph, Tmax=r.Tmax,
                        cem=r.cem43)
            errs = (ref3.errors(meta, ref, maps, dict(EL=r.EL, TS=r.TS, z_m=r.z_m))
                    if meta is not None else None)
            rec[storage] = {"value": vs / (ms / 1e3) / 1e9, "unit": UNIT, "ms_per_plan": ms,
                            "fdtd_kernel_ms": kt["stress_ms"] + kt["velocity_ms"],
                            "errors_vs_fp64_oracle": errs}
            del maps, amp, ph, r
            pl.close()
        rec["speedup_f16_vs_f32"] = rec["f32"]["ms_per_plan"] / rec["f16"]["ms_per_plan"]
        rec["fdtd_kernel_speedup_f16_vs_f32"] = (rec["f32"]["fdtd_kernel_ms"]
                                                 / rec["f16"]["fdtd_kernel_ms"])
        out["%dkHz" % int(round(f0 / 1e3))] = rec
        del idx
        torch.cuda.empty_cache()
    out["oracle_reference"] = ("FP64 oracle, whole runs on the full grids, stored as planes "
                               "through the focus (tests/golden/make_config3_reference.py)")
    return out


def run_bvf(args):
    import torch
    rank, world, local = dist_env()
    c3_future = None
    if rank == 0 and not args.no_config3:
        # the config-3 phantoms are generated on the host cores while the
        # headline is timed (a spawned process: no CUDA state is inherited)
        import concurrent.futures as cf
        import multiprocessing as mp
        c3_pool = cf.ProcessPoolExecutor(max_workers=2, mp_context=mp.get_context("spawn"))
        c3_future = {f0: c3_pool.submit(_config3_case, f0) for f0 in (250e3, 700e3)}
    sweep_futs = None
    if rank == 0 and not args.no_sweep:
        import concurrent.futures as cf
        import multiprocessing as mp
        sw_pool = cf.ProcessPoolExecutor(max_workers=min(12, os.cpu_count() or 1),
                                         mp_context=mp.get_context("spawn"))
        sweep_futs = make_sweep_cases(args.sweep_domains, args.sweep_steps, pool=sw_pool)
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if pg:
        pg.barrier()
    from paper_2301_12727_gb300 import plan as planmod
    case = make_case(args, rank)
    planner = planmod.Planner(case, storage=args.storage)
    idx_dev = torch.from_numpy(case.index).cuda()
    bowl = case.bowl
    mats = case.materials

    def barrier():
        torch.cuda.synchronize()
        if pg:
            pg.barrier()

    for _ in range(args.warmup):
        res = planner.run(idx_dev, mats, bowl)
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    l0 = planner.launches()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        res = planner.run(idx_dev, mats, bowl)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    clocks = sampler.stop()
    launches = planner.launches() - l0
    # kernel roofline pass: the same plans with the water run after the skull
    # run (not beside it), so that the CUDA events recorded around every
    # launch on its stream bracket that kernel alone
    roof_plans = 2
    planner.kernel_timing(True)
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    for _ in range(roof_plans):
        planner.run(idx_dev, mats, bowl, serial=True)
    r1.record(stream)
    torch.cuda.synchronize()
    ms_serial_plan = r0.elapsed_time(r1) / roof_plans
    kt = planner.kernel_times()
    planner.kernel_timing(False)
    # thermal + auxiliary kernels are counted through the context counters;
    # the transmission reductions (3 kernels) and RS (1) per plan are context-free
    launches += args.steps * 4
    ms = max_over_ranks(ms, pg, "cuda")
    vox_per_plan = res.voxel_steps
    value = whole_job_rate(world, args.steps, vox_per_plan, ms)

    # ---- end to end through the C-ABI call with host buffers (bvf_plan_host:
    # the index copied in from pinned host memory and the peak, T_max and
    # CEM43 maps copied out inside the call, every plan)
    e2e = None
    if not args.no_e2e:
        idx_host = torch.from_numpy(case.index).pin_memory()
        out_peak = torch.empty(case.index.shape, dtype=torch.float32).pin_memory()
        out_tmax = torch.empty(case.index.shape, dtype=torch.float32).pin_memory()
        out_cem = torch.empty(case.index.shape, dtype=torch.float64).pin_memory()
        planner.run_host(idx_host, mats, bowl, out_peak, out_tmax, out_cem)      # staging
        barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            planner.run_host(idx_host, mats, bowl, out_peak, out_tmax, out_cem)
        f1.record(stream)
        barrier()
        ms_e2e = max_over_ranks(f0.elapsed_time(f1), pg, "cuda")
        e2e = {"value": whole_job_rate(world, args.steps, vox_per_plan, ms_e2e), "unit": UNIT,
               "h2d_bytes_per_step": int(idx_host.numel()),
               "d2h_bytes_per_step": int(out_peak.numel() * 4 + out_tmax.numel() * 4
                                         + out_cem.numel() * 8)}

    # ---- the same plans with the other state storage: throughput and the
    # differences of every plan output from the headline run
    mixed = None
    if not args.no_mixed:
        other = "f16" if args.storage == "f32" else "f32"
        pl2 = planmod.Planner(case, storage=other)
        for _ in range(max(1, args.warmup)):
            r2 = pl2.run(idx_dev, mats, bowl)
        barrier()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(args.steps):
            r2 = pl2.run(idx_dev, mats, bowl)
        g1.record(stream)
        barrier()
        ms2 = max_over_ranks(g0.elapsed_time(g1), pg, "cuda")
        ref, tst = (res, r2) if other == "f16" else (r2, res)
        pk32 = float(ref.peak.max())
        am32 = float(ref.amp.max())
        mixed = {"storage": "f16", "arithmetic": "f32",
                 "value": whole_job_rate(world, args.steps, vox_per_plan,
                                         ms2 if other == "f16" else ms),
                 "speedup_vs_f32": (ms / ms2) if other == "f16" else (ms2 / ms),
                 "errors_vs_f32": {
                     "focal_peak_rel": abs(float(tst.peak.max()) - pk32) / pk32,
                     "peak_max_abs_rel": float((tst.peak - ref.peak).abs().max()) / pk32,
                     "amp_max_abs_rel": float((tst.amp - ref.amp).abs().max()) / am32,
                     "EL_rel": abs(tst.EL - ref.EL) / ref.EL,
                     "Tmax_max_abs_C": float((tst.Tmax - ref.Tmax).abs().max()),
                     "cem43_at_max_rel": abs(float(tst.cem43.max()) - float(ref.cem43.max()))
                                         / max(float(ref.cem43.max()), 1e-300)}}
        pl2.close()

    config3 = None
    if c3_future is not None:
        config3 = config3_leg({f0: fut.result() for f0, fut in c3_future.items()})
        c3_pool.shutdown()

    sweep = None
    if sweep_futs is not None:
        sweep = sweep_leg([f.result() for f in sweep_futs], 2, 1)
        sw_pool.shutdown()

    surrogate = None
    if not args.no_surrogate and rank == 0:
        surrogate = surrogate_leg(case, args.steps, args.warmup, ms / args.steps,
                                  (kt["stress_ms"] + kt["velocity_ms"]) / roof_plans,
                                  cpu_baseline=not args.no_cpu_baseline)

    # ---- roofline of the dominant kernel (stress + memory variables)
    N = case.voxels
    n_runs = 2 * roof_plans          # FDTD runs of the roofline pass
    es = 4.0 if args.storage == "f32" else 2.0      # bytes per state element
    # stress: read 3 v, read + write 6 sigma and 12 memory variables, index
    # byte, FP32 peak read + write (+ FP64 C, S read + write in the DFT window);
    # velocity: read 6 sigma + 3 v, write 3 v, index byte
    b_str, b_vel = 39.0 * es + 9.0, 12.0 * es + 1.0
    stress_bytes = N * (b_str * case.n_steps + 32.0 * case.dft_steps) * n_runs
    achieved = stress_bytes / (kt["stress_ms"] / 1e3) / 1e9
    peak, peak_kind = measured_peak_hbm()
    tr = stress_traffic_per_voxel(case.dft_steps / case.n_steps) if args.storage == "f32" else None
    vel_bytes = N * b_vel * case.n_steps * n_runs
    # whole FDTD step: the two-kernel design's bytes, and the minimum one
    # read + write of the 21-word state plus index and peak
    fdtd_s = (kt["stress_ms"] + kt["velocity_ms"]) / 1e3
    design = (stress_bytes + vel_bytes) / fdtd_s / 1e9
    minimum = N * ((42.0 * es + 9.0) * case.n_steps + 32.0 * case.dft_steps) * n_runs / fdtd_s / 1e9
    roofline = {"bound": "hbm", "kernel": "k_stress_tma<2> (stress + SLS memory + source + capture)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_kind": peak_kind,
                "traffic": (tr * N if tr is not None else None),
                "algorithmic_bytes_per_launch": stress_bytes / kt["stress_launches"],
                "avg_launch_ms": kt["stress_ms"] / kt["stress_launches"],
                "velocity_kernel": {"achieved": vel_bytes / (kt["velocity_ms"] / 1e3) / 1e9,
                                    "frac": vel_bytes / (kt["velocity_ms"] / 1e3) / 1e9 / peak,
                                    "avg_launch_ms": kt["velocity_ms"] / kt["velocity_launches"]},
                "fdtd_step": {"design_bytes_per_voxel": b_str + b_vel,
                              "min_bytes_per_voxel": 42.0 * es + 9.0,
                              "achieved_design": design, "frac_design": design / peak,
                              "achieved_min": minimum, "frac_min": minimum / peak},
                "fdtd_share_of_serial_plan": (kt["stress_ms"] + kt["velocity_ms"]) / roof_plans
                                             / ms_serial_plan,
                "timing": "per-launch CUDA events on the launching stream in a separate pass of "
                          "%d plans with the two FDTD runs serialised (the headline plans run "
                          "the water companion concurrently and record no per-launch events)"
                          % roof_plans,
                "plan_ms_serial": ms_serial_plan, "plan_ms_concurrent": ms / args.steps,
                "concurrency_gain": ms_serial_plan / (ms / args.steps)}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.storage == "f32" else "f16 storage, f32 arithmetic",
            "data": "synthetic",
            "config": bench_config(case, args.storage),
            "results": {"EL": res.EL, "TS": res.TS, "z_m": res.z_m},
            "roofline": roofline, "gpu_launches": int(launches), "e2e": e2e, "clocks": clocks,
            "mixed_precision": mixed, "config3": config3, "sweep": sweep, "surrogate": surrogate}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_oracle(case)
    if rank == 0:
        print(json.dumps(line), flush=True)
    planner.close()
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


# --------------------------------------------------------------------------
def _sweep_domain(spec_steps):
    from paper_2301_12727_gb300 import synth
    spec, n_steps = spec_steps
    return synth.sweep_case(spec, n_steps=n_steps)


def sweep_leg(cases, steps, warmup):
    """Batched planning sweep over `cases` (seeded domains of uneven size,
    frequency, tilt and skull): the same FDTD runs of every domain timed
    (CUDA events, min over `steps` repetitions after `warmup`) in six modes:
    one after another (with the default and with the tuned tiles),
    per-domain launches on 8 streams, the sweep recorded as one CUDA graph of
    per-domain launches on 8 branches (with the default tiles, and with the
    tile of the graph-mode autotuner), and the persistent work-list kernels
    replayed from a graph; the sequential runs are timed again with the
    tiles of the per-domain autotuner.  Every mode gives the sequential results bit for
    bit (checked on the peak maps)."""
    import torch
    from paper_2301_12727_gb300 import bvf
    solvers = []
    for c in cases:
        s = bvf.Solver(c.nx, c.ny, c.nz, c.dx, c.dt, c.f0, n_sls=2, n_pml=c.n_pml)
        s.set_materials(c.index, c.materials)
        s.set_source(bvf.rs_plane(c.bowl, c.nx, c.ny, c.dx, c.k_src * c.dx, c.f0), c.k_src, c.c0,
                     c.envelope)
        solvers.append(s)
    vox = sum(c.voxels for c in cases)
    n = cases[0].n_steps
    caps = [(0, 0, 0)] * len(solvers)
    stream = torch.cuda.current_stream()
    batch = bvf.Batch(solvers)

    def timed(fn):
        for s in solvers:
            s.reset()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    def sequential():
        for s in solvers:
            s.run(n, peak_from=0)

    def streams():
        batch.run_streams(n, caps=caps, n_streams=8)

    def graph():
        batch.run_graph(n, caps=caps, n_branches=8)

    def best(fn):
        for _ in range(max(1, warmup)):
            timed(fn)
        return min(timed(fn) for _ in range(max(1, steps)))

    ms_seq = best(sequential)
    ref = [s.peak() for s in solvers]
    ms_str = best(streams)
    same = all(bool(torch.equal(a, s.peak())) for a, s in zip(ref, solvers))
    ms_graph_default = best(graph)
    same = same and all(bool(torch.equal(a, s.peak())) for a, s in zip(ref, solvers))
    tuned = batch.tune_domains(trial_steps=10)
    ms_seq_tuned = best(sequential)
    gtile, _ = batch.tune_graph(trial_steps=20, n_branches=8)
    ms_graph = best(graph)
    same = same and all(bool(torch.equal(a, s.peak())) for a, s in zip(ref, solvers))
    best_kc, _ = batch.tune(trial_steps=20, candidates=(6, 8, 10, 13, 16, 24))
    ms_pers = best(lambda: batch.run(n, caps=caps, kchunk=best_kc, graph_steps=50))
    same = same and all(bool(torch.equal(a, s.peak())) for a, s in zip(ref, solvers))
    rate = lambda ms: vox * n / (ms / 1e3) / 1e9
    out = {"domains": len(cases), "voxels_total": vox, "fdtd_steps_each": n,
           "sequential": {"value": rate(ms_seq), "ms": ms_seq},
           "sequential_tuned_tiles": {"value": rate(ms_seq_tuned), "ms": ms_seq_tuned,
                                      "tiles_chosen": {"stress %d / velocity %d rows, z %d" % t:
                                                       sum(1 for x in tuned if x == t)
                                                       for t in sorted(set(tuned))}},
           "streams_8": {"value": rate(ms_str), "ms": ms_str,
                         "speedup_vs_sequential": ms_seq / ms_str},
           "graph_8_branches": {"value": rate(ms_graph_default), "ms": ms_graph_default,
                                "speedup_vs_sequential": ms_seq / ms_graph_default, "launches": 1,
                                "tiles": "defaults (stress 8, velocity 16 rows)"},
           "graph_8_branches_tuned": {"value": rate(ms_graph), "ms": ms_graph,
                                      "speedup_vs_sequential": ms_seq / ms_graph,
                                      "speedup_vs_sequential_tuned": ms_seq_tuned / ms_graph,
                                      "launches": 1,
                                      "tile": "stress %d / velocity %d rows, z %d" % gtile},
           "persistent_graph": {"value": rate(ms_pers), "ms": ms_pers,
                                "speedup_vs_sequential": ms_seq / ms_pers, "z_chunk": best_kc},
           "unit": UNIT, "results_equal_sequential": bool(same)}
    batch.close()
    for s in solvers:
        s.close()
    return out


def make_sweep_cases(n_domains, n_steps, pool=None):
    """Seeded sweep domains (96..200 cells per axis, 250/500/700 kHz at 6 points
    per wavelength, tilt +-15 deg) generated on the host cores by spawned
    processes (no CUDA state is inherited)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    from paper_2301_12727_gb300 import synth
    specs = synth.sweep_specs(n=n_domains, seed=4321)
    own = pool is None
    if own:
        pool = cf.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1),
                                      mp_context=mp.get_context("spawn"))
    futs = [pool.submit(_sweep_domain, (sp, n_steps)) for sp in specs]
    if own:
        out = [f.result() for f in futs]
        pool.shutdown()
        return out
    return futs


def run_sweep(args):
    """The batched planning sweep alone, as its own JSON line."""
    cases = make_sweep_cases(args.sweep_domains, args.sweep_steps)
    import torch  # noqa: F401  (CUDA is first touched after the spawned generation)
    import __graft_entry__
    __graft_entry__.build()
    leg = sweep_leg(cases, args.steps, args.warmup)
    g = leg["graph_8_branches_tuned"]
    line = {"metric": "sweep Gvoxel-steps/s", "value": g["value"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": g["ms"] / leg["fdtd_steps_each"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "planning sweep: %d skull domains, 96..200 cells per axis, "
                                   "250/500/700 kHz, tilt +-15 deg, %d steps each"
                                   % (leg["domains"], leg["fdtd_steps_each"]),
                       "mode": "one CUDA graph of per-domain launches on 8 branches"},
            "sweep": leg, "gpu_launches": 2 * leg["fdtd_steps_each"] * leg["domains"]}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep:
        return run_sweep(args)
    if args.surrogate:
        return run_surrogate(args)
    return run_bvf(args)


if __name__ == "__main__":
    sys.exit(main())
