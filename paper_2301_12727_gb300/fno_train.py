"""Training of the surrogate on fields the FDTD of this library computes,
with the library's hand-written BF16 tensor-core kernels (offline tool).

Data: seeded synthetic skulls with tilted bowls (synth.sweep_case) on one
grid; each placement runs one plan of the library (bvf_plan through
plan.Planner: the skull FDTD and its water companion, E_L on the plane of
maximal water intensity; no thermal step).  Targets: output channel 0 is the
FP64 skull-run amplitude over the capture window divided by the bowl's
surface pressure, channel 1's spatial mean is the transmission efficiency
E_L.  Inputs: the 8-channel feature volume of bvf_fno_features.

Training: bvf_fno_bf16_adam (forward, loss, backward and the Adam step all in
the library's BF16 kernels; no autograd, no framework FFT), one-cycle
learning rate.  Evaluation on held-out skulls with the trained weights,
through both CUDA inference paths (TF32 three-product and BF16): relative L2
error of the field, error of the focal amplitude (the field maximum),
distance between the predicted and the FDTD focus, and the E_L error; then
the time of one plan of the library on the same grid against one surrogate
inference (feature volume + network), i.e. the speed-up on the workload the
accuracy is measured on.

    python -m paper_2301_12727_gb300.fno_train --train 1000 --test 100 --epochs 20
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

FEATURES = 8


def make_dataset(n, seed, grid, dx, f0, dft_cycles=6):
    """n placements on one grid: features [n, 8, nz, ny, nx], amplitude / p0
    [n, nz, ny, nx] (float32 CUDA tensors) and E_L [n] (float32)."""
    import torch
    from . import bvf, fno, plan, synth
    nx, ny, nz = grid
    feats = torch.empty((n, FEATURES, nz, ny, nx), dtype=torch.float32, device="cuda")
    amps = torch.empty((n, nz, ny, nx), dtype=torch.float32, device="cuda")
    els = torch.empty(n, dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(seed)
    planner, dt0 = None, None
    no_heat = plan.ThermalRegime(t_on=0.0, t_off=0.0)
    for i in range(n):
        spec = dict(nx=nx, ny=ny, nz=nz, f0=f0, dx=dx, tilt_deg=float(rng.uniform(-15.0, 15.0)),
                    seed=int(seed) * 100000 + i)
        c = synth.sweep_case(spec, dft_cycles=dft_cycles)
        if planner is None:
            planner, dt0 = plan.Planner(c), c.dt
        if c.dt != dt0:
            raise RuntimeError("time step differs between cases of one grid")
        planner.case = c
        idx = torch.from_numpy(c.index).cuda()
        r = planner.run(idx, c.materials, c.bowl, no_heat)
        amps[i] = (r.amp / c.bowl["p0"]).float()
        els[i] = r.EL
        src = bvf.rs_plane(c.bowl, nx, ny, dx, c.k_src * dx, f0)
        fno.bvf_fno_features(idx, c.materials, synth.water_row(f0), f0, c.k_src, src,
                             c.bowl["p0"], feats[i])
    torch.cuda.synchronize()
    planner.close()
    return feats, amps, els


def initial_weights(d, seed):
    """Seeded weights (synth.fno_weights) with the spectral blocks scaled down
    by the width once more (R ~ 1/width^2), which keeps the first steps stable."""
    from . import synth
    w = synth.fno_weights(d, seed).astype(np.float64)
    W, m, ci = d["width"], d["modes"], d["c_in"]
    pos = W * ci + W
    nR = (2 * m) * (2 * m) * m * W * W * 2
    for _ in range(d["n_layers"]):
        w[pos:pos + nR] /= W
        pos += nR + W * W + W
    return w.astype(np.float32)


def one_cycle(step, total, lr_max, warm=0.3):
    """Learning rate: linear warm-up over the first 30 %, then cosine decay."""
    if step < warm * total:
        return lr_max * (0.04 + 0.96 * step / (warm * total))
    t = (step - warm * total) / max(1.0, (1.0 - warm) * total)
    return lr_max * (0.02 + 0.98 * 0.5 * (1.0 + math.cos(math.pi * t)))


def focal_metrics(pred, true, dx):
    """Relative L2 field error, focal amplitude error and focus distance (m)."""
    import torch
    rl2 = float(torch.linalg.vector_norm(pred - true) / torch.linalg.vector_norm(true))
    pt, pp = float(true.max()), float(pred.max())
    it = np.array(np.unravel_index(int(torch.argmax(true)), true.shape[-3:]))
    ip = np.array(np.unravel_index(int(torch.argmax(pred)), pred.shape[-3:]))
    return rl2, abs(pp - pt) / pt, float(np.linalg.norm((ip - it) * dx))


def time_plan_vs_surrogate(grid, dx, f0, d, weights, seed, reps=5):
    """Milliseconds of one plan of the library (both FDTD runs, E_L, the 40 s /
    30 % / 80 s BHTE), of the same plan without the thermal step, and of one
    surrogate inference (features + network) on the same placement: TF32 and
    BF16 paths launched call by call, and the TF32 path replayed from a
    recorded CUDA graph (one launch, as a planning service would repeat it)."""
    import torch
    from . import bvf, fno, plan, synth
    nx, ny, nz = grid
    spec = dict(nx=nx, ny=ny, nz=nz, f0=f0, dx=dx, tilt_deg=5.0, seed=seed)
    c = synth.sweep_case(spec, dft_cycles=6)
    pl = plan.Planner(c)
    idx = torch.from_numpy(c.index).cuda()

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_plan = timed(lambda: pl.run(idx, c.materials, c.bowl))
    ms_fdtd = timed(lambda: pl.run(idx, c.materials, c.bowl, plan.ThermalRegime(t_on=0.0, t_off=0.0)))
    pl.close()
    src = bvf.rs_plane(c.bowl, nx, ny, dx, c.k_src * dx, f0)
    feats = torch.empty((FEATURES, nz, ny, nx), dtype=torch.float32, device="cuda")
    out = torch.empty((d["c_out"], nz, ny, nx), dtype=torch.float32, device="cuda")
    tf32 = fno.Surrogate(d, weights)
    bf = fno.Bf16Net(d, weights, grid, max_batch=1)

    def feat():
        fno.bvf_fno_features(idx, c.materials, synth.water_row(f0), f0, c.k_src, src,
                             c.bowl["p0"], feats)

    def infer():
        feat()
        tf32(feats, out)

    def infer_bf16():
        feat()
        bf.forward(feats[None], out[None])

    def graphed(fn):
        # fn recorded once in a CUDA graph (after a warm call on a side stream)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            fn()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        return g

    ms_tf32 = timed(infer)
    ms_bf16 = timed(infer_bf16)
    g32, g16 = graphed(infer), graphed(infer_bf16)
    ms_graph = timed(g32.replay)
    ms_graph16 = timed(g16.replay)
    tf32.close()
    bf.close()
    return dict(plan=ms_plan, plan_without_bhte=ms_fdtd, surrogate_tf32=ms_tf32,
                surrogate_tf32_graph=ms_graph, surrogate_bf16=ms_bf16,
                surrogate_bf16_graph=ms_graph16)


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=1000)
    ap.add_argument("--test", type=int, default=100)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--el-weight", type=float, default=10.0)
    ap.add_argument("--grid", default="64,64,96")
    ap.add_argument("--dx", type=float, default=1e-3)
    ap.add_argument("--f0", type=float, default=2.5e5)
    ap.add_argument("--width", type=int, default=32)
    ap.add_argument("--modes", type=int, default=12)
    ap.add_argument("--layers", type=int, default=4)
    ap.add_argument("--hidden", type=int, default=128)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--save", default="", help="write the trained blob (float32) to this .npy")
    args = ap.parse_args(argv)
    from . import build as _b
    _b.build()
    from . import fno
    grid = tuple(int(v) for v in args.grid.split(","))
    d = dict(c_in=FEATURES, width=args.width, modes=args.modes, n_layers=args.layers,
             hidden=args.hidden, c_out=2)
    t0 = time.time()
    xtr, ytr, etr = make_dataset(args.train, args.seed, grid, args.dx, args.f0)
    xte, yte, ete = make_dataset(args.test, args.seed + 1, grid, args.dx, args.f0)
    t_data = time.time() - t0

    net = fno.Bf16Net(d, initial_weights(d, args.seed), grid, max_batch=args.batch)
    steps_per_epoch = max(1, args.train // args.batch)
    total = args.epochs * steps_per_epoch
    gen = torch.Generator(device="cpu").manual_seed(args.seed)
    t1 = time.time()
    hist, step = [], 0
    for ep in range(args.epochs):
        perm = torch.randperm(args.train, generator=gen)
        run = 0.0
        for k in range(steps_per_epoch):
            sel = perm[k * args.batch:(k + 1) * args.batch].cuda()
            x, y, e = xtr[sel].contiguous(), ytr[sel].contiguous(), etr[sel].contiguous()
            run += net.adam(x, y, one_cycle(step, total, args.lr), e, args.el_weight)
            step += 1
        hist.append(run / steps_per_epoch)
    net.synchronize()
    t_train = time.time() - t1
    w = net.weights()
    net.close()
    if args.save:
        np.save(args.save, w)

    # held-out skulls through both CUDA inference paths with the trained weights
    tf32 = fno.Surrogate(d, w)
    bf = fno.Bf16Net(d, w, grid, max_batch=1)
    rows, el_err, agree = [], [], 0.0
    with torch.no_grad():
        for i in range(args.test):
            o32 = tf32(xte[i].contiguous())
            o16 = bf.forward(xte[i:i + 1].contiguous())[0]
            agree = max(agree, float((o32[0] - o16[0]).abs().max() / o32[0].abs().max()))
            r32 = focal_metrics(o32[0], yte[i], args.dx)
            r16 = focal_metrics(o16[0], yte[i], args.dx)
            el32 = fno.bvf_fno_mean(o32[1].contiguous())
            el16 = fno.bvf_fno_mean(o16[1].contiguous())
            rows.append(r32 + r16)
            el_err.append((abs(el32 - float(ete[i])) / float(ete[i]),
                           abs(el16 - float(ete[i])) / float(ete[i])))
    tf32.close()
    bf.close()
    rows, el_err = np.array(rows), np.array(el_err)
    # the accuracy figures are printed first, so that a failure of the timing
    # leg does not lose them
    print(json.dumps({"held_out_focal_amp_err_median_tf32": float(np.median(rows[:, 1])),
                      "train_loss_first_last": [hist[0], hist[-1]]}), flush=True)
    tm = time_plan_vs_surrogate(grid, args.dx, args.f0, d, w, 999)
    q = lambda a, p: float(np.quantile(a, p))
    tr_max = ytr.flatten(1).max(dim=1).values
    res = {"grid": list(grid), "dx_m": args.dx, "f0_hz": args.f0, "dims": d,
           "training": "bvf_fno_bf16_adam: BF16 tensor-core forward and backward, FP32 master "
                       "weights, Adam, one-cycle lr %.1e, batch %d" % (args.lr, args.batch),
           "train_focal_range_p0": [float(tr_max.min()), float(tr_max.max())],
           "train_cases": args.train, "test_cases": args.test, "epochs": args.epochs,
           "data_s": t_data, "train_s": t_train, "train_loss_first_last": [hist[0], hist[-1]],
           "tf32": {"rel_l2_median": q(rows[:, 0], 0.5),
                    "focal_amp_err_median": q(rows[:, 1], 0.5),
                    "focal_amp_err_p90": q(rows[:, 1], 0.9),
                    "focus_dist_mm_median": q(rows[:, 2], 0.5) * 1e3,
                    "focus_dist_mm_p90": q(rows[:, 2], 0.9) * 1e3,
                    "EL_rel_err_median": q(el_err[:, 0], 0.5), "EL_rel_err_p90": q(el_err[:, 0], 0.9)},
           "bf16": {"rel_l2_median": q(rows[:, 3], 0.5),
                    "focal_amp_err_median": q(rows[:, 4], 0.5),
                    "focal_amp_err_p90": q(rows[:, 4], 0.9),
                    "focus_dist_mm_median": q(rows[:, 5], 0.5) * 1e3,
                    "EL_rel_err_median": q(el_err[:, 1], 0.5), "EL_rel_err_p90": q(el_err[:, 1], 0.9)},
           "tf32_vs_bf16_max_rel": agree,
           "same_workload_timing_ms": tm,
           "speedup_vs_plan": {"tf32": tm["plan"] / tm["surrogate_tf32"],
                               "tf32_graph": tm["plan"] / tm["surrogate_tf32_graph"],
                               "bf16": tm["plan"] / tm["surrogate_bf16"],
                               "bf16_graph": tm["plan"] / tm["surrogate_bf16_graph"]},
           "speedup_vs_plan_fdtd": {"tf32_graph": tm["plan_without_bhte"]
                                    / tm["surrogate_tf32_graph"],
                                    "bf16_graph": tm["plan_without_bhte"]
                                    / tm["surrogate_bf16_graph"]}}
    print(json.dumps(res), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
