"""Training of the surrogate on FDTD fields (offline tool).

Training data come from the CUDA FDTD of this package (bvf.Solver): seeded
synthetic skulls with tilted bowls (synth.sweep_case), the FP64 amplitude of
the ramped-CW field over the capture window as the target (divided by the
bowl's surface pressure), and the feature volume of bvf_fno_features as the
input.  The network is the one of include/bvf_fno.h, trained with PyTorch
autograd: an offline step, not the planning-time path.  The trained weights
are exported in the flat blob layout and evaluated through the CUDA inference
(fno.Surrogate) on held-out skulls: relative L2 error of the field, error of
the focal amplitude (the field maximum) and distance between the predicted
and the FDTD focus.

    python -m paper_2301_12727_gb300.fno_train --train 400 --test 40 --epochs 30
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np


def make_dataset(n, seed, grid, dx, f0, dft_cycles=6):
    """n (features, target) pairs on one grid; returns CUDA tensors
    [n, 8, nz, ny, nx] and [n, 1, nz, ny, nx] (float32)."""
    import torch
    from . import bvf, fno, synth
    nx, ny, nz = grid
    feats = torch.empty((n, 8, nz, ny, nx), dtype=torch.float32, device="cuda")
    amps = torch.empty((n, 1, nz, ny, nx), dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(seed)
    sol = None
    for i in range(n):
        spec = dict(nx=nx, ny=ny, nz=nz, f0=f0, dx=dx, tilt_deg=float(rng.uniform(-15.0, 15.0)),
                    seed=int(seed) * 100000 + i)
        c = synth.sweep_case(spec, dft_cycles=dft_cycles)
        if sol is None:
            sol = bvf.Solver(nx, ny, nz, dx, c.dt, f0, n_sls=c.n_sls, n_pml=c.n_pml)
            dt0 = c.dt
        if c.dt != dt0:
            raise RuntimeError("time step differs between cases of one grid")
        idx = torch.from_numpy(c.index).cuda()
        sol.reset()
        sol.set_materials(idx, c.materials)
        plane = bvf.rs_plane(c.bowl, nx, ny, dx, c.k_src * dx, f0)
        sol.set_source(plane, c.k_src, c.c0, bvf.BVF_ENV_RAMP_CW)
        sol.run(c.n_steps, peak_from=-1, dft_start=c.dft_start, dft_steps=c.dft_steps)
        amp, _ = sol.amp_phase()
        amps[i, 0] = (amp / c.bowl["p0"]).float()
        fno.bvf_fno_features(idx, c.materials, synth.water_row(f0), f0, c.k_src, plane,
                             c.bowl["p0"], feats[i])
    sol.synchronize()
    sol.close()
    return feats, amps


class TorchFNO:
    """The network of include/bvf_fno.h as PyTorch parameters (for training)."""

    def __init__(self, d, seed=0, device="cuda"):
        import torch
        g = torch.Generator().manual_seed(seed)
        self.d = d
        w, m, ci, h, co = d["width"], d["modes"], d["c_in"], d["hidden"], d["c_out"]

        def p(*shape, scale):
            return (torch.randn(*shape, generator=g) * scale).to(device).requires_grad_()

        self.Wp, self.bp = p(w, ci, scale=1 / math.sqrt(ci)), p(w, scale=0.1)
        self.R, self.W, self.b = [], [], []
        for _ in range(d["n_layers"]):
            self.R.append(p(2 * m, 2 * m, m, w, w, 2, scale=1.0 / (w * w)))
            self.W.append(p(w, w, scale=1 / math.sqrt(w)))
            self.b.append(p(w, scale=0.1))
        self.Q1, self.q1 = p(h, w, scale=1 / math.sqrt(w)), p(h, scale=0.1)
        self.Q2, self.q2 = p(co, h, scale=1 / math.sqrt(h)), p(co, scale=0.1)

    def params(self):
        out = [self.Wp, self.bp]
        for l in range(self.d["n_layers"]):
            out += [self.R[l], self.W[l], self.b[l]]
        return out + [self.Q1, self.q1, self.Q2, self.q2]

    def blob(self) -> np.ndarray:
        """Weights in the flat layout of include/bvf_fno.h (same order as params)."""
        return np.concatenate([t.detach().float().cpu().numpy().ravel()
                               for t in self.params()]).astype(np.float32)

    def spectral(self, v, R):
        import torch
        m = self.d["modes"]
        B, C, nz, ny, nx = v.shape
        j = torch.arange(2 * m, device=v.device)
        iz = torch.where(j < m, j, j - 2 * m) % nz
        iy = torch.where(j < m, j, j - 2 * m) % ny
        vh = torch.fft.rfftn(v, dim=(2, 3, 4))
        kept = vh[:, :, iz][:, :, :, iy][..., :m]
        out_k = torch.einsum("bczyk,zykco->bozyk", kept, torch.view_as_complex(R))
        full = torch.zeros((B, R.shape[4], nz, ny, nx // 2 + 1), dtype=vh.dtype, device=v.device)
        full[:, :, iz[:, None], iy[None, :], :m] = out_k
        return torch.fft.irfftn(full, s=(nz, ny, nx), dim=(2, 3, 4))

    def __call__(self, a):
        import torch
        import torch.nn.functional as F
        v = torch.einsum("oi,bizyx->bozyx", self.Wp, a) + self.bp[None, :, None, None, None]
        L = self.d["n_layers"]
        for l in range(L):
            s = (self.spectral(v, self.R[l]) + torch.einsum("oc,bczyx->bozyx", self.W[l], v)
                 + self.b[l][None, :, None, None, None])
            v = F.gelu(s) if l < L - 1 else s
        h = F.gelu(torch.einsum("hc,bczyx->bhzyx", self.Q1, v) + self.q1[None, :, None, None, None])
        return torch.einsum("oh,bhzyx->bozyx", self.Q2, h) + self.q2[None, :, None, None, None]


def focal_metrics(pred, true, dx):
    """Relative L2 field error, focal amplitude error and focus distance (m)."""
    import torch
    rl2 = float(torch.linalg.vector_norm(pred - true) / torch.linalg.vector_norm(true))
    pt, pp = float(true.max()), float(pred.max())
    it = np.array(np.unravel_index(int(torch.argmax(true)), true.shape[-3:]))
    ip = np.array(np.unravel_index(int(torch.argmax(pred)), pred.shape[-3:]))
    return rl2, abs(pp - pt) / pt, float(np.linalg.norm((ip - it) * dx))


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=400)
    ap.add_argument("--test", type=int, default=40)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--grid", default="64,64,96")
    ap.add_argument("--dx", type=float, default=1e-3)
    ap.add_argument("--f0", type=float, default=2.5e5)
    ap.add_argument("--width", type=int, default=32)
    ap.add_argument("--modes", type=int, default=12)
    ap.add_argument("--layers", type=int, default=4)
    ap.add_argument("--hidden", type=int, default=128)
    ap.add_argument("--seed", type=int, default=7)
    args = ap.parse_args(argv)
    from . import build as _b
    _b.build()
    from . import fno
    grid = tuple(int(v) for v in args.grid.split(","))
    d = dict(c_in=8, width=args.width, modes=args.modes, n_layers=args.layers,
             hidden=args.hidden, c_out=1)
    t0 = time.time()
    xtr, ytr = make_dataset(args.train, args.seed, grid, args.dx, args.f0)
    xte, yte = make_dataset(args.test, args.seed + 1, grid, args.dx, args.f0)
    t_data = time.time() - t0

    model = TorchFNO(d, seed=args.seed)
    opt = torch.optim.Adam(model.params(), lr=args.lr)
    steps_per_epoch = max(1, args.train // args.batch)
    total = args.epochs * steps_per_epoch
    sched = torch.optim.lr_scheduler.OneCycleLR(opt, max_lr=args.lr, total_steps=total)
    gen = torch.Generator(device="cpu").manual_seed(args.seed)
    t1 = time.time()
    hist = []
    for ep in range(args.epochs):
        perm = torch.randperm(args.train, generator=gen)
        run = 0.0
        for k in range(steps_per_epoch):
            sel = perm[k * args.batch:(k + 1) * args.batch].cuda()
            x, y = xtr[sel], ytr[sel]
            p = model(x)
            num = torch.linalg.vector_norm((p - y).flatten(1), dim=1)
            den = torch.linalg.vector_norm(y.flatten(1), dim=1)
            loss = (num / den).mean()
            opt.zero_grad(set_to_none=True)
            loss.backward()
            opt.step()
            sched.step()
            run += float(loss.detach())
        hist.append(run / steps_per_epoch)
    torch.cuda.synchronize()
    t_train = time.time() - t1

    # held-out skulls through the CUDA inference with the exported weights
    net = fno.Surrogate(d, model.blob())
    rows = []
    cons = 0.0
    with torch.no_grad():
        for i in range(args.test):
            out = net(xte[i].contiguous())
            pt = model(xte[i:i + 1])[0]
            cons = max(cons, float((out - pt).abs().max() / pt.abs().max()))
            rows.append(focal_metrics(out, yte[i], args.dx))
    net.close()
    rows = np.array(rows)
    # focal amplitudes (units of p0) the training set covers: the range that
    # fno.predict_amplitude accepts before it falls back to the FDTD
    tmax = ytr.flatten(1).max(dim=1).values
    res = {"grid": list(grid), "dx_m": args.dx, "f0_hz": args.f0, "dims": d,
           "train_focal_range_p0": [float(tmax.min()), float(tmax.max())],
           "train_cases": args.train, "test_cases": args.test, "epochs": args.epochs,
           "data_s": t_data, "train_s": t_train, "train_loss_first_last": [hist[0], hist[-1]],
           "test_rel_l2_median": float(np.median(rows[:, 0])),
           "test_focal_amp_err_median": float(np.median(rows[:, 1])),
           "test_focal_amp_err_p90": float(np.quantile(rows[:, 1], 0.9)),
           "test_focus_dist_mm_median": float(np.median(rows[:, 2]) * 1e3),
           "test_focus_dist_mm_p90": float(np.quantile(rows[:, 2], 0.9) * 1e3),
           "cuda_vs_torch_max_rel": cons}
    print(json.dumps(res), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
