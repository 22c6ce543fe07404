"""Stored FP64 oracle results of the mixed-precision workload family, and the
comparison of a library run with them.

The result files are written by make_config3_reference.py, which calls only
the oracle and the seeded input generator; this module holds no arithmetic of
the method (it reads the files, cuts the same planes out of a run's maps and
measures differences), so the GPU tests and the benchmark may use it."""
from __future__ import annotations

import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OUTPUTS = ("p", "peak", "amp", "phase", "Tmax", "cem")
FREQS = (250e3, 700e3)


def path_for(f0: float) -> str:
    return os.path.join(HERE, "config3_%dkhz.npz" % int(round(f0 / 1e3)))


def sample_step(f0: float) -> int:
    """In-plane sampling of the stored planes (every voxel at 250 kHz, every
    second one at 700 kHz)."""
    return 1 if f0 < 5e5 else 2


def planes(vol, focus, step):
    """x-z plane at the focus' y, y-z plane at its x, x-y plane at its z
    (vol is (nz, ny, nx); focus is (i, j, k))."""
    i, j, k = focus
    return (vol[:, j, ::step][::step], vol[:, ::step, i][::step], vol[k, ::step, ::step])


def load(f0: float):
    """(meta dict, {output_tag: float64 plane})."""
    z = np.load(path_for(f0))
    meta = json.loads(str(z["meta"]))
    return meta, {k: z[k].astype(np.float64) for k in z.files if k != "meta"}


def errors(meta, ref, maps, scalars):
    """Differences of a run from the stored oracle results.  maps: full
    (nz, ny, nx) arrays named as OUTPUTS; scalars: EL, TS, z_m.  Amplitude-like
    outputs give the relative L2 over the three planes and the largest
    difference relative to the reference's largest value there; the phase is
    compared where the amplitude exceeds a tenth of its largest value; T_max
    in degrees C."""
    step, focus = meta["step"], tuple(meta["focus"])

    def host(a):      # numpy arrays, or device tensors (only the planes are copied)
        return a.cpu().numpy() if hasattr(a, "cpu") else np.asarray(a)

    got = {}
    for name in OUTPUTS:
        for tag, pl in zip(("xz", "yz", "xy"), planes(maps[name], focus, step)):
            got["%s_%s" % (name, tag)] = host(pl).astype(np.float64)

    def stack(name, src):
        return np.concatenate([src["%s_%s" % (name, t)].ravel() for t in ("xz", "yz", "xy")])

    out = {}
    for name in ("p", "peak", "amp", "cem"):
        a, b = stack(name, got), stack(name, ref)
        out[name + "_rel_l2"] = float(np.linalg.norm(a - b) / np.linalg.norm(b))
        out[name + "_max_abs_rel"] = float(np.abs(a - b).max() / np.abs(b).max())
    amp = stack("amp", ref)
    beam = amp > 0.1 * amp.max()
    dphi = np.angle(np.exp(1j * (stack("phase", got) - stack("phase", ref))))
    out["phase_max_abs_rad_in_beam"] = float(np.abs(dphi[beam]).max())
    out["Tmax_max_abs_C"] = float(np.abs(stack("Tmax", got) - stack("Tmax", ref)).max())
    out["focal_peak_rel"] = abs(float(maps["peak"].max()) - meta["peak_max"]) / meta["peak_max"]
    out["EL_rel"] = abs(scalars["EL"] - meta["EL"]) / meta["EL"]
    out["TS_rel"] = abs(scalars["TS"] - meta["TS"]) / meta["TS"]
    out["z_m"] = [int(scalars["z_m"]), int(meta["z_m"])]
    out["cem43_max_rel"] = abs(float(maps["cem"].max()) - meta["cem_max"]) / meta["cem_max"]
    return out
