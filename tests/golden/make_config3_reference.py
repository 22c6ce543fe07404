"""Writes the FP64 oracle's results for the mixed-precision workload family
(the synthetic skull at 9 points per water wavelength, 250 kHz on 128 x 128 x
108 and 700 kHz on 360 x 360 x 300, transit + 10 cycles, 10-cycle FP64
amplitude window, water companion run, E_L and I_SPPA scaling (Sec. 2.4,
Eq. 2), then the 40 s / 30 % / 80 s BHTE with CEM43 (Sec. 4.1.1)).

Only the oracle (oracle/) and the seeded input generator (synth) are called.
The result file holds the plan's scalars and, for each output map (final
pressure, peak, amplitude, phase, T_max, CEM43), three planes through the
focus (the largest skull-run amplitude in the brain): x-z, y-z and x-y,
sampled every `step` voxels in-plane.  The GPU tests and the benchmark compare
the library's runs with these values.

Usage: python tests/golden/make_config3_reference.py 250e3 [700e3]
(about 3 minutes at 250 kHz and 2 hours at 700 kHz on 8 cores; 26 GB of RAM
at 700 kHz)."""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)

import oracle  # noqa: E402
from paper_2301_12727_gb300 import synth  # noqa: E402  (seeded inputs only)

from config3 import path_for, planes, sample_step, OUTPUTS  # noqa: E402

I_SPPA_BRAIN = 5.0e4          # 5 W/cm^2 (Sec. 2.4)


def main(f0: float):
    t0 = time.time()
    grid = synth.CONFIG3_GRIDS[f0]
    c = synth.config3_case(f0, *grid)
    reg = synth.thermal_regime(c.dx, c.materials)
    oracle.build()
    b = c.bowl
    src = oracle.rs_plane(b["aperture"], b["roc"], b["apex"], b["dir"], c.nx, c.ny, c.dx,
                          c.k_src * c.dx, c.f0, c.c0, b["p0"])
    water_idx = np.zeros_like(c.index)
    water = np.array([synth.water_row(c.f0)])
    out = {}
    for name, idx, mats in (("skull", c.index, c.materials), ("water", water_idx, water)):
        A = oracle.Acoustic(c.nx, c.ny, c.nz, c.dx, c.dt, idx, mats, c.f0, qc=c.qc,
                            n_sls=c.n_sls, n_pml=c.n_pml, pml_R=c.pml_R)
        A.set_source(src, c.k_src, c.c0, oracle.ENV_RAMP_CW)
        rc = A.run(c.n_steps, peak_from=0, dft_start=c.dft_start, dft_steps=c.dft_steps)
        assert rc == 0, rc
        amp, ph = A.amp_phase(c.dft_steps)
        if name == "skull":
            out.update(p=A.pressure(), peak=A.peak.copy(), amp=amp, phase=ph)
        else:
            out["amp_w"] = amp
        del A
        print("%s run done after %.0f s" % (name, time.time() - t0), flush=True)
    EL, zm = oracle.transmission(c.index, c.materials, out["amp"], water_idx, water,
                                 out["amp_w"])
    iw_max = float((out["amp_w"] ** 2 / (2.0 * water[0, 0] * water[0, 1])).max())
    p_scale = float(np.sqrt(I_SPPA_BRAIN / (EL * iw_max)))
    rc, T, Tmax, cem = oracle.bhte_run(c.index, c.materials, c.dx, out["amp"], p_scale,
                                       reg["dt"], reg["n_on"], reg["n_off"], reg["duty"],
                                       reg["T_a"], reg["rhob_cb"])
    assert rc == 0, rc
    out.update(Tmax=Tmax, cem=cem)
    brain_amp = np.where(c.index == 1, out["amp"], 0.0)
    k, j, i = np.unravel_index(np.argmax(brain_amp), brain_amp.shape)
    focus = (int(i), int(j), int(k))
    step = sample_step(f0)
    arrays = {}
    for name in OUTPUTS:
        for tag, pl in zip(("xz", "yz", "xy"), planes(out[name], focus, step)):
            arrays["%s_%s" % (name, tag)] = np.ascontiguousarray(pl, dtype=np.float32)
    meta = dict(f0=f0, grid=list(grid), dx=c.dx, dt=c.dt, n_steps=c.n_steps,
                dft_start=c.dft_start, dft_steps=c.dft_steps, k_src=c.k_src, seed=1234,
                regime=reg, EL=EL, TS=float(np.sqrt(EL)), z_m=int(zm), Iw_max=iw_max,
                p_scale=p_scale, focus=list(focus), step=step,
                peak_max=float(out["peak"].max()), amp_max=float(out["amp"].max()),
                Tmax_max=float(Tmax.max()), cem_max=float(cem.max()),
                amp_w_max=float(out["amp_w"].max()),
                oracle_seconds=time.time() - t0, threads=os.cpu_count(),
                writer="tests/golden/make_config3_reference.py (FP64 oracle)")
    np.savez_compressed(path_for(f0), meta=np.array(json.dumps(meta)), **arrays)
    print(json.dumps(meta), flush=True)


if __name__ == "__main__":
    for a in sys.argv[1:] or ["250e3"]:
        main(float(a))
