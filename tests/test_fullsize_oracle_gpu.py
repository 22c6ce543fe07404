"""The benchmark's own workload against the FP64 oracle, output by output.

One whole plan exactly as bench.py times it (240 x 240 x 200 synthetic skull,
dx 0.5 mm, 500 kHz, 1500 FDTD steps, ramped CW bowl source, peak map from
step 1, 10-cycle FP64 amplitude window, the water-only companion run, E_L on
the plane of maximal water intensity, I_SPPA scaling and the 40 s / 30 % /
80 s BHTE with CEM43), run through bvf_plan in the bench's launch
configuration (TMA kernels, default z-chunk), and the same plan computed by
the FP64 C oracle on the host cores: the oracle's own Rayleigh-Sommerfeld
plane, both FDTD runs, E_L, the scaling and the BHTE.  Nothing is shared but
the seeded inputs.

Tolerances follow the accuracy target (1e-4 relative L2 on pressure for the
FP32 solver) and the arithmetic of each output:
  pressure at step 1500, peak map, skull and water amplitudes: relative L2
    below 1e-4 (FP32 rounding over 1500 steps stays near 1e-5);
  phase, where the skull amplitude exceeds a tenth of its maximum: 1e-3 rad;
  E_L and T_S: 1e-4 relative; z_m: equal;
  T_max: 2e-3 C (FP32 temperature over 1200 explicit steps, increments of
    about 1e-3 C against an FP32 ulp of 4e-6 C at 37 C);
  CEM43: 2e-3 relative at its maximum and in L2 (the dose is exp(ln 4 T), so
    a T error dT moves it by 1.4 dT relative).
The measured errors are printed, and written as JSON to the file named by
BVF_PARITY_REPORT when that variable is set."""
import json
import os
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def test_fullsize_plan_matches_the_fp64_oracle(orc):
    import torch
    assert torch.cuda.is_available()
    from paper_2301_12727_gb300 import build
    build.build()
    from paper_2301_12727_gb300 import plan, synth

    c = synth.skull_case(240, 240, 200, dx=0.5e-3, f0=5e5, n_steps=1500, seed=1234,
                         dft_cycles=10)
    regime = plan.ThermalRegime()
    # ---- GPU: one plan through bvf_plan, as the bench runs it
    pl = plan.Planner(c)
    r = pl.run(torch.from_numpy(c.index).cuda(), c.materials, c.bowl, regime)
    torch.cuda.synchronize()
    g = dict(p=pl.skull.pressure().cpu().numpy(), peak=r.peak.cpu().numpy(),
             Tmax=r.Tmax.cpu().numpy(), cem=r.cem43.cpu().numpy())
    a, ph = pl.skull.amp_phase()
    aw = pl.water.amp_phase()[0]
    g.update(amp=a.cpu().numpy(), phase=ph.cpu().numpy(), amp_w=aw.cpu().numpy())
    torch.cuda.synchronize()
    pl.close()

    # ---- oracle: the same plan in FP64 on the host cores
    t0 = time.perf_counter()
    b = c.bowl
    plane = orc.rs_plane(b["aperture"], b["roc"], b["apex"], b["dir"], c.nx, c.ny, c.dx,
                         c.k_src * c.dx, c.f0, c.c0, b["p0"])
    ref = {}
    water_idx = np.zeros_like(c.index)
    water = np.array([synth.water_row(c.f0)])
    for name, idx, mats in (("skull", c.index, c.materials), ("water", water_idx, water)):
        A = orc.Acoustic(c.nx, c.ny, c.nz, c.dx, c.dt, idx, mats, c.f0, qc=c.qc, n_sls=c.n_sls,
                         n_pml=c.n_pml, pml_R=c.pml_R)
        A.set_source(plane, c.k_src, c.c0, orc.ENV_RAMP_CW)
        assert A.run(c.n_steps, peak_from=0, dft_start=c.dft_start, dft_steps=c.dft_steps) == 0
        amp, phase = A.amp_phase(c.dft_steps)
        if name == "skull":
            ref.update(p=A.pressure(), peak=A.peak.copy(), amp=amp, phase=phase)
        else:
            ref.update(amp_w=amp)
        del A
    t_fdtd = time.perf_counter() - t0
    EL, zm = orc.transmission(c.index, c.materials, ref["amp"], water_idx, water, ref["amp_w"])
    iw_max = float((ref["amp_w"] ** 2 / (2.0 * water[0, 0] * water[0, 1])).max())
    p_scale = np.sqrt(plan.I_SPPA_BRAIN_DEFAULT / (EL * iw_max))
    rc, T, Tmax, cem = orc.bhte_run(c.index, c.materials, c.dx, ref["amp"], p_scale, regime.dt,
                                    regime.n_on, regime.n_off, regime.duty, regime.T_a,
                                    regime.rhob_cb)
    assert rc == 0
    t_all = time.perf_counter() - t0

    beam = ref["amp"] > 0.1 * ref["amp"].max()
    dphi = np.abs(np.angle(np.exp(1j * (g["phase"] - ref["phase"]))))[beam]
    errs = {
        "pressure_rel_l2": rel_l2(g["p"], ref["p"]),
        "peak_rel_l2": rel_l2(g["peak"], ref["peak"]),
        "focal_peak_rel": abs(float(g["peak"].max()) - ref["peak"].max()) / ref["peak"].max(),
        "amp_rel_l2": rel_l2(g["amp"], ref["amp"]),
        "phase_max_abs_rad_in_beam": float(dphi.max()),
        "amp_water_rel_l2": rel_l2(g["amp_w"], ref["amp_w"]),
        "EL_rel": abs(r.EL - EL) / EL,
        "TS_rel": abs(r.TS - np.sqrt(EL)) / np.sqrt(EL),
        "zm": [r.z_m, zm],
        "Tmax_max_abs_C": float(np.abs(g["Tmax"] - Tmax).max()),
        "Tmax_rise_max_C": float(Tmax.max() - regime.T_a),
        "cem43_rel_at_max": abs(float(g["cem"].max()) - cem.max()) / cem.max(),
        "cem43_rel_l2": rel_l2(g["cem"], cem),
        "oracle_seconds": {"fdtd_two_runs": t_fdtd, "whole_plan": t_all,
                           "threads": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count()))},
        "EL": EL, "TS": float(np.sqrt(EL)),
    }
    print("full-size parity:", json.dumps(errs))
    out = os.environ.get("BVF_PARITY_REPORT")
    if out:
        with open(out, "w") as f:
            json.dump(errs, f, indent=1)
    assert errs["pressure_rel_l2"] < 1e-4
    assert errs["peak_rel_l2"] < 1e-4
    assert errs["amp_rel_l2"] < 1e-4
    assert errs["amp_water_rel_l2"] < 1e-4
    assert errs["phase_max_abs_rad_in_beam"] < 1e-3
    assert errs["EL_rel"] < 1e-4 and errs["TS_rel"] < 1e-4
    assert r.z_m == zm
    assert errs["Tmax_max_abs_C"] < 2e-3
    assert errs["cem43_rel_at_max"] < 2e-3 and errs["cem43_rel_l2"] < 2e-3
