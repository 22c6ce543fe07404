"""The mixed-precision workload family against the FP64 oracle, per output.

The synthetic skull at 9 points per water wavelength, 250 kHz on 128 x 128 x
108 and 700 kHz on 360 x 360 x 300 (transit + 10 cycles, 10-cycle FP64
amplitude window, water companion run, E_L, I_SPPA scaling, then the 40 s /
30 % / 80 s BHTE with perfusion and CEM43), planned through bvf_plan with the
acoustic state stored in FP32 and in scaled FP16 (FP32 arithmetic either way;
FP64 DFT sums and dose on the GPU).  The oracle's results were computed once
by tests/golden/make_config3_reference.py (FP64, whole runs on the full
grids) and stored as planes through the focus; the run is compared with them
element by element.

Tolerances.  FP32 storage: the accuracy target's 1e-4 relative L2 on pressure,
peak and amplitude; 1e-3 rad of phase in the beam; 1e-4 on E_L.  FP16 storage
(11 significant bits, relative rounding 4.9e-4 per stored value): the 1 %
peak-pressure bound of the mixed-precision target for the peak and amplitude
maps, the focal peak and E_L; 1e-2 rad of phase.  Thermal outputs, in either
storage: the temperature is an FP32 sum of n small increments on T near
37 C, where an FP32 value carries a rounding of at most half an ulp,
32 * 2^-24 C = 2^-19 C = 1.9e-6 C, per step; so T_max may differ by up to
n * 1.9e-6 C (at least 2e-3 C), and CEM43, whose rate R^(43 - T) moves by
ln 4 = 1.39 per C, by 1.39 times that, relative (at least 2e-3).  The
measured errors are printed."""
import json

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = {
    "f32": dict(p_rel_l2=1e-4, peak_rel_l2=1e-4, amp_rel_l2=1e-4, phase=1e-3, EL=1e-4,
                focal=1e-4),
    "f16": dict(p_rel_l2=1e-2, peak_rel_l2=1e-2, amp_rel_l2=1e-2, phase=1e-2, EL=1e-2,
                focal=1e-2),
}


def thermal_tol(n_thermal_steps):
    """(T_max in C, CEM43 relative) bounds of an FP32 temperature summed over
    n steps near 37 C (see the module header)."""
    t = max(2e-3, n_thermal_steps * 2.0 ** -19)
    return t, max(2e-3, np.log(4.0) * t)

_cases = {}


def case_for(f0):
    from paper_2301_12727_gb300 import synth
    if f0 not in _cases:
        _cases[f0] = synth.config3_case(f0, *synth.CONFIG3_GRIDS[f0])
    return _cases[f0]


def run_plan(c, storage):
    """One plan through bvf_plan; the full maps named as the stored outputs."""
    import torch
    from paper_2301_12727_gb300 import plan, synth
    reg = synth.thermal_regime(c.dx, c.materials)
    regime = plan.ThermalRegime(dt=reg["dt"], duty=reg["duty"])
    pl = plan.Planner(c, storage=storage)
    r = pl.run(torch.from_numpy(c.index).cuda(), c.materials, c.bowl, regime)
    amp, ph = pl.skull.amp_phase()
    maps = dict(p=pl.skull.pressure().cpu().numpy(), peak=r.peak.cpu().numpy(),
                amp=amp.cpu().numpy(), phase=ph.cpu().numpy(), Tmax=r.Tmax.cpu().numpy(),
                cem=r.cem43.cpu().numpy())
    pl.close()
    return maps, dict(EL=r.EL, TS=r.TS, z_m=r.z_m)


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("f0", [250e3, 700e3])
def test_config3_plan_against_the_fp64_oracle(f0, storage):
    import torch
    assert torch.cuda.is_available()
    from paper_2301_12727_gb300 import build
    build.build()
    from tests.golden import config3
    meta, ref = config3.load(f0)
    c = case_for(f0)
    assert [c.nx, c.ny, c.nz] == meta["grid"] and c.n_steps == meta["n_steps"]
    assert c.dt == meta["dt"]
    maps, sc = run_plan(c, storage)
    e = config3.errors(meta, ref, maps, sc)
    print("config3 %g kHz %s vs FP64 oracle: %s" % (f0 / 1e3, storage, json.dumps(e)))
    t = TOL[storage]
    assert e["p_rel_l2"] < t["p_rel_l2"]
    assert e["peak_rel_l2"] < t["peak_rel_l2"]
    assert e["amp_rel_l2"] < t["amp_rel_l2"]
    assert e["focal_peak_rel"] < t["focal"]
    assert e["phase_max_abs_rad_in_beam"] < t["phase"]
    assert e["EL_rel"] < t["EL"]
    assert e["z_m"][0] == e["z_m"][1]
    reg = meta["regime"]
    t_T, t_cem = thermal_tol(reg["n_on"] + reg["n_off"])
    assert e["Tmax_max_abs_C"] < t_T
    assert e["cem_rel_l2"] < t_cem and e["cem43_max_rel"] < t_cem
