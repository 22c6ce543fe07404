"""One transcranial plan through libbvf: the paper's transcranial-modelling and
thermal-modelling steps for one transducer placement (Sec. 2.3, Sec. 2.4).

  1. property table -> viscoelastic coefficients        (bvf_set_materials)
  2. Rayleigh-Sommerfeld field of the bowl on the entry plane   (bvf_rs_plane)
  3. FDTD through the skull with peak and FP64 amplitude capture (bvf_run_acoustic)
  4. the same FDTD in water only (Sec. 2.3: water-only field)
  5. E_L on the plane of maximal water intensity, T_S = sqrt(E_L)   (bvf_transmission)
  6. scaling to I_SPPA-brain (default 5 W/cm^2, Sec. 2.4)
  7. BHTE with duty cycle, T_max and CEM43                          (bvf_run_thermal)

Every numerical step runs in the CUDA library; this module only sequences the
calls and moves buffers.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import bvf
from .synth import Case, water_row

I_SPPA_BRAIN_DEFAULT = 5.0e4     # 5 W/cm^2 in W/m^2 (Sec. 2.4)


@dataclass
class ThermalRegime:
    """Sec. 4.1.1 regime: 40 s on at 30 % duty cycle, then 80 s off."""
    t_on: float = 40.0
    t_off: float = 80.0
    duty: float = 0.3
    dt: float = 0.1
    T_a: float = 37.0
    rhob_cb: float = 1050.0 * 3617.0

    @property
    def n_on(self) -> int:
        return int(round(self.t_on / self.dt))

    @property
    def n_off(self) -> int:
        return int(round(self.t_off / self.dt))


@dataclass
class PlanResult:
    peak: "object"          # max |p| map of the skull run (float32, device or host)
    amp: "object"           # FP64 pressure amplitude of the skull run (device)
    amp_water: "object"     # FP64 amplitude of the water run (not kept by bvf_plan: None)
    Tmax: "object"          # float32 max temperature map
    cem43: "object"         # FP64 thermal dose map (minutes at 43 C)
    EL: float
    TS: float
    z_m: int
    Iw_max: float
    p_scale: float
    voxel_steps: int


class Planner:
    """Two contexts (skull run, water run) on one grid, reused across plans.
    storage: "f32" or "f16" (scaled FP16 acoustic state, FP32 arithmetic)."""

    def __init__(self, case: Case, storage: str = "f32"):
        import torch
        self.case = case
        c = case
        self.skull = bvf.Solver(c.nx, c.ny, c.nz, c.dx, c.dt, c.f0, qc=c.qc, n_sls=c.n_sls,
                                n_pml=c.n_pml, pml_R=c.pml_R, storage=storage)
        self.water = bvf.Solver(c.nx, c.ny, c.nz, c.dx, c.dt, c.f0, qc=c.qc, n_sls=c.n_sls,
                                n_pml=c.n_pml, pml_R=c.pml_R, storage=storage)
        self.water_idx = torch.zeros((c.nz, c.ny, c.nx), dtype=torch.uint8, device="cuda")
        self.water_table = np.array([water_row(c.f0)])
        self.water.set_materials(self.water_idx, self.water_table)

    def close(self):
        self.skull.close()
        self.water.close()

    def launches(self) -> int:
        return self.skull.stats().kernel_launches + self.water.stats().kernel_launches

    def kernel_timing(self, enable: bool):
        self.skull.kernel_timing(enable)
        self.water.kernel_timing(enable)

    def kernel_times(self):
        a, b = self.skull.kernel_times(), self.water.kernel_times()
        return dict(velocity_launches=a.velocity_launches + b.velocity_launches,
                    stress_launches=a.stress_launches + b.stress_launches,
                    velocity_ms=a.velocity_ms + b.velocity_ms,
                    stress_ms=a.stress_ms + b.stress_ms)

    def run(self, index, materials, bowl: dict, regime: ThermalRegime | None = None,
            i_sppa_brain: float = I_SPPA_BRAIN_DEFAULT, serial: bool = False) -> PlanResult:
        """index: (nz, ny, nx) uint8 CUDA tensor; materials: (n, 9) rows; bowl:
        aperture, roc, apex, dir, p0 (see bvf_bowl).  One bvf_plan call; the
        outputs are fresh tensors of this run.  serial: run the water
        companion after the skull run instead of beside it (same results)."""
        import torch
        c = self.case
        regime = regime or ThermalRegime()
        shape = (c.nz, c.ny, c.nx)
        peak = torch.empty(shape, dtype=torch.float32, device="cuda")
        amp = torch.empty(shape, dtype=torch.float64, device="cuda")
        T = torch.empty(shape, dtype=torch.float32, device="cuda")
        Tmax = torch.empty(shape, dtype=torch.float32, device="cuda")
        cem = torch.empty(shape, dtype=torch.float64, device="cuda")
        th = bvf.Thermal(regime.dt, regime.n_on, regime.n_off, regime.duty, regime.T_a,
                         regime.rhob_cb, 0.0)
        pp = bvf.PlanParams(c.n_steps, c.dft_start, c.dft_steps, i_sppa_brain, th,
                            1 if serial else 0)
        r = bvf.bvf_plan(self.skull, self.water, index, materials, self.water_table[0],
                         dict(bowl), c.k_src, pp, peak, amp, T, Tmax, cem)
        return PlanResult(peak, amp, None, Tmax, cem, r.EL, r.TS, r.z_m, r.Iw_max, r.p_scale,
                          2 * c.n_steps * c.voxels)

    def run_host(self, index, materials, bowl: dict, peak, Tmax, cem, T=None,
                 regime: ThermalRegime | None = None,
                 i_sppa_brain: float = I_SPPA_BRAIN_DEFAULT, serial: bool = False):
        """The same plan with host buffers (bvf_plan_host): index (nz, ny, nx)
        uint8 and the outputs peak, Tmax (float32), cem (float64) and T
        (float32, optional) are host arrays or pinned CPU tensors; the copies
        run inside the call.  Returns the PlanOut scalars."""
        c = self.case
        regime = regime or ThermalRegime()
        th = bvf.Thermal(regime.dt, regime.n_on, regime.n_off, regime.duty, regime.T_a,
                         regime.rhob_cb, 0.0)
        pp = bvf.PlanParams(c.n_steps, c.dft_start, c.dft_steps, i_sppa_brain, th,
                            1 if serial else 0)
        return bvf.bvf_plan_host(self.skull, self.water, index, materials, self.water_table[0],
                                 dict(bowl), c.k_src, pp, peak, T, Tmax, cem)
