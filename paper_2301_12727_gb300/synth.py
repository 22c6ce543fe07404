"""Seeded synthetic inputs shared by the tests, the oracle legs and the benchmark.

This module holds input recipes only (phantom geometry, tissue tables, bowl
poses, the time-step rule); none of the solver's arithmetic lives here.  It
stands in for the paper's CT/MRI subject data (Sec. 3.2: five CT scans, not
distributed with the paper) with shapes and tissue layering taken from it:

  * skin / skull / brain label mask, skull split cortical 10 % / trabecular
    80 % / cortical 10 % (Sec. 2.2.1);
  * CT-like HU in [300, 2000] quantised into bins that index a property table
    (Sec. 2.2.2 quantises HU at 12 bits and maps HU to density, speed and
    attenuation);
  * single-element focused bowl placed a few millimetres above the skin
    (Sec. 2 "Single", Sec. 3.2 "Modeling");
  * homogenised tissue values of Table 1 for skin and brain.

The HU -> property map is linear, anchored at water (HU 0) and at cortical bone
(HU 2000: rho 1850, cL 2800, cS 1500, alpha 85 Np/m at 500 kHz); the paper does
not print the coefficients of its own mappings.  Thermal constants are
literature-typical values (the paper gives none).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Material row layout used throughout: rho, cL, cS, alphaL, alphaS (Np/m at f0),
# k_th (W/m/K), c_th (J/kg/K), perf (1/s), heat_frac (fraction of alphaL -> heat).
MAT_COLS = ("rho", "cL", "cS", "alphaL", "alphaS", "k_th", "c_th", "perf", "heat_frac")

WATER_THERMAL = (0.60, 4178.0, 0.0, 1.0)
SKIN_THERMAL = (0.37, 3391.0, 0.008, 1.0)
BRAIN_THERMAL = (0.51, 3630.0, 0.008, 1.0)
BONE_THERMAL = (0.32, 1313.0, 0.008, 0.16)   # 0.16 of bone attenuation -> heat (Sec. 2.4)

COURANT_3D_O4 = 6.0 / (7.0 * math.sqrt(3.0))  # stability limit c dt / dx of the O(4) scheme


def water_row(f0: float) -> list:
    return [1000.0, 1500.0, 0.0, 0.0, 0.0, *WATER_THERMAL]


def skin_row(f0: float) -> list:       # Table 1: 1116, 1537, 4.6 f Np/m/MHz
    return [1116.0, 1537.0, 0.0, 4.6 * f0 / 1e6, 0.0, *SKIN_THERMAL]


def brain_row(f0: float) -> list:      # Table 1: 1041, 1562, 6.9 f Np/m/MHz
    return [1041.0, 1562.0, 0.0, 6.9 * f0 / 1e6, 0.0, *BRAIN_THERMAL]


def bone_row_from_hu(hu: float, f0: float) -> list:
    rho = 1000.0 + 0.425 * hu
    cL = 1500.0 + 0.65 * hu
    cS = 0.75 * hu
    aL = 85.0 * (hu / 2000.0) * (f0 / 5e5)
    return [rho, cL, cS, aL, 2.0 * aL, *BONE_THERMAL]


def choose_dt(dx: float, c_max: float, f0: float, courant_fraction: float = 0.5) -> tuple:
    """Time step: courant_fraction of the O(4) 3-D limit, shrunk so that one
    period is an integer number M of steps.  Returns (dt, M)."""
    dt0 = courant_fraction * COURANT_3D_O4 * dx / c_max
    M = int(math.ceil(1.0 / (f0 * dt0)))
    return 1.0 / (f0 * M), M


@dataclass
class Case:
    """One synthetic problem: grid, materials, source and run lengths."""
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    f0: float
    dt: float
    steps_per_period: int
    n_steps: int
    index: np.ndarray            # (nz, ny, nx) uint8
    materials: np.ndarray        # (n, 9) float64
    k_src: int
    envelope: int                # 1 burst, 2 ramp + CW
    n_cycles: int = 0
    plane: np.ndarray | None = None       # complex (ny, nx) source map, or None for a bowl
    bowl: dict | None = None              # aperture, roc, apex (m), dir, p0
    n_pml: int = 8
    pml_R: float = 1e-4
    n_sls: int = 2
    qc: float = 1.0
    c0: float = 1500.0
    dft_cycles: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def dft_steps(self) -> int:
        return self.dft_cycles * self.steps_per_period

    @property
    def dft_start(self) -> int:
        return self.n_steps - self.dft_steps + 1

    @property
    def voxels(self) -> int:
        return self.nx * self.ny * self.nz


def slab_case(n: int = 64, dx: float = 0.5e-3, f0: float = 5e5, n_steps: int = 400,
              p0: float = 1e5, n_pml: int = 8, k_src: int = 10) -> Case:
    """Flat 6 mm skull slab in water, plane 3-cycle burst (64^3 at 0.5 mm, 400 steps).

    Slab from z = 12 mm: cortical 1.5 mm | trabecular 3 mm | cortical 1.5 mm.
    Cortical: rho 1850, cL 2800, cS 1500, alphaL 85 Np/m; trabecular: rho 1700,
    cL 2300, cS 1200, alphaL 81 Np/m; alphaS = 2 alphaL (Table 1 ratio)."""
    mats = np.array([
        water_row(f0),
        [1850.0, 2800.0, 1500.0, 85.0, 170.0, *BONE_THERMAL],
        [1700.0, 2300.0, 1200.0, 81.0, 162.0, *BONE_THERMAL],
    ])
    index = np.zeros((n, n, n), dtype=np.uint8)
    z = (np.arange(n) + 0.0) * dx
    z0 = 12e-3
    cort1 = (z >= z0 - 1e-9) & (z < z0 + 1.5e-3 - 1e-9)
    trab = (z >= z0 + 1.5e-3 - 1e-9) & (z < z0 + 4.5e-3 - 1e-9)
    cort2 = (z >= z0 + 4.5e-3 - 1e-9) & (z < z0 + 6.0e-3 - 1e-9)
    index[cort1] = 1
    index[trab] = 2
    index[cort2] = 1
    dt, M = choose_dt(dx, mats[:, 1].max(), f0)
    plane = np.full((n, n), p0, dtype=np.complex128)
    return Case("slab%d" % n, n, n, n, dx, f0, dt, M, n_steps, index, mats, k_src, 1,
                n_cycles=3, plane=plane, n_pml=n_pml)


def _smooth_noise(shape, cell, rng):
    """Smooth field in [0, 1]: a coarse uniform random lattice (spacing `cell`
    voxels) trilinearly interpolated onto `shape`."""
    coarse = [int(math.ceil(s / cell)) + 2 for s in shape]
    lat = rng.random(coarse)
    axes = [np.arange(s) / cell for s in shape]
    idx = [np.floor(a).astype(np.int64) for a in axes]
    frac = [a - i for a, i in zip(axes, idx)]
    out = np.zeros(shape)
    for dz in (0, 1):
        wz = frac[0] if dz else 1 - frac[0]
        for dy in (0, 1):
            wy = frac[1] if dy else 1 - frac[1]
            for dxx in (0, 1):
                wx = frac[2] if dxx else 1 - frac[2]
                v = lat[np.ix_(idx[0] + dz, idx[1] + dy, idx[2] + dxx)]
                out += v * (wz[:, None, None] * wy[None, :, None] * wx[None, None, :])
    lo, hi = out.min(), out.max()
    return (out - lo) / (hi - lo) if hi > lo else np.zeros(shape)


def skull_case(nx: int = 240, ny: int = 240, nz: int = 200, dx: float = 0.5e-3,
               f0: float = 5e5, n_steps: int | None = None, seed: int = 1234,
               aperture: float = 64e-3, roc: float = 63e-3, p0: float = 6e4,
               n_pml: int = 8, dft_cycles: int = 10, n_bins: int = 125,
               symmetric: bool = False, tilt_deg: float = 0.0) -> Case:
    """Synthetic skull: ellipsoidal shell (semi-axes 70, 85, 60 mm) whose cap
    crosses the beam, 6-9 mm thick from seeded smooth noise, with 3 mm of skin
    outside and brain inside; HU quantised into `n_bins` bone bins (table
    indices 3 .. 3 + n_bins - 1; 0 water, 1 brain, 2 skin).  The bowl (64 mm
    aperture, 63 mm radius of curvature, axis +z through the lateral centre)
    has its apex 15 mm above the outer skull surface on the axis.

    `symmetric=True` mirrors the noise so the phantom is symmetric under
    x -> -x and y -> -y about the axis (for symmetry checks)."""
    rng = np.random.default_rng(seed)
    Lx, Ly = nx * dx, ny * dx
    xc, yc = 0.5 * (nx - 1) * dx, 0.5 * (ny - 1) * dx
    k_src = n_pml + 2
    z_src = k_src * dx
    z_outer = z_src + 5e-3                    # outer bone surface on the axis
    A, B, C = 70e-3, 85e-3, 60e-3
    zc = z_outer + C
    x = np.arange(nx) * dx - xc
    y = np.arange(ny) * dx - yc
    z = np.arange(nz) * dx - zc
    X, Y, Z = x[None, None, :], y[None, :, None], z[:, None, None]
    r = np.sqrt(X * X + Y * Y + Z * Z) + 1e-12
    ux, uy, uz = X / r, Y / r, Z / r
    r_out = 1.0 / np.sqrt(ux * ux / A ** 2 + uy * uy / B ** 2 + uz * uz / C ** 2)
    depth = r_out - r                          # > 0 inside the outer surface
    # thickness 6 + 3 n(u), n smooth over directions
    lat = rng.random((9, 9, 9))
    if symmetric:
        lat = 0.25 * (lat + lat[:, :, ::-1] + lat[:, ::-1, :] + lat[:, ::-1, ::-1])
    g = (np.stack([uz, uy, ux], axis=0) + 1.0) * 4.0   # map [-1,1] -> [0,8]
    gi = np.clip(np.floor(g).astype(np.int64), 0, 7)
    gf = g - gi
    tn = np.zeros(r.shape)
    for a in (0, 1):
        for b in (0, 1):
            for c in (0, 1):
                w = ((gf[0] if a else 1 - gf[0]) * (gf[1] if b else 1 - gf[1]) *
                     (gf[2] if c else 1 - gf[2]))
                tn += w * lat[gi[0] + a, gi[1] + b, gi[2] + c]
    tn = (tn - tn.min()) / max(tn.max() - tn.min(), 1e-12)
    thick = 6e-3 + 3e-3 * tn
    # HU fields
    cell = max(2, int(round(4e-3 / dx)))
    n_cort = _smooth_noise((nz, ny, nx), cell, rng)
    n_trab = _smooth_noise((nz, ny, nx), cell, rng)
    if symmetric:
        n_cort = 0.25 * (n_cort + n_cort[:, :, ::-1] + n_cort[:, ::-1, :] + n_cort[:, ::-1, ::-1])
        n_trab = 0.25 * (n_trab + n_trab[:, :, ::-1] + n_trab[:, ::-1, :] + n_trab[:, ::-1, ::-1])
    frac = depth / thick
    bone = (depth >= 0) & (frac < 1.0)
    cortical = bone & ((frac < 0.1) | (frac >= 0.9))
    hu = np.where(cortical, 1500.0 + 500.0 * n_cort, 300.0 + 700.0 * n_trab)
    hu = np.clip(hu, 300.0, 2000.0)
    width = 1700.0 / n_bins
    bins = np.clip(np.floor((hu - 300.0) / width).astype(np.int64), 0, n_bins - 1)
    index = np.zeros((nz, ny, nx), dtype=np.uint8)
    index[(depth < 0) & (depth >= -3e-3)] = 2
    index[depth >= thick] = 1
    index[bone] = (3 + bins[bone]).astype(np.uint8)
    if symmetric:
        # exact mirror symmetry: copy the low half of each lateral axis onto the high half
        hx, hy = nx // 2, ny // 2
        index[:, :, nx - hx:] = index[:, :, :hx][:, :, ::-1]
        index[:, ny - hy:, :] = index[:, :hy, :][:, ::-1, :]
    rows = [water_row(f0), brain_row(f0), skin_row(f0)]
    for b in range(n_bins):
        rows.append(bone_row_from_hu(300.0 + (b + 0.5) * width, f0))
    mats = np.array(rows)
    dt, M = choose_dt(dx, mats[:, 1].max(), f0)
    if n_steps is None:
        # transit of 1.3 x the domain depth in water plus the DFT window
        n_steps = int(math.ceil(1.3 * nz * dx / 1500.0 / dt)) + dft_cycles * M
    t = math.radians(tilt_deg)
    direction = (math.sin(t), 0.0, math.cos(t))
    apex_z = z_outer - 15e-3
    bowl = dict(aperture=aperture, roc=roc, apex=(xc, yc, apex_z), dir=direction, p0=p0)
    return Case("skull%dx%dx%d" % (nx, ny, nz), nx, ny, nz, dx, f0, dt, M, n_steps, index,
                mats, k_src, 2, plane=None, bowl=bowl, n_pml=n_pml, dft_cycles=dft_cycles)


def config3_case(f0: float, nx: int, ny: int, nz: int, seed: int = 1234) -> Case:
    """Mixed-precision workload family: the skull phantom at 9 points per
    water wavelength (dx = 1500 / (9 f0): 0.667 mm at 250 kHz, 0.238 mm at
    700 kHz), run for the transit of 1.3 x the domain depth plus 10 cycles that
    enter the FP64 amplitude window."""
    return skull_case(nx, ny, nz, dx=1500.0 / (9.0 * f0), f0=f0, n_steps=None, seed=seed,
                      dft_cycles=10)


# Config-3 grids: the same physical domain (85 x 85 x 72 mm) at 250 and 700 kHz.
CONFIG3_GRIDS = {250e3: (128, 128, 108), 700e3: (360, 360, 300)}


def thermal_regime(dx: float, materials=None) -> dict:
    """Exposure of Sec. 4.1.1 (40 s on at 30 % duty cycle, 80 s off) with the
    largest thermal step among 0.1, 0.05, 0.025 ... s that keeps the explicit
    scheme stable on every tissue, dt <= dx^2 min(rho c_th / k_th) / 6."""
    rows = np.asarray(materials if materials is not None else
                      [water_row(0.0), skin_row(0.0), brain_row(0.0)], dtype=np.float64)
    lim = dx * dx * float((rows[:, 0] * rows[:, 6] / rows[:, 5]).min()) / 6.0
    dt = 0.1
    while dt > lim:
        dt *= 0.5
    return dict(dt=dt, n_on=int(round(40.0 / dt)), n_off=int(round(80.0 / dt)), duty=0.3,
                T_a=37.0, rhob_cb=1050.0 * 3617.0)


def water_like(case: Case) -> Case:
    """The same grid, source and run filled with water only (the companion run
    used for the energy-loss factor, Sec. 2.3 / Sec. 2.4)."""
    c = Case(**{k: getattr(case, k) for k in case.__dataclass_fields__})
    c.name = case.name + "_water"
    c.index = np.zeros_like(case.index)
    c.materials = np.array([water_row(case.f0)])
    return c


def sweep_specs(n: int = 64, seed: int = 4321, n_min: int = 96, n_max: int = 200,
                ppw: float = 6.0):
    """Domains of a planning sweep: per domain, sizes drawn uniformly from
    [n_min, n_max] per axis (nx rounded up to a multiple of 16, the TMA row
    rule), a drive frequency from {250, 500, 700} kHz with dx = lambda_water /
    ppw, and a bowl tilt uniform in [-15, 15] degrees; seeded."""
    rng = np.random.default_rng(seed)
    out = []
    for d in range(n):
        nx, ny, nz = (int(v) for v in rng.integers(n_min, n_max + 1, size=3))
        nx = min(((nx + 15) // 16) * 16, ((n_max + 15) // 16) * 16)
        f0 = float(rng.choice([2.5e5, 5e5, 7e5]))
        tilt = float(rng.uniform(-15.0, 15.0))
        out.append(dict(nx=nx, ny=ny, nz=nz, f0=f0, dx=1500.0 / f0 / ppw, tilt_deg=tilt,
                        seed=int(seed) * 1000 + d))
    return out


def sweep_case(spec: dict, n_steps: int | None = None, dft_cycles: int = 10) -> Case:
    """The synthetic skull of one sweep domain (see skull_case).  The tilted
    bowl's apex is lowered so that its rim stays 2 mm below the source plane."""
    c = skull_case(spec["nx"], spec["ny"], spec["nz"], dx=spec["dx"], f0=spec["f0"],
                   n_steps=n_steps, seed=spec["seed"], tilt_deg=spec["tilt_deg"],
                   dft_cycles=dft_cycles)
    b = dict(c.bowl)
    a, R = 0.5 * b["aperture"], b["roc"]
    h = R - math.sqrt(R * R - a * a)
    t = math.radians(abs(spec["tilt_deg"]))
    top = h * math.cos(t) + a * math.sin(t)
    ax, ay, az = b["apex"]
    b["apex"] = (ax, ay, min(az, c.k_src * c.dx - 2e-3 - top))
    c.bowl = b
    return c


def fno_weights(dims: dict, seed: int, gain: float = 1.0) -> np.ndarray:
    """Seeded float32 weights in the surrogate's flat blob layout (lift, then
    per layer spectral R, pointwise W and b, then the projection), scaled by
    fan-in so that every layer keeps O(1) activations; the spectral weights
    take 1/width."""
    rng = np.random.default_rng(seed)
    ci, w, m, L, h, co = (dims["c_in"], dims["width"], dims["modes"], dims["n_layers"],
                          dims["hidden"], dims["c_out"])
    m3 = (2 * m) * (2 * m) * m
    parts = [rng.standard_normal(w * ci) * gain / np.sqrt(ci), rng.standard_normal(w) * 0.1]
    for _ in range(L):
        parts += [rng.standard_normal(m3 * w * w * 2) * gain / w,
                  rng.standard_normal(w * w) * gain / np.sqrt(w), rng.standard_normal(w) * 0.1]
    parts += [rng.standard_normal(h * w) * gain / np.sqrt(w), rng.standard_normal(h) * 0.1,
              rng.standard_normal(co * h) * gain / np.sqrt(h), rng.standard_normal(co) * 0.1]
    return np.concatenate(parts).astype(np.float32)


def fno_inputs(c_in: int, nx: int, ny: int, nz: int, seed: int) -> np.ndarray:
    """Seeded float32 feature volume [c_in, nz, ny, nx]: smooth random fields
    (sums of a few low Fourier modes) plus white noise, like material maps."""
    rng = np.random.default_rng(seed)
    z = np.arange(nz)[:, None, None] / nz
    y = np.arange(ny)[None, :, None] / ny
    x = np.arange(nx)[None, None, :] / nx
    out = np.empty((c_in, nz, ny, nx), dtype=np.float32)
    for c in range(c_in):
        f = 0.1 * rng.standard_normal((nz, ny, nx))
        for _ in range(4):
            a, b, k = rng.integers(-3, 4, size=3)
            ph = rng.uniform(0, 2 * np.pi)
            f += rng.standard_normal() * np.cos(2 * np.pi * (a * z + b * y + k * x) + ph)
        out[c] = f
    return out

