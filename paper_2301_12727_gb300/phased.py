"""Multi-element phased sources over the C ABI: element layouts, steering
weights and time-reversal (phase-conjugation) refocusing.

The paper plans with single-element bowls (Sec. 2); these helpers serve
steered and aberration-corrected planning with a user-supplied element
layout.  Every field is computed by the library (bvf_rs_elements, the FDTD
kernels); this module builds element tables and sequences calls.
"""
from __future__ import annotations

import math

import numpy as np

from . import bvf


def bowl_array(aperture: float, roc: float, apex, direction=(0.0, 0.0, 1.0), n_rings: int = 8,
               n_inner: int = 6) -> np.ndarray:
    """Elements on a spherical cap (aperture diameter, radius of curvature,
    apex, unit axis): ring r (of n_rings rings of equal polar-angle width)
    holds n_inner * (r + 1) equal elements; each element carries the area of
    its patch.  Returns rows (x, y, z, area, 1, 0)."""
    a, R = 0.5 * aperture, roc
    thmax = math.asin(a / R)
    u = np.asarray(direction, dtype=np.float64)
    u = u / np.linalg.norm(u)
    # rotation taking +z to u (Rodrigues, about z x u)
    kx, ky = -u[1], u[0]
    sn, cs = math.hypot(kx, ky), u[2]
    if sn > 0.0:
        kx, ky = kx / sn, ky / sn
    rows = []
    for r in range(n_rings):
        t0, t1 = thmax * r / n_rings, thmax * (r + 1) / n_rings
        tc = 0.5 * (t0 + t1)
        m = n_inner * (r + 1)
        area = 2.0 * math.pi * R * R * (math.cos(t0) - math.cos(t1)) / m
        for e in range(m):
            ph = 2.0 * math.pi * (e + 0.5) / m
            p = np.array([R * math.sin(tc) * math.cos(ph), R * math.sin(tc) * math.sin(ph),
                          R * (1.0 - math.cos(tc))])
            kdp = kx * p[0] + ky * p[1]
            cr = np.array([ky * p[2], -kx * p[2], kx * p[1] - ky * p[0]])
            q = p * cs + cr * sn + np.array([kx, ky, 0.0]) * kdp * (1.0 - cs)
            rows.append([apex[0] + q[0], apex[1] + q[1], apex[2] + q[2], area, 1.0, 0.0])
    return np.array(rows)


def steer(elements: np.ndarray, target, f0: float, c0: float = 1500.0) -> np.ndarray:
    """Phase every element so that its wave arrives at `target` in phase with
    the others (geometric delays in a medium of speed c0): w_e = exp(+i k r_te)."""
    el = np.array(elements, dtype=np.float64)
    k = 2.0 * math.pi * f0 / c0
    r = np.linalg.norm(el[:, :3] - np.asarray(target, dtype=np.float64), axis=1)
    w = np.exp(1j * k * r)
    el[:, 4], el[:, 5] = w.real, w.imag
    return el


def time_reversal_plane(solver: "bvf.Solver", target_ijk, k_src: int, f0: float, dt: float,
                        n_steps: int, c0: float = 1500.0):
    """Phase-conjugation refocusing through the solver's medium: a CW point
    source at the target voxel (i, j, k) is run to steady state, the complex
    amplitude P it leaves on source plane k_src is captured over the last two
    periods (FP64 DFT), and conj(P), normalised to a largest magnitude of 1,
    is returned as a complex (ny, nx) array to drive that plane.  The solver's
    state and capture are reset before and after."""
    import torch
    nz, ny, nx = solver.shape
    i, j, k = target_ijk
    M = int(round(1.0 / (f0 * dt)))
    src = np.zeros((ny, nx), dtype=np.complex128)
    src[j, i] = 1.0
    solver.reset()
    solver.set_source(src, k, c0, bvf.BVF_ENV_RAMP_CW)
    solver.run(n_steps, dft_start=n_steps - 2 * M + 1, dft_steps=2 * M)
    solver.synchronize()
    amp, ph = solver.amp_phase()
    P = (amp[k_src] * torch.exp(1j * ph[k_src])).cpu().numpy()
    solver.reset()
    m = np.abs(P).max()
    return np.conj(P) / m if m > 0 else P
