"""Multi-element phased sources over the C ABI: element layouts, steering
weights and time-reversal (phase-conjugation) refocusing.

The paper plans with single-element bowls (Sec. 2); these helpers serve
steered and aberration-corrected planning with a user-supplied element
layout.  Every number is computed by the library (bvf_bowl_array,
bvf_steer_weights, bvf_rs_elements, bvf_time_reversal_plane); this module only
marshals arguments.
"""
from __future__ import annotations

from . import bvf


def bowl_array(aperture: float, roc: float, apex, direction=(0.0, 0.0, 1.0), n_rings: int = 8,
               n_inner: int = 6):
    """Elements on a spherical cap (aperture diameter, radius of curvature,
    apex, unit axis): ring r (of n_rings rings of equal polar-angle width)
    holds n_inner * (r + 1) equal elements; each element carries the area of
    its patch.  Returns rows (x, y, z, area, 1, 0)."""
    bowl = bvf.Bowl(aperture, roc, tuple(float(v) for v in apex),
                    tuple(float(v) for v in direction), 0.0, 1500.0, 0.0)
    return bvf.bvf_bowl_array(bowl, n_rings, n_inner)


def steer(elements, target, f0: float, c0: float = 1500.0):
    """Phase every element so that its wave arrives at `target` in phase with
    the others (geometric delays in a medium of speed c0): w_e = exp(+i k r_te)."""
    return bvf.bvf_steer_weights(elements, target, f0, c0)


def time_reversal_plane(solver: "bvf.Solver", target_ijk, k_src: int, n_steps: int,
                        c0: float = 1500.0):
    """Phase-conjugation refocusing through the solver's medium: a CW point
    source at the target voxel (i, j, k) runs n_steps steps, and the
    conjugate of the complex amplitude it leaves on plane k_src over the last
    two periods, normalised to a largest magnitude of 1, comes back as a
    float32 CUDA tensor (ny, nx, 2) ready for Solver.set_source.  The solver's
    state, capture and source are reset."""
    import torch
    nz, ny, nx = solver.shape
    out = torch.empty((ny, nx, 2), dtype=torch.float32, device="cuda")
    bvf.bvf_time_reversal_plane(solver.ctx, target_ijk, k_src, n_steps, c0, out)
    return out
