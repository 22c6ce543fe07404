"""Closed-form solutions used to pin the oracle (and, independently, the GPU path).

Each function states the mathematics it evaluates; none of them calls the
oracle or the product library.
"""
from __future__ import annotations

import numpy as np

C1, C2 = 9.0 / 8.0, -1.0 / 24.0
FIELDS = ("vx", "vy", "vz", "sxx", "syy", "szz", "sxy", "sxz", "syz")
# staggered offsets (x, y, z) in cells of each field's grid points
OFFSETS = {"vx": (0.5, 0, 0), "vy": (0, 0.5, 0), "vz": (0, 0, 0.5),
           "sxx": (0, 0, 0), "syy": (0, 0, 0), "szz": (0, 0, 0),
           "sxy": (0.5, 0.5, 0), "sxz": (0.5, 0, 0.5), "syz": (0, 0.5, 0.5)}


def staggered_symbol(k, dx):
    """Symbol of the O(4) staggered difference: D e^{-ikx} = -i K e^{-ikx},
    K = (2/dx) (c1 sin(k dx/2) + c2 sin(3 k dx/2))."""
    return (2.0 / dx) * (C1 * np.sin(k * dx / 2) + C2 * np.sin(3 * k * dx / 2))


def discrete_plane_wave(shape, dx, dt, rho, piR, mu, kvec, mode):
    """Exact plane-wave solution of the lossless staggered O(4) leapfrog scheme
    in a homogeneous isotropic medium.

    With K_a the staggered symbol per axis and Omega = (2/dt) sin(w dt/2):
    P mode (velocity along K): rho Omega^2 = pi |K|^2;
    S mode (velocity normal to K): rho Omega^2 = mu |K|^2.
    Stress amplitudes follow from the stress rate:
    sigma_ij = -(lambda delta_ij K.V + mu (K_i V_j + K_j V_i)) / Omega.
    Returns (omega, fields(t_v, t_s)) where fields() gives every component on
    its own staggered points, velocities at time t_v and stresses at t_s."""
    kvec = np.asarray(kvec, dtype=np.float64)
    K = staggered_symbol(kvec, dx)
    lam = piR - 2.0 * mu
    if mode == "P":
        Om = np.sqrt(piR / rho) * np.linalg.norm(K)
        V = K / np.linalg.norm(K)
    else:
        Om = np.sqrt(mu / rho) * np.linalg.norm(K)
        V = np.cross(K, [1.0, 0.0, 0.0])
        V /= np.linalg.norm(V)
    omega = (2.0 / dt) * np.arcsin(Om * dt / 2.0)
    sig = -(lam * np.eye(3) * (K @ V) + mu * (np.outer(K, V) + np.outer(V, K))) / Om
    amp = {"vx": V[0], "vy": V[1], "vz": V[2], "sxx": sig[0, 0], "syy": sig[1, 1],
           "szz": sig[2, 2], "sxy": sig[0, 1], "sxz": sig[0, 2], "syz": sig[1, 2]}
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")

    def fields(t_v, t_s):
        out = {}
        for f in FIELDS:
            ox, oy, oz = OFFSETS[f]
            t = t_v if f[0] == "v" else t_s
            ph = omega * t - (kvec[0] * (x + ox) + kvec[1] * (y + oy) + kvec[2] * (z + oz)) * dx
            out[f] = amp[f] * np.cos(ph)
        zero_ghost_half_points(out)
        return out

    return omega, amp, fields


def zero_ghost_half_points(f):
    """The last half-grid point of each axis (position n - 1/2) is a ghost."""
    f["vx"][:, :, -1] = 0
    f["vy"][:, -1, :] = 0
    f["vz"][-1] = 0
    f["sxy"][:, :, -1] = 0
    f["sxy"][:, -1, :] = 0
    f["sxz"][:, :, -1] = 0
    f["sxz"][-1] = 0
    f["syz"][:, -1, :] = 0
    f["syz"][-1] = 0


def sls_modulus_factor(omega, tau, tau_sigma):
    """Complex modulus factor of L standard linear solids (tau method):
    M(w) / M_R = 1 + tau sum_l i w ts_l / (1 + i w ts_l)."""
    m = 1.0 + 0j
    for ts in tau_sigma:
        m += tau * (1j * omega * ts) / (1.0 + 1j * omega * ts)
    return m


def sls_ramp_response(t, M_R, tau, tau_sigma, rate):
    """Stress of the continuous SLS under a constant strain rate switched on at
    t = 0:  sigma(t) = M_R rate [t + tau sum_l ts_l (1 - exp(-t/ts_l))]."""
    s = t.copy() if isinstance(t, np.ndarray) else t
    s = s + tau * sum(ts * (1.0 - np.exp(-t / ts)) for ts in tau_sigma)
    return M_R * rate * s


def oneil_on_axis(z, a, R, k, p0):
    """O'Neil: on-axis pressure magnitude of a spherical cap (aperture radius a,
    radius of curvature R), z from the apex:  |p| = p0 |2/(1 - z/R)| |sin(k (r_e - z)/2)|,
    r_e = sqrt((z - h)^2 + a^2), h = R - sqrt(R^2 - a^2)."""
    h = R - np.sqrt(R * R - a * a)
    re = np.sqrt((z - h) ** 2 + a * a)
    return p0 * np.abs(2.0 / (1.0 - z / R)) * np.abs(np.sin(k * (re - z) / 2.0))


def oneil_on_axis_complex(z, a, R, k, p0):
    """The on-axis Rayleigh integral of a spherical cap in closed form (the
    e^{+i w t} convention): p(z) = p0 R/(R - z) (e^{-ikz} - e^{-i k r_e})."""
    h = R - np.sqrt(R * R - a * a)
    re = np.sqrt((z - h) ** 2 + a * a)
    return p0 * R / (R - z) * (np.exp(-1j * k * z) - np.exp(-1j * k * re))


def pennes_gaussian(r2, t, theta0, s0, D, wprime):
    """Pennes equation with uniform perfusion rate w' and no source, Gaussian
    initial excess: theta = theta0 (s0^2/(s0^2 + 2Dt))^(3/2) exp(-r^2/(2(s0^2+2Dt))) exp(-w' t)."""
    s2 = s0 * s0 + 2.0 * D * t
    return theta0 * (s0 * s0 / s2) ** 1.5 * np.exp(-r2 / (2.0 * s2)) * np.exp(-wprime * t)


def lattice_wavenumber(omega, dt, dx, c):
    """theta = k dx of the propagating mode of the staggered O(4) leapfrog
    scheme: (2/dt) sin(w dt/2) = (2c/dx) (c1 sin(theta/2) + c2 sin(3 theta/2)),
    the root below the maximum of the right side (bisection)."""
    target = (2.0 / dt) * np.sin(omega * dt / 2.0) * dx / (2.0 * c)
    g = lambda th: C1 * np.sin(th / 2) + C2 * np.sin(3 * th / 2) - target
    # c1 sin(x) + c2 sin(3x) increases on [0, pi/2] for the O(4) coefficients
    lo, hi = 0.0, np.pi
    assert g(hi) > 0 >= g(lo)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if g(mid) > 0:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def soft_source_far_field(S, d, omega, dt, dx, c):
    """Far field of a soft pressure source on one plane of the staggered O(4)
    leapfrog scheme in a homogeneous fluid (exact for the discrete scheme).

    The source adds 2 c S/dx to the pressure rate of its plane at half steps
    (complex amplitude S, e^{+i w t} convention).  Taking the lattice Fourier
    transform along the axis, the pressure is P(theta) = i s Omega /
    (c^2 K(theta)^2 - Omega^2) with Omega = (2/dt) sin(w dt/2); the outgoing
    pole at the lattice wavenumber theta_d gives, |d| cells away,
    P(d) = S e^{-i theta_d |d|} / (c1 cos(theta_d/2) + 3 c2 cos(3 theta_d/2))
    (evanescent roots of the 4th-order stencil decay within a few cells)."""
    th = lattice_wavenumber(omega, dt, dx, c)
    g = C1 * np.cos(th / 2) + 3 * C2 * np.cos(3 * th / 2)
    return S * np.exp(-1j * th * np.abs(d)) / g
