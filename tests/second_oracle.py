"""A second FP64 implementation of the acoustic step, in array form (numpy),
used to pin the index conventions of the C oracle on small grids.

It is written from the scheme's definition, not from the C loops:

* zero ghosts: every field is padded by two zero layers per side;
* the last half point of each axis is a ghost that is never updated;
* D+ and D- are the 4th-order staggered differences (c1 = 9/8, c2 = -1/24)
  taken at s + 1/2 and at s;
* buoyancy 2/(rho_a + rho_b) on the velocity faces;
* on the shear edges, the harmonic mean of mu over the four cells (0 if any
  is 0) and the mean of tau_S;
* Crank-Nicolson memory variables;
* the soft stress source at (n + 1/2) dt.

CPML is left out (n_pml = 0). The per-material relaxed moduli and tau come
from the oracle's fit, which is pinned separately (Q and phase speed).
"""
from __future__ import annotations

import numpy as np

C1, C2 = 9.0 / 8.0, -1.0 / 24.0


def _pad(f):
    return np.pad(f, 2)


def _s(F, dz, dy, dx, shape):
    """View of the padded field F shifted by (dz, dy, dx) over the interior."""
    nz, ny, nx = shape
    return F[2 + dz:2 + dz + nz, 2 + dy:2 + dy + ny, 2 + dx:2 + dx + nx]


def d_plus(f, axis, h):
    """(c1 (f[s+1] - f[s]) + c2 (f[s+2] - f[s-1])) / h along axis (0 z, 1 y, 2 x)."""
    F, sh = _pad(f), f.shape

    def at(o):
        d = [0, 0, 0]
        d[axis] = o
        return _s(F, d[0], d[1], d[2], sh)
    return (C1 * (at(1) - at(0)) + C2 * (at(2) - at(-1))) / h


def d_minus(f, axis, h):
    """(c1 (f[s] - f[s-1]) + c2 (f[s+1] - f[s-2])) / h along axis."""
    F, sh = _pad(f), f.shape

    def at(o):
        d = [0, 0, 0]
        d[axis] = o
        return _s(F, d[0], d[1], d[2], sh)
    return (C1 * (at(0) - at(-1)) + C2 * (at(1) - at(-2))) / h


def _next(a, axis):
    """a at s + 1 along axis (edge-replicated beyond the end; only used where masked)."""
    idx = [slice(None)] * 3
    out = np.empty_like(a)
    idx[axis] = slice(0, -1)
    src = [slice(None)] * 3
    src[axis] = slice(1, None)
    out[tuple(idx)] = a[tuple(src)]
    last = [slice(None)] * 3
    last[axis] = slice(-1, None)
    out[tuple(last)] = a[tuple(last)]
    return out


def _below_last(shape, axis):
    m = np.ones(shape, dtype=bool)
    idx = [slice(None)] * 3
    idx[axis] = -1
    m[tuple(idx)] = False
    return m


def step(state, index, rho, coef, ts, dt, h, n, src=None, k_src=0, c0=1500.0, f0=5e5,
         env=None):
    """Advance state [9 + 6L][nz][ny][nx] by one step n -> n+1 (new array)."""
    st = state.copy()
    L = len(ts)
    shape = index.shape
    vx, vy, vz = st[0], st[1], st[2]
    sxx, syy, szz, sxy, sxz, syz = st[3], st[4], st[5], st[6], st[7], st[8]
    r = st[9:9 + 6 * L].reshape(L, 6, *shape)
    rv = rho[index]
    piR, muR, tP, tS = (coef[:, c][index] for c in range(4))

    # velocities (faces s + 1/2; the last face of each axis is a ghost)
    for comp, axis, terms in ((vx, 2, (d_plus(sxx, 2, h), d_minus(sxy, 1, h), d_minus(sxz, 0, h))),
                              (vy, 1, (d_minus(sxy, 2, h), d_plus(syy, 1, h), d_minus(syz, 0, h))),
                              (vz, 0, (d_minus(sxz, 2, h), d_minus(syz, 1, h), d_plus(szz, 0, h)))):
        b = 2.0 / (rv + _next(rv, axis))
        upd = comp + dt * b * ((terms[0] + terms[1]) + terms[2])
        m = _below_last(shape, axis)
        comp[m] = upd[m]

    hh = dt / (2.0 * np.asarray(ts))
    ca = (1.0 - hh) / (1.0 + hh)
    cb = (dt / np.asarray(ts)) / (1.0 + hh)

    def relax(c, The):
        total = np.zeros(shape)
        for l in range(L):
            rn = ca[l] * r[l, c] - cb[l] * The
            total = total + (rn + r[l, c])
            r[l, c] = rn
        return total

    # normal stresses at the cell centres
    e = (d_minus(vx, 2, h), d_minus(vy, 1, h), d_minus(vz, 0, h))
    th = (e[0] + e[1]) + e[2]
    for c, sig in enumerate((sxx, syy, szz)):
        dev = th - e[c]
        Psi = piR * (1.0 + L * tP) * th - 2.0 * muR * (1.0 + L * tS) * dev
        The = piR * tP * th - 2.0 * muR * tS * dev
        sig += dt * (Psi + 0.5 * relax(c, The))

    # shear stresses on the edges: (component, first axis, second axis, strain)
    for c, sig, a1, a2, ev in ((3, sxy, 2, 1, d_plus(vx, 1, h) + d_plus(vy, 2, h)),
                               (4, sxz, 2, 0, d_plus(vx, 0, h) + d_plus(vz, 2, h)),
                               (5, syz, 1, 0, d_plus(vy, 0, h) + d_plus(vz, 1, h))):
        u00, t00 = muR, tS
        u10, t10 = _next(muR, a1), _next(tS, a1)
        u01, t01 = _next(muR, a2), _next(tS, a2)
        u11, t11 = _next(_next(muR, a1), a2), _next(_next(tS, a1), a2)
        allpos = (u00 > 0) & (u10 > 0) & (u01 > 0) & (u11 > 0)
        with np.errstate(divide="ignore"):
            muh = np.where(allpos, 4.0 / ((1.0 / u00 + 1.0 / u10) + (1.0 / u01 + 1.0 / u11)), 0.0)
        tsh = 0.25 * ((t00 + t10) + (t01 + t11))
        Psi = muh * (1.0 + L * tsh) * ev
        The = muh * tsh * ev
        m = _below_last(shape, a1) & _below_last(shape, a2)
        r_before = r[:, c].copy()
        total = relax(c, The)
        upd = sig + dt * (Psi + 0.5 * total)
        sig[m] = upd[m]
        r[:, c][:, ~m] = r_before[:, ~m]       # edges on a ghost keep their memory

    # soft stress source on plane k_src at t = (n + 1/2) dt
    if src is not None and env is not None:
        t = (n + 0.5) * dt
        A, phi = np.abs(src), np.angle(src)
        sv = env(t) * A * np.sin(2.0 * np.pi * f0 * t + phi)
        for sig in (sxx, syy, szz):
            sig[k_src] -= (2.0 * c0 * dt / h) * sv
    return st
