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

With `cpml` given, each derivative normal to an absorbing slab is replaced
by df + psi, psi <- b psi + a df. (a, b) are the Komatitsch-Martin profile
(kappa = 1, d = d0 xi^2, alpha = pi f0 (1 - xi)), taken at the integer point
for a D- derivative and at the half point for a D+ one.  The 18 psi arrays
follow the state's ordering: (vx, vy, vz) x (x, y, z); the normal strains;
then the shear pairs xy (y, x), xz (z, x), yz (z, y).  The per-material
relaxed moduli and tau come from the oracle's fit, which is pinned separately
(Q and phase speed).
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


def cpml_profile(n, P, h, dt, f0, R, cmax, half):
    """(a, b) along an axis of n points at the integer (half=False) or half
    points; zero outside the two slabs of P cells."""
    pos2 = 2.0 * np.arange(n) + (1.0 if half else 0.0)
    xi = np.maximum((2.0 * P - pos2) / (2.0 * P), (pos2 - 2.0 * (n - 1 - P)) / (2.0 * P))
    inside = xi > 0.0
    xi = np.clip(xi, 0.0, 1.0)
    d = (-3.0 * cmax * np.log(R) / (2.0 * P * h)) * xi * xi
    al = np.pi * f0 * (1.0 - xi)
    b = np.where(inside, np.exp(-(d + al) * dt), 0.0)
    with np.errstate(invalid="ignore", divide="ignore"):
        a = np.where(inside & (d + al > 0.0), d * (b - 1.0) / (d + al), 0.0)
    return a, b


def step(state, index, rho, coef, ts, dt, h, n, src=None, k_src=0, c0=1500.0, f0=5e5,
         env=None, cpml=None):
    """Advance state [9 + 6L (+18 psi)][nz][ny][nx] by one step n -> n+1 (new
    array).  cpml: dict (P, R, cmax) for absorbing slabs of P cells."""
    st = state.copy()
    L = len(ts)
    shape = index.shape
    prof = {}
    if cpml is not None:
        for axis in range(3):
            for half in (False, True):
                a, b = cpml_profile(shape[axis], cpml["P"], h, dt, f0, cpml["R"], cpml["cmax"], half)
                bshape = [1, 1, 1]
                bshape[axis] = shape[axis]
                prof[(axis, half)] = (a.reshape(bshape), b.reshape(bshape))

    def absorb(df, q, axis, half, mask=None):
        """df + psi with psi_q updated where the slab coefficients are non-zero."""
        if cpml is None:
            return df
        a, b = prof[(axis, half)]
        a, b = np.broadcast_to(a, shape), np.broadcast_to(b, shape)
        psi = st[9 + 6 * L + q]
        active = (a != 0.0) | (b != 0.0)
        if mask is not None:
            active = active & mask
        new = b * psi + a * df
        psi[active] = new[active]
        return np.where(active, df + new, df)
    vx, vy, vz = st[0], st[1], st[2]
    sxx, syy, szz, sxy, sxz, syz = st[3], st[4], st[5], st[6], st[7], st[8]
    r = st[9:9 + 6 * L].reshape(L, 6, *shape)
    rv = rho[index]
    piR, muR, tP, tS = (coef[:, c][index] for c in range(4))

    # velocities (faces s + 1/2; the last face of each axis is a ghost).  Each
    # term: (derivative, psi slot, axis, taken at the half point)
    for comp, axis, q0, terms in (
            (vx, 2, 0, ((d_plus(sxx, 2, h), 2, True), (d_minus(sxy, 1, h), 1, False),
                        (d_minus(sxz, 0, h), 0, False))),
            (vy, 1, 3, ((d_minus(sxy, 2, h), 2, False), (d_plus(syy, 1, h), 1, True),
                        (d_minus(syz, 0, h), 0, False))),
            (vz, 0, 6, ((d_minus(sxz, 2, h), 2, False), (d_minus(syz, 1, h), 1, False),
                        (d_plus(szz, 0, h), 0, True)))):
        m = _below_last(shape, axis)
        t = [absorb(df, q0 + i, ax, half, m) for i, (df, ax, half) in enumerate(terms)]
        b = 2.0 / (rv + _next(rv, axis))
        upd = comp + dt * b * ((t[0] + t[1]) + t[2])
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
    e = (absorb(d_minus(vx, 2, h), 9, 2, False), absorb(d_minus(vy, 1, h), 10, 1, False),
         absorb(d_minus(vz, 0, h), 11, 0, False))
    th = (e[0] + e[1]) + e[2]
    for c, sig in enumerate((sxx, syy, szz)):
        dev = th - e[c]
        Psi = piR * (1.0 + L * tP) * th - 2.0 * muR * (1.0 + L * tS) * dev
        The = piR * tP * th - 2.0 * muR * tS * dev
        sig += dt * (Psi + 0.5 * relax(c, The))

    # shear stresses on the edges: (component, first axis, second axis, strain)
    def shear_strain(c, a1, a2):
        m = _below_last(shape, a1) & _below_last(shape, a2)
        if c == 3:
            return (absorb(d_plus(vx, 1, h), 12, 1, True, m) +
                    absorb(d_plus(vy, 2, h), 13, 2, True, m))
        if c == 4:
            return (absorb(d_plus(vx, 0, h), 14, 0, True, m) +
                    absorb(d_plus(vz, 2, h), 15, 2, True, m))
        return (absorb(d_plus(vy, 0, h), 16, 0, True, m) +
                absorb(d_plus(vz, 1, h), 17, 1, True, m))

    for c, sig, a1, a2 in ((3, sxy, 2, 1), (4, sxz, 2, 0), (5, syz, 1, 0)):
        ev = shear_strain(c, a1, a2)
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


def bhte_run(T0, index, mat, h, amp, p_scale, dt, n_on, n_off, duty, T_a=37.0,
             rhob_cb=1050.0 * 3617.0):
    """Pennes BHTE in array form (Sec. 2.4): forward Euler, 7-point stencil
    with the harmonic-mean face conductivity, borders held at T_a, perfusion,
    the duty-cycled source during the first n_on steps, then T_max and CEM43
    (R = 0.5 at T >= 43, else 0.25) after every step.  Returns (T, Tmax, cem)."""
    rho, cL, aL = mat[:, 0][index], mat[:, 1][index], mat[:, 3][index]
    k, cth, perf, heat = (mat[:, c][index] for c in (5, 6, 7, 8))
    Q = heat * aL * (p_scale * amp) ** 2 / (rho * cL)
    border = np.zeros(index.shape, dtype=bool)
    border[0], border[-1] = True, True
    border[:, 0], border[:, -1] = True, True
    border[:, :, 0], border[:, :, -1] = True, True
    T = T0.copy()
    Tmax, cem = T.copy(), np.zeros(index.shape)
    inv_h2 = 1.0 / (h * h)
    for n in range(n_on + n_off):
        dc = duty if n < n_on else 0.0
        lap = np.zeros(index.shape)
        # faces in the order -x, +x, -y, +y, -z, +z (np.roll wraps only at the
        # borders, which are overwritten below)
        for axis, shift in ((2, 1), (2, -1), (1, 1), (1, -1), (0, 1), (0, -1)):
            kn = np.roll(k, shift, axis=axis)
            Tn_b = np.roll(T, shift, axis=axis)
            lap = lap + (2.0 * k * kn / (k + kn)) * (Tn_b - T)
        rhs = lap * inv_h2 - perf * rhob_cb * (T - T_a) + dc * Q
        Tn = T + dt * rhs / (rho * cth)
        Tn[border] = T_a
        T = Tn
        Tmax = np.maximum(Tmax, T)
        R = np.where(T >= 43.0, 0.5, 0.25)
        cem = cem + dt / 60.0 * np.power(R, 43.0 - T)
    return T, Tmax, cem
