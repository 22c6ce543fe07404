"""Pins of the FP64 oracle against closed forms, invariants and special cases.

Each test pins the oracle to something other than itself: exact solutions of
the discrete scheme, conserved quantities, continuum physics within the
scheme's error, or textbook formulas.  A plausible slip in the oracle (a
dropped term, a wrong sign, index or staggering offset, a transposed operand)
fails at least one of them.
"""
import math

import numpy as np
import pytest

from tests import analytic as an

F0 = 5e5


def mat_row(rho, cL, cS=0.0, aL=0.0, aS=0.0, k=0.5, c=3600.0, perf=0.0, heat=1.0):
    return [rho, cL, cS, aL, aS, k, c, perf, heat]


def load_fields(A, fields):
    for f in an.FIELDS:
        A.field(f)[...] = fields[f]


# --------------------------------------------------------------------------
# Eq. 1 + Sec. 2.3 scheme: exact discrete plane waves
# --------------------------------------------------------------------------
@pytest.mark.parametrize("cL,cS,mode", [(1500.0, 0.0, "P"), (2800.0, 1400.0, "P"),
                                        (2800.0, 1400.0, "S")])
def test_discrete_plane_wave_is_exact(orc, cL, cS, mode):
    """An oblique plane wave obeying the O(4) staggered dispersion relation
    rho (2/dt sin(w dt/2))^2 = M |K|^2 is reproduced to rounding inside the
    region the zero-ghost walls cannot reach in s steps (3 cells per step)."""
    n, dx, rho = 40, 1e-3, 1000.0
    dt = 0.3 * dx / cL
    kvec = np.array([2 * np.pi / (7 * dx), 2 * np.pi / (9 * dx), 2 * np.pi / (11 * dx)])
    A = orc.Acoustic(n, n, n, dx, dt, np.zeros((n, n, n)), [mat_row(rho, cL, cS)], F0,
                     n_sls=2, n_pml=0)
    om, amp, fields = an.discrete_plane_wave((n, n, n), dx, dt, rho, rho * cL ** 2,
                                             rho * cS ** 2, kvec, mode)
    load_fields(A, fields(-0.5 * dt, 0.0))
    s = 4
    assert A.run(s) == 0
    ex = fields((s - 0.5) * dt, s * dt)
    m = 3 * s + 3
    sl = (slice(m, n - m),) * 3
    vscale = max(abs(amp[f]) for f in an.FIELDS if f[0] == "v")
    sscale = max(abs(amp[f]) for f in an.FIELDS if f[0] == "s")
    for f in an.FIELDS:
        err = np.abs(A.field(f)[sl] - ex[f][sl]).max() / (vscale if f[0] == "v" else sscale)
        assert err < 1e-11, (f, err)
    # the continuum would differ by a visible amount: the pin discriminates
    om_cont = np.sqrt((rho * cL ** 2 if mode == "P" else rho * cS ** 2) / rho) * np.linalg.norm(kvec)
    assert abs(om / om_cont - 1) > 1e-4


def test_dispersion_discriminates_wrong_coefficients():
    """Second-order coefficients (1, 0) or swapped (c2, c1) give a different
    symbol, so the plane-wave pin would fail for them."""
    k, dx = 2 * np.pi / 6e-3, 1e-3
    K4 = an.staggered_symbol(k, dx)
    K2 = (2 / dx) * np.sin(k * dx / 2)
    assert abs(K4 / K2 - 1) > 1e-3
    assert abs(K4 / k - 1) < 1e-2       # 4th order: within 1 % of k at 6 PPW
    assert abs(K2 / k - 1) > 2e-2       # 2nd order: off by more than 2 %


# --------------------------------------------------------------------------
# Energy conservation (lossless, heterogeneous, zero ghosts = closed box)
# --------------------------------------------------------------------------
def _energy(orc, A, before, after, coef, index):
    """E^n = 1/2 sum rho_bar v^{n+1/2}.v^{n-1/2} + W(sigma^n)."""
    rho = A.mat[:, 0][index]
    piR, mu = coef[:, 0][index], coef[:, 1][index]
    kin = 0.0
    rb = 0.5 * (rho[:, :, :-1] + rho[:, :, 1:])
    kin += np.sum(rb * before["vx"][:, :, :-1] * after["vx"][:, :, :-1])
    rb = 0.5 * (rho[:, :-1, :] + rho[:, 1:, :])
    kin += np.sum(rb * before["vy"][:, :-1, :] * after["vy"][:, :-1, :])
    rb = 0.5 * (rho[:-1] + rho[1:])
    kin += np.sum(rb * before["vz"][:-1] * after["vz"][:-1])
    sm = (before["sxx"] + before["syy"] + before["szz"]) / 3.0
    K = piR - 4.0 * mu / 3.0
    W = np.sum(sm * sm / (2 * K))
    dev = (before["sxx"] - sm) ** 2 + (before["syy"] - sm) ** 2 + (before["szz"] - sm) ** 2
    solid = mu > 0
    W += np.sum(dev[solid] / (4 * mu[solid]))
    assert np.abs(dev[~solid]).max(initial=0) < 1e-20 * max(1.0, np.abs(sm).max())

    def hmean(u00, u10, u01, u11):
        out = np.zeros_like(u00)
        ok = (u00 > 0) & (u10 > 0) & (u01 > 0) & (u11 > 0)
        out[ok] = 4.0 / (1 / u00[ok] + 1 / u10[ok] + 1 / u01[ok] + 1 / u11[ok])
        return out
    for name, mh in (("sxy", hmean(mu[:, :-1, :-1], mu[:, :-1, 1:], mu[:, 1:, :-1], mu[:, 1:, 1:])),
                     ("sxz", hmean(mu[:-1, :, :-1], mu[:-1, :, 1:], mu[1:, :, :-1], mu[1:, :, 1:])),
                     ("syz", hmean(mu[:-1, :-1, :], mu[:-1, 1:, :], mu[1:, :-1, :], mu[1:, 1:, :]))):
        s = before[name]
        s = s[:, :-1, :-1] if name == "sxy" else (s[:-1, :, :-1] if name == "sxz" else s[:-1, :-1, :])
        pos = mh > 0
        W += np.sum(s[pos] ** 2 / (2 * mh[pos]))
        assert np.abs(s[~pos]).max(initial=0) == 0.0     # no shear stress in fluids
    return 0.5 * kin + W


def test_energy_conserved_in_lossless_heterogeneous_box(orc):
    """With zero ghosts the restricted D+ and D- are exact negative adjoints, so
    the leapfrog energy is conserved to rounding, for any heterogeneous
    layout of fluids and solids (this pins the staggering, the pairing of
    stress components with derivatives, and the material averaging)."""
    n, dx = 18, 1e-3
    rng = np.random.default_rng(7)
    mats = [mat_row(1000.0, 1500.0), mat_row(1850.0, 2800.0, 1500.0),
            mat_row(1700.0, 2300.0, 1200.0), mat_row(1100.0, 1600.0)]
    blocks = rng.integers(0, 4, size=(3, 3, 3))
    index = np.kron(blocks, np.ones((6, 6, 6), dtype=np.int64)).astype(np.uint8)
    dt = 0.8 * orc.courant_limit() * dx / 2800.0
    A = orc.Acoustic(n, n, n, dx, dt, index, mats, F0, n_sls=2, n_pml=0)
    for f in ("vx", "vy", "vz"):
        A.field(f)[...] = rng.standard_normal((n, n, n))
    fz = {f: A.field(f).copy() for f in an.FIELDS}
    an.zero_ghost_half_points(fz)
    load_fields(A, fz)
    rc, coef, _ = orc.material_coefs(mats, F0, 1.0, 2)
    assert rc == 0
    energies = []
    for _ in range(150):
        before = {f: A.field(f).copy() for f in an.FIELDS}
        assert A.run(1) == 0
        after = {f: A.field(f).copy() for f in an.FIELDS}
        energies.append(_energy(orc, A, before, after, coef, index))
    e = np.array(energies)
    assert np.abs(e / e[0] - 1).max() < 1e-11
    # the fields really moved (the check is not vacuous)
    assert np.abs(A.field("sxx")).max() > 1e3


# --------------------------------------------------------------------------
# SLS memory variables (Sec. 3.2: relaxation constants matched to Q)
# --------------------------------------------------------------------------
def _sls_ramp_errors(orc, dt_div):
    """Homogeneous slow solid driven by a linear velocity field: in the
    interior the stresses follow the continuous SLS ramp response."""
    n, dx, rho = 26, 1e-3, 1000.0
    cL, cS = 30.0, 15.0
    QP, QS = 10.0, 8.0
    w = 2 * np.pi * F0
    aL, aS = w / (2 * cL * QP), w / (2 * cS * QS)
    mats = [mat_row(rho, cL, cS, aL, aS)]
    rc, coef, ts = orc.material_coefs(mats, F0, 1.0, 2)
    assert rc == 0
    dt = ts.min() / dt_div
    nsteps = int(round(3 * ts.max() / dt))
    A = orc.Acoustic(n, n, n, dx, dt, np.zeros((n, n, n)), mats, F0, n_sls=2, n_pml=0)
    g, gp = 1.0, 0.7
    x = (np.arange(n) + 0.5 - (n - 1) / 2) * dx
    y = (np.arange(n) - (n - 1) / 2) * dx
    A.field("vx")[...] = g * x[None, None, :] + gp * y[None, :, None]
    A.field("vx")[:, :, -1] = 0.0
    assert A.run(nsteps) == 0
    t = nsteps * dt
    piR, muR, tP, tS = coef[0]
    c = slice(n // 2 - 2, n // 2 + 2)
    sxx = an.sls_ramp_response(t, piR, tP, ts, g)
    syy = an.sls_ramp_response(t, piR, tP, ts, g) - 2 * an.sls_ramp_response(t, muR, tS, ts, g)
    sxy = an.sls_ramp_response(t, muR, tS, ts, gp)
    got = {"sxx": A.field("sxx")[c, c, c], "syy": A.field("syy")[c, c, c],
           "szz": A.field("szz")[c, c, c], "sxy": A.field("sxy")[c, c, c]}
    return {"sxx": np.abs(got["sxx"] / sxx - 1).max(), "syy": np.abs(got["syy"] / syy - 1).max(),
            "szz": np.abs(got["szz"] / syy - 1).max(), "sxy": np.abs(got["sxy"] / sxy - 1).max()}


def test_sls_ramp_response_matches_continuum_second_order(orc):
    """sigma(t) = M_R rate [t + tau sum ts (1 - e^{-t/ts})] with pi/mu, tau_P/tau_S
    in the right places; the trapezoidal (Crank-Nicolson) update converges at
    second order in dt."""
    e1 = _sls_ramp_errors(orc, 10)
    e2 = _sls_ramp_errors(orc, 20)
    for k in e1:
        assert e1[k] < 2e-3, (k, e1)
        assert e2[k] < e1[k] / 3.0, (k, e1[k], e2[k])   # ~4x per halving


@pytest.mark.parametrize("L", [1, 2, 3])
@pytest.mark.parametrize("c,alpha,qc", [(2800.0, 85.0, 1.0), (1500.0, 20.0, 3.0), (2300.0, 81.0, 0.6)])
def test_q_fit_reaches_target_q_and_phase_speed(orc, L, c, alpha, qc):
    """Eq. 3 (Q = w/(2 c alpha)) with Q = Q0 q_c: the fitted tau gives
    Re M / Im M = Q at f0 and the relaxed modulus gives phase speed c at f0."""
    rho = 1800.0
    rc, coef, ts = orc.material_coefs([mat_row(rho, c, 0.0, alpha)], F0, qc, L)
    if rc != 0:
        pytest.skip("Q below the reach of %d mechanisms" % L)
    w = 2 * np.pi * F0
    piR, _, tP, _ = coef[0]
    M = piR * an.sls_modulus_factor(w, tP, ts)
    assert M.real / M.imag == pytest.approx(qc * w / (2 * c * alpha), rel=1e-12)
    k = w * np.sqrt(rho / M)
    assert w / k.real == pytest.approx(c, rel=1e-12)


def test_q_fit_rejects_unreachable_q(orc):
    """Two mechanisms at f0/3 and 3 f0 cannot reach Q < 5/3: rejected, not clipped."""
    w = 2 * np.pi * F0
    c = 2800.0
    alpha = w / (2 * c * 1.5)
    rc, _, _ = orc.material_coefs([mat_row(1800.0, c, 0.0, alpha)], F0, 1.0, 2)
    assert rc == orc.E_MATERIAL


@pytest.mark.parametrize("row", [
    mat_row(0.0, 1500.0), mat_row(1000.0, 0.0), mat_row(1000.0, 1500.0, -1.0),
    mat_row(1000.0, 1500.0, 1400.0),           # nu < -1
    mat_row(1000.0, 1500.0, 0.0, -1.0), mat_row(1000.0, 1500.0, k=0.0),
    mat_row(1000.0, 1500.0, heat=1.5)])
def test_material_validation(orc, row):
    """rho, speeds, attenuation and thermal constants must be physical; the
    Poisson ratio must lie in [-1, 0.5] (Sec. 3.2)."""
    rc, _, _ = orc.material_coefs([row], F0, 1.0, 2)
    assert rc == orc.E_MATERIAL


def test_point_source_attenuation_matches_sls(orc):
    """A CW point source in a homogeneous SLS fluid: |p| r decays as
    exp(-alpha r) with alpha = Im k, k = w sqrt(rho / M(w)) (the lossless run
    removes the grid's own geometric-spreading error)."""
    f0, dx, n, P = 3e5, 0.5e-3, 56, 8
    c, rho, alpha_in = 1500.0, 1000.0, 50.0
    from paper_2301_12727_gb300 import synth
    dt, M = synth.choose_dt(dx, c, f0)
    ks, r1, r2 = 12, 6, 24
    amps = {}
    for a in (alpha_in, 0.0):
        mats = [mat_row(rho, c, 0.0, a)]
        A = orc.Acoustic(n, n, n, dx, dt, np.zeros((n, n, n)), mats, f0, n_sls=2, n_pml=P)
        plane = np.zeros((n, n), complex)
        plane[n // 2, n // 2] = 1.0
        A.set_source(plane, ks, c, orc.ENV_RAMP_CW)
        ncyc, nd = 9, 4
        nsteps = ncyc * M
        assert A.run(nsteps, dft_start=nsteps - nd * M + 1, dft_steps=nd * M) == 0
        amp, _ = A.amp_phase(nd * M)
        amps[a] = (amp[ks + r1, n // 2, n // 2], amp[ks + r2, n // 2, n // 2])
    ratio = lambda t: math.log(t[0] * r1 / (t[1] * r2))
    alpha_meas = (ratio(amps[alpha_in]) - ratio(amps[0.0])) / ((r2 - r1) * dx)
    rc, coef, ts = orc.material_coefs([mat_row(rho, c, 0.0, alpha_in)], f0, 1.0, 2)
    w = 2 * np.pi * f0
    Mw = coef[0, 0] * an.sls_modulus_factor(w, coef[0, 2], ts)
    alpha_exact = abs((w * np.sqrt(rho / Mw)).imag)
    assert alpha_meas == pytest.approx(alpha_exact, rel=0.02)
    assert alpha_exact == pytest.approx(alpha_in, rel=0.01)


# --------------------------------------------------------------------------
# Interfaces: normal-incidence reflection (Z2 - Z1)/(Z2 + Z1)
# --------------------------------------------------------------------------
def test_normal_incidence_reflection_water_cortical(orc):
    """Plane burst from water onto a cortical half-space (rho 1850, cL 2800):
    R = (Z2 - Z1)/(Z2 + Z1) = 0.5509.  The reflected pulse is the difference
    between runs with and without the solid (lateral-edge effects cancel)."""
    f0, dx = 5e5, 0.25e-3
    nx = ny = 32
    nz, P = 160, 8
    from paper_2301_12727_gb300 import synth
    dt, M = synth.choose_dt(dx, 2800.0, f0)
    ks, krec, kint = 20, 50, 80
    traces = {}
    for solid in (True, False):
        mats = [mat_row(1000.0, 1500.0), mat_row(1850.0, 2800.0, 1500.0)]
        index = np.zeros((nz, ny, nx), np.uint8)
        if solid:
            index[kint:] = 1
        A = orc.Acoustic(nx, ny, nz, dx, dt, index, mats, f0, n_sls=2, n_pml=P)
        A.set_source(np.ones((ny, nx)), ks, 1500.0, orc.ENV_BURST, 3)
        tr = []
        nsteps = int(22e-6 / dt)
        for _ in range(nsteps // 10):
            assert A.run(10) == 0
            tr.append(A.pressure()[krec, ny // 2, nx // 2])
        traces[solid] = np.array(tr)
    t = (np.arange(len(traces[True])) + 1) * 10 * dt
    inc = np.abs(traces[False][t < 13e-6]).max()
    refl = np.abs((traces[True] - traces[False])[t > 13e-6]).max()
    Z1, Z2 = 1000.0 * 1500.0, 1850.0 * 2800.0
    assert refl / inc == pytest.approx((Z2 - Z1) / (Z2 + Z1), rel=0.02)
    assert (Z2 - Z1) / (Z2 + Z1) == pytest.approx(0.5509, abs=1e-4)


def test_normal_incidence_reflection_cortical_trabecular(orc):
    """Solid to solid, negative coefficient: a plane burst in cortical bone
    (rho 1850, cL 2800, cS 1500) onto trabecular bone (1700, 2300, 1200):
    R = (Z2 - Z1)/(Z2 + Z1) = -0.1397 with Z = rho cL (no mode conversion at
    normal incidence).  The receiver sits 1.5 mm above the interface, so the
    incident and reflected pulses travel nearly the same path; the run with
    the interface minus the run without it isolates the reflection.  The
    material averaging at the interface faces is first-order-accurate in
    position, so the measured |R| converges to the exact one: within 2 % at
    dx = 0.125 mm (on a 12-cell-wide column; 1.2 % on a 32-cell one), with the
    error at least halved from dx = 0.25 mm, and the reflected pulse inverted."""
    f0 = 5e5
    from paper_2301_12727_gb300 import synth
    Z1, Z2 = 1850.0 * 2800.0, 1700.0 * 2300.0
    R = (Z2 - Z1) / (Z2 + Z1)
    assert R == pytest.approx(-0.1397, abs=1e-4)
    errs = []
    for dx in (0.25e-3, 0.125e-3):
        r = int(round(0.25e-3 / dx))
        nx = ny = 12                  # laterally uniform: the width does not enter
        nz, P = 176 * r, 4
        dt, M = synth.choose_dt(dx, 2800.0, f0)
        ks, kint = 12 * r, 110 * r
        krec = kint - 6 * r
        traces = {}
        for interface in (True, False):
            mats = [mat_row(1850.0, 2800.0, 1500.0), mat_row(1700.0, 2300.0, 1200.0)]
            index = np.zeros((nz, ny, nx), np.uint8)
            if interface:
                index[kint:] = 1
            A = orc.Acoustic(nx, ny, nz, dx, dt, index, mats, f0, n_sls=2, n_pml=P)
            A.set_source(np.ones((ny, nx)), ks, 2800.0, orc.ENV_BURST, 3)
            tr = []
            for _ in range(int(17e-6 / dt) // 5):
                assert A.run(5) == 0
                tr.append(A.pressure()[krec, ny // 2, nx // 2])
            traces[interface] = np.array(tr)
        inc = traces[False]
        diff = traces[True] - traces[False]
        errs.append(abs(np.abs(diff).max() / np.abs(inc).max() - abs(R)) / abs(R))
        # inverted copy: the strongest cross-correlation over the delays is negative
        cc = [float(np.dot(diff[sft:], inc[:len(inc) - sft])) for sft in range(len(inc) // 2)]
        assert cc[int(np.argmax(np.abs(cc)))] < 0.0
    assert errs[1] < 0.02 and errs[1] < 0.5 * errs[0], errs


# --------------------------------------------------------------------------
# CFL limit 6/(7 sqrt 3)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("frac,grows", [(0.98, False), (1.03, True)])
def test_cfl_threshold(orc, frac, grows):
    """Random data in a closed fluid box: bounded below the O(4) 3-D limit
    S = 6/(7 sqrt 3), exponential growth just above it."""
    n, dx, c = 14, 1e-3, 1500.0
    dt = frac * orc.courant_limit() * dx / c
    A = orc.Acoustic(n, n, n, dx, dt, np.zeros((n, n, n)), [mat_row(1000.0, c)], F0,
                     n_sls=0, n_pml=0)
    rng = np.random.default_rng(3)
    p = rng.standard_normal((n, n, n))
    for f in ("sxx", "syy", "szz"):
        A.field(f)[...] = p
    if grows:
        assert A.run(10) == orc.E_CFL       # the limit is enforced by default
    assert A.run(1500, check_cfl=False) == 0
    m = np.abs(A.pressure()).max()
    assert (m > 1e6) == grows, m
    assert orc.courant_limit() == pytest.approx(6 / (7 * math.sqrt(3)), rel=1e-15)


# --------------------------------------------------------------------------
# Mirror symmetry (bitwise) with CPML, SLS and a source
# --------------------------------------------------------------------------
def test_mirror_symmetry_is_bitwise(orc):
    """A medium and source symmetric under x -> (nx-1) - x and y -> (ny-1) - y
    give a pressure field with the same symmetry to the last bit."""
    from paper_2301_12727_gb300 import synth
    c = synth.skull_case(40, 40, 36, dx=0.5e-3, n_steps=60, symmetric=True, n_pml=6)
    A = orc.Acoustic(c.nx, c.ny, c.nz, c.dx, c.dt, c.index, c.materials, c.f0, n_sls=2,
                     n_pml=c.n_pml)
    assert np.array_equal(c.index, c.index[:, :, ::-1]) and np.array_equal(c.index, c.index[:, ::-1, :])
    x = np.arange(c.nx) - (c.nx - 1) / 2
    r2 = x[None, :] ** 2 + x[:, None] ** 2
    plane = np.exp(-r2 / 60.0) * np.exp(1j * 0.01 * r2)
    A.set_source(plane, c.k_src, 1500.0, orc.ENV_RAMP_CW)
    assert A.run(c.n_steps, peak_from=0) == 0
    p = A.pressure()
    assert np.abs(p).max() > 0
    assert np.array_equal(p, p[:, :, ::-1])
    assert np.array_equal(p, p[:, ::-1, :])
    assert np.array_equal(A.peak, A.peak[:, :, ::-1])


def test_cpml_absorbs_outgoing_pulse(orc):
    """After a burst has left through the CPML, the energy left in the box is
    small compared with the peak (a lossless closed box keeps all of it)."""
    n, dx, f0 = 48, 0.5e-3, 5e5
    from paper_2301_12727_gb300 import synth
    dt, M = synth.choose_dt(dx, 1500.0, f0)
    res = {}
    for P in (8, 0):
        A = orc.Acoustic(n, n, n, dx, dt, np.zeros((n, n, n)), [mat_row(1000.0, 1500.0)], f0,
                         n_sls=0, n_pml=P)
        plane = np.zeros((n, n), complex)
        plane[n // 2, n // 2] = 1.0
        A.set_source(plane, n // 2, 1500.0, orc.ENV_BURST, 1)
        assert A.run(3 * M) == 0
        e0 = np.sum(A.pressure() ** 2)
        assert A.run(int(2.5 * n * dx / 1500.0 / dt)) == 0
        res[P] = np.sum(A.pressure() ** 2) / e0
    assert res[8] < 5e-3
    assert res[0] > 0.1


# --------------------------------------------------------------------------
# Rayleigh-Sommerfeld (Sec. 2.3): O'Neil on-axis field of a bowl
# --------------------------------------------------------------------------
@pytest.mark.parametrize("ds,tol", [(1.0 / 16, 2e-3), (0.25, 1e-2)])
def test_rs_matches_oneil_on_axis(orc, ds, tol):
    """Element sum of i k p0/(2 pi) dA e^{-ikr}/r over the cap vs O'Neil's exact
    on-axis integral, in the focal region (default lambda^2/16 elements: 1 %)."""
    a, R, f0, c0, p0 = 32e-3, 63e-3, 5e5, 1500.0, 1.0
    k = 2 * np.pi * f0 / c0
    zs = np.linspace(0.75 * R, 1.2 * R, 7)
    got = []
    for z in zs:
        p = orc.rs_plane(2 * a, R, (0.0, 0.0, 0.0), (0.0, 0.0, 1.0), 1, 1, 1e-3, z, f0, c0, p0,
                         ds_over_lambda=ds)
        got.append(p[0, 0])
    got = np.array(got)
    ref = an.oneil_on_axis(zs, a, R, k, p0)
    assert np.abs(np.abs(got) / ref - 1).max() < tol
    # the complex value (phase convention included) of the exact on-axis integral
    refc = an.oneil_on_axis_complex(zs, a, R, k, p0)
    assert np.abs(got - refc).max() / np.abs(refc).max() < 2 * tol


def test_bowl_elements_area_and_tilt(orc):
    """Element areas sum to the cap area 2 pi R^2 (1 - cos theta_max); tilting
    rotates the elements rigidly about the apex."""
    a, R, lam = 32e-3, 63e-3, 3e-3
    el = orc.bowl_elements(2 * a, R, (0, 0, 0), (0, 0, 1), lam)
    cap = 2 * np.pi * R * R * (1 - math.sqrt(1 - (a / R) ** 2))
    assert el[:, 3].sum() == pytest.approx(cap, rel=1e-12)
    assert np.abs(el[:, 3] / (lam * lam / 16) - 1).max() < 0.35
    t = math.radians(12.0)
    el2 = orc.bowl_elements(2 * a, R, (0, 0, 0), (math.sin(t), 0, math.cos(t)), lam)
    # distances to the centre of curvature are all R in both poses
    assert np.allclose(np.linalg.norm(el[:, :3] - [0, 0, R], axis=1), R, rtol=1e-12)
    ctr = np.array([R * math.sin(t), 0, R * math.cos(t)])
    assert np.allclose(np.linalg.norm(el2[:, :3] - ctr, axis=1), R, rtol=1e-12)


# --------------------------------------------------------------------------
# BHTE (Sec. 2.4): Pennes Gaussian diffusion with perfusion; CEM43
# --------------------------------------------------------------------------
def _bhte_gauss_err(orc, n, s0_cells):
    dx = 0.5e-3 * 32 / n
    k, rho, cth, wb, rbcb = 0.5, 1000.0, 4000.0, 0.01, 1050.0 * 3617.0
    mats = [mat_row(rho, 1500.0, k=k, c=cth, perf=wb)]
    index = np.zeros((n, n, n), np.uint8)
    D = k / (rho * cth)
    wprime = wb * rbcb / (rho * cth)
    s0 = s0_cells * 0.5e-3
    dt = 0.5 * dx * dx / D / 6
    t_end = s0 * s0 / (2 * D)                        # variance doubles
    nsteps = int(round(t_end / dt))
    x = (np.arange(n) - (n - 1) / 2) * dx
    r2 = x[None, None, :] ** 2 + x[None, :, None] ** 2 + x[:, None, None] ** 2
    T0 = 37.0 + an.pennes_gaussian(r2, 0.0, 5.0, s0, D, wprime)
    rc, T, Tmax, cem = orc.bhte_run(index, mats, dx, None, 0.0, dt, nsteps, 0, 1.0, T_a=37.0,
                                    rhob_cb=rbcb, T_init=T0)
    assert rc == 0
    ref = 37.0 + an.pennes_gaussian(r2, nsteps * dt, 5.0, s0, D, wprime)
    core = r2 < (2 * s0) ** 2
    return np.abs(T - ref)[core].max() / 5.0


def test_bhte_gaussian_diffusion_with_perfusion(orc):
    """Pennes with uniform perfusion and a Gaussian initial excess follows
    theta0 (s0^2/(s0^2+2Dt))^{3/2} e^{-r^2/2(s0^2+2Dt)} e^{-w' t}; the 7-point
    FTCS error falls at second order in dx."""
    e1 = _bhte_gauss_err(orc, 32, 3.0)
    e2 = _bhte_gauss_err(orc, 64, 3.0)
    assert e1 < 1e-2
    assert e2 < e1 / 3.0


@pytest.mark.parametrize("T,R", [(37.0, 0.25), (45.0, 0.5), (43.0, 0.5)])
def test_cem43_at_constant_temperature(orc, T, R):
    """Uniform T everywhere (T_a = T, no heating): CEM43 = t R^{43-T} / 60 with
    R = 0.5 at or above 43 C, 0.25 below (Sapareto-Dewey)."""
    n = 8
    index = np.zeros((n, n, n), np.uint8)
    mats = [mat_row(1000.0, 1500.0, perf=0.01)]
    dt, nsteps = 0.05, 400
    rc, Tf, Tmax, cem = orc.bhte_run(index, mats, 1e-3, np.ones((n, n, n)), 0.0, dt, nsteps, 0,
                                     1.0, T_a=T)
    assert rc == 0
    assert np.all(Tf == T) and np.all(Tmax == T)
    assert np.allclose(cem, nsteps * dt * R ** (43.0 - T) / 60.0, rtol=1e-12)


def test_bhte_heating_energy_balance(orc):
    """With no perfusion, sealed by a wide margin and a short exposure, the heat
    deposited (sum Q dt) equals the stored excess sum rho c (T - T_a) dx^3."""
    n, dx = 24, 0.5e-3
    index = np.zeros((n, n, n), np.uint8)
    rho, c, k, aL, cL = 1041.0, 3630.0, 0.51, 3.45, 1562.0
    mats = [mat_row(rho, cL, 0.0, aL, k=k, c=c, perf=0.0)]
    amp = np.zeros((n, n, n))
    amp[10:14, 10:14, 10:14] = 1e6
    dt, n_on = 0.01, 20
    rc, T, Tmax, cem = orc.bhte_run(index, mats, dx, amp, 1.0, dt, n_on, 0, 0.3, T_a=37.0)
    assert rc == 0
    Q = aL * 1e12 / (rho * cL)
    deposited = 0.3 * Q * 64 * dx ** 3 * n_on * dt
    stored = np.sum(rho * c * (T - 37.0)) * dx ** 3
    assert stored == pytest.approx(deposited, rel=1e-9)


# --------------------------------------------------------------------------
# E_L (Eq. 2) and T_S = sqrt(E_L)
# --------------------------------------------------------------------------
def test_transmission_on_constructed_maps(orc):
    """Water map with its maximum on plane z0; skull map = 0.5 x water with the
    same rho c there -> E_L = 0.25 and z_m = z0; identical runs -> E_L = 1."""
    n = 16
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    amp_w = np.exp(-((z - 9) ** 2 + (y - 7) ** 2 + (x - 8) ** 2) / 8.0)
    idx = np.zeros((n, n, n), np.uint8)
    mw = [mat_row(1000.0, 1500.0)]
    el, zm = orc.transmission(idx, mw, 0.5 * amp_w, idx, mw, amp_w)
    assert zm == 9 and el == pytest.approx(0.25, rel=1e-14)
    el, zm = orc.transmission(idx, mw, amp_w, idx, mw, amp_w)
    assert el == 1.0
    # a different rho c at the skull-run voxels scales the intensity by Z_w / Z_b
    ib = np.ones_like(idx)
    mb = [mat_row(1000.0, 1500.0), mat_row(1041.0, 1562.0)]
    el, _ = orc.transmission(ib, mb, amp_w, idx, mw, amp_w)
    assert el == pytest.approx(1500.0 * 1000.0 / (1041.0 * 1562.0), rel=1e-14)


def test_source_amplitude_of_soft_plane_source(orc):
    """The soft plane source scaled by 2 c0 dt/dx launches plane waves of
    amplitude A in both directions (1-D Green's function of a plane mass
    source), checked on the axis of a wide CW plane source."""
    f0, dx = 5e5, 0.25e-3
    n, nz, P = 40, 120, 8
    from paper_2301_12727_gb300 import synth
    dt, M = synth.choose_dt(dx, 1500.0, f0)
    A = orc.Acoustic(n, n, nz, dx, dt, np.zeros((nz, n, n)), [mat_row(1000.0, 1500.0)], f0,
                     n_sls=0, n_pml=P)
    A.set_source(np.full((n, n), 2.0), 40, 1500.0, orc.ENV_RAMP_CW)
    nsteps = 8 * M
    assert A.run(nsteps, dft_start=nsteps - 2 * M + 1, dft_steps=2 * M) == 0
    amp, _ = A.amp_phase(2 * M)
    assert amp[60, n // 2, n // 2] == pytest.approx(2.0, rel=0.02)
    assert amp[25, n // 2, n // 2] == pytest.approx(2.0, rel=0.02)


def test_soft_source_phase_matches_lattice_green_function(orc):
    """Complex amplitude (phase included) of the captured field of a CW plane
    source against the exact far field of the discrete scheme: the source
    value A e^{i phi} drives the pressure rate with A sin(w t + phi) at half
    steps (complex amplitude -i A e^{i phi}), the capture reads p at whole
    steps, and the DFT returns p = amp cos(w t + phase).  Checked 4-12 cells
    on both sides of the source at 6 points per wavelength, where the
    lattice amplitude factor is 1.027 and the phase advance per cell 1.06 rad."""
    f0, dx = 5e5, 0.5e-3
    n, nz, P, ks = 16, 120, 8, 40
    from paper_2301_12727_gb300 import synth
    dt, M = synth.choose_dt(dx, 1500.0, f0)
    A = orc.Acoustic(n, n, nz, dx, dt, np.zeros((nz, n, n)), [mat_row(1000.0, 1500.0)], f0,
                     n_sls=0, n_pml=P)
    a0, phi = 2.0, 0.7
    A.set_source(np.full((n, n), a0 * np.exp(1j * phi)), ks, 1500.0, orc.ENV_RAMP_CW)
    nsteps = 10 * M
    assert A.run(nsteps, dft_start=nsteps - 2 * M + 1, dft_steps=2 * M) == 0
    amp, ph = A.amp_phase(2 * M)
    w = 2 * np.pi * f0
    for d in (-12, -8, -4, 4, 8, 12):
        got = amp[ks + d, n // 2, n // 2] * np.exp(1j * ph[ks + d, n // 2, n // 2])
        ref = an.soft_source_far_field(-1j * a0 * np.exp(1j * phi), d, w, dt, dx, 1500.0)
        assert abs(got) / abs(ref) - 1 == pytest.approx(0.0, abs=3e-3), d
        assert np.angle(got / ref) == pytest.approx(0.0, abs=3e-3), d


def test_bhte_insulating_sheet_blocks_conduction(orc):
    """Series resistance at material interfaces: heat crossing the face
    between two voxels passes both half-voxels in turn, so a one-voxel sheet
    of (almost) zero conductivity stops conduction whatever conducts on
    either side.  A hot block on one side leaves the far side at T_a."""
    n, nz, dx = 12, 30, 1e-3
    idx = np.zeros((nz, n, n), np.uint8)
    idx[15] = 1
    tissue = mat_row(1000.0, 1500.0, k=0.5, c=3600.0)
    sheet = mat_row(1000.0, 1500.0, k=1e-9, c=3600.0)
    T0 = np.full(idx.shape, 37.0)
    T0[3:14, 2:-2, 2:-2] = 45.0
    rc, T, Tmax, cem = orc.bhte_run(idx, [tissue, sheet], dx, None, 0.0, 0.05, 400, 0, 0.0,
                                    T_init=T0)
    assert rc == 0
    assert T[10, n // 2, n // 2] > 38.0            # the hot side is still warm and conducting
    assert T[14, n // 2, n // 2] > 37.5            # heat reached the sheet
    assert np.abs(T[16:] - 37.0).max() < 1e-6      # and nothing crossed it


def test_rs_elements_single_element_and_steered_array(orc):
    """Weighted-element Rayleigh sum: one element of area dA gives
    |p| = k p0 dA / (2 pi r) everywhere; an array whose weights are
    exp(+i k r_t,e) (steered at target t) adds coherently there:
    p(t) = i k p0 / (2 pi) sum_e dA_e / r_t,e."""
    f0, c0, p0 = 5e5, 1500.0, 1e4
    k = 2 * np.pi * f0 / c0
    dx, nx, ny, zp = 0.5e-3, 9, 7, 0.03
    one = np.array([[1e-3, 2e-3, 0.0, 4e-6, 1.0, 0.0]])
    p = orc.rs_elements(one, p0, c0, nx, ny, dx, zp, f0)
    X, Y = np.meshgrid(np.arange(nx) * dx, np.arange(ny) * dx)
    r = np.sqrt((X - 1e-3) ** 2 + (Y - 2e-3) ** 2 + zp ** 2)
    assert np.abs(np.abs(p) - k * p0 * 4e-6 / (2 * np.pi * r)).max() < 1e-12 * np.abs(p).max()
    rng = np.random.default_rng(4)
    ne = 64
    pos = np.stack([rng.uniform(-0.02, 0.02, ne), rng.uniform(-0.02, 0.02, ne),
                    rng.uniform(-0.01, 0.0, ne)], axis=1)
    area = rng.uniform(1e-6, 4e-6, ne)
    tgt = np.array([3 * dx, 2 * dx, zp])                   # grid point (3, 2) of the plane
    rt = np.linalg.norm(pos - tgt, axis=1)
    w = np.exp(1j * k * rt)
    el = np.column_stack([pos, area, w.real, w.imag])
    p = orc.rs_elements(el, p0, c0, nx, ny, dx, zp, f0)
    expect = 1j * k * p0 / (2 * np.pi) * np.sum(area / rt)
    assert abs(p[2, 3] - expect) < 1e-12 * abs(expect)
    assert np.abs(p).max() == pytest.approx(abs(p[2, 3]), rel=1e-12)   # the target is the maximum


def _table1_rows(f):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_materials.txt")
    rows = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        n, rho, cl0, cl1, cs0, cs1, al, as_ = line.split()
        fm = f / 1e6
        rows[n] = mat_row(float(rho), float(cl0) + float(cl1) * f, float(cs0) + float(cs1) * f,
                          float(al) * fm, float(as_) * fm)
    return rows


@pytest.mark.parametrize("f", [2e5, 5e5, 1e6])
@pytest.mark.parametrize("qc", [0.4, 1.0, 3.0, 4.0, 7.0])
def test_table1_q_fit_over_the_papers_sweep(orc, f, qc):
    """Table 1 tissues over the study's frequencies (0.2-1 MHz) and correction
    factors q_c (Sec. 3.2): every material is fitted exactly when
    Q = q_c w/(2 c alpha) exceeds what two mechanisms can reach (5/3) and
    rejected otherwise; the fit reproduces Q and the phase speed at f."""
    rows = _table1_rows(f)
    w = 2 * np.pi * f
    for name, row in rows.items():
        rho, cL, cS, aL, aS = row[:5]
        reach = all(a == 0 or qc * w / (2 * c * a) > 5.0 / 3.0 for c, a in ((cL, aL), (cS, aS)))
        rc, coef, ts = orc.material_coefs([row], f, qc, 2)
        assert (rc == 0) == reach, (name, f, qc)
        if rc:
            continue
        for (c, a, M, tau) in ((cL, aL, coef[0, 0], coef[0, 2]), (cS, aS, coef[0, 1], coef[0, 3])):
            if c == 0:
                assert M == 0.0
                continue
            Mw = M * an.sls_modulus_factor(w, tau, ts)
            if a > 0:
                assert Mw.real / Mw.imag == pytest.approx(qc * w / (2 * c * a), rel=1e-12)
            assert w / (w * np.sqrt(rho / Mw)).real == pytest.approx(c, rel=1e-12)
