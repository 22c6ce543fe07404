"""Index conventions of the C oracle pinned against a second FP64
implementation in array form (tests/second_oracle.py) on small grids: random
heterogeneous media (fluid cells with mu = 0 included), random initial
velocities, stresses and memory variables, one and two SLS mechanisms, and a
plane burst source.  Every field agrees to 1e-12 of its largest value after a
few steps, so a wrong neighbour, a swapped staggering, a misplaced shear cell
or a dropped memory-variable term in either would show."""
import numpy as np
import pytest

from tests import second_oracle as so


def _media(rng):
    # rho, cL, cS, alphaL, alphaS, k, c_th, perf, heat_frac
    return np.array([[1000.0, 1500.0, 0.0, 0.0, 0.0, 0.6, 4180, 0, 0],
                     [1900.0, 2850.0, 1450.0, 180.0, 360.0, 0.32, 1300, 0, 0.16],
                     [1050.0, 1560.0, 0.0, 40.0, 0.0, 0.5, 3600, 0, 1],
                     [1700.0, 2300.0, 1100.0, 120.0, 240.0, 0.4, 1500, 0, 0.16]])


def _setup(orc, shape, L, seed):
    rng = np.random.default_rng(seed)
    mat = _media(rng)
    nz, ny, nx = shape
    index = rng.integers(0, len(mat), size=shape).astype(np.uint8)
    dx, f0 = 0.5e-3, 5e5
    rc, coef, ts = orc.material_coefs(mat, f0, 1.0, L)
    assert rc == 0
    dt = 0.3 * orc.courant_limit() * dx / 3200.0
    A = orc.Acoustic(nx, ny, nz, dx, dt, index, mat, f0, n_sls=L, n_pml=0)
    st = np.zeros_like(A.state)
    st[:9 + 6 * L] = rng.standard_normal((9 + 6 * L,) + shape)
    st[0][:, :, -1] = 0.0           # ghost half points of each axis
    st[1][:, -1, :] = 0.0
    st[2][-1, :, :] = 0.0
    A.state[:] = st
    return A, mat, index, coef, ts, dx, dt, f0, st[:9 + 6 * L].copy()


@pytest.mark.parametrize("shape,L", [((10, 12, 14), 2), ((9, 11, 8), 1), ((20, 6, 7), 2)])
def test_random_state_steps_agree(orc, shape, L):
    A, mat, index, coef, ts, dx, dt, f0, s = _setup(orc, shape, L, seed=sum(shape) + L)
    n_steps = 3
    assert A.run(n_steps, peak_from=-1) == 0
    for n in range(n_steps):
        s = so.step(s, index, mat[:, 0], coef, ts, dt, dx, n)
    for f in range(9 + 6 * L):
        ref = A.state[f]
        scale = max(np.abs(ref).max(), 1e-300)
        assert np.abs(s[f] - ref).max() <= 1e-12 * scale, f


def test_plane_burst_source_agrees(orc):
    shape, L = (12, 10, 11), 2
    A, mat, index, coef, ts, dx, dt, f0, _ = _setup(orc, shape, L, seed=3)
    A.state[:] = 0.0
    rng = np.random.default_rng(4)
    plane = (rng.standard_normal(shape[1:]) + 1j * rng.standard_normal(shape[1:])) * 1e3
    k_src, n_cycles = 4, 2
    A.set_source(plane, k_src, 1500.0, orc.ENV_BURST, n_cycles)
    n_steps = 6
    assert A.run(n_steps, peak_from=-1) == 0
    s = np.zeros((9 + 6 * L,) + shape)

    def env(t):
        return 1.0 if 0.0 <= t < n_cycles / f0 else 0.0

    for n in range(n_steps):
        s = so.step(s, index, mat[:, 0], coef, ts, dt, dx, n, src=plane, k_src=k_src,
                    c0=1500.0, f0=f0, env=env)
    for f in range(9 + 6 * L):
        ref = A.state[f]
        scale = max(np.abs(ref).max(), 1e-300)
        assert np.abs(s[f] - ref).max() <= 1e-12 * scale, f
    assert np.abs(A.state[3]).max() > 0.0


def test_second_oracle_catches_a_shifted_stencil(orc):
    """The comparison is sharp: the same step with D- taken at s+1/2 instead
    of s (a one-cell staggering slip) differs from the C oracle by O(1)."""
    shape, L = (8, 9, 10), 1
    A, mat, index, coef, ts, dx, dt, f0, s = _setup(orc, shape, L, seed=9)
    assert A.run(1, peak_from=-1) == 0
    good = so.step(s, index, mat[:, 0], coef, ts, dt, dx, 0)
    orig = so.d_minus
    try:
        so.d_minus = lambda f, axis, h: so.d_plus(f, axis, h)
        bad = so.step(s, index, mat[:, 0], coef, ts, dt, dx, 0)
    finally:
        so.d_minus = orig
    ref = A.state[3]
    assert np.abs(good[3] - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(bad[3] - ref).max() > 1e-3 * np.abs(ref).max()


@pytest.mark.parametrize("shape,L,P", [((16, 14, 18), 2, 3), ((12, 15, 13), 1, 2)])
def test_cpml_slabs_agree(orc, shape, L, P):
    """The same comparison with absorbing slabs on every axis: each psi
    recursion sits on the right derivative, at integer or half points, and
    all 18 memories match the C oracle's after a few steps."""
    rng = np.random.default_rng(sum(shape) + 7 * P)
    mat = _media(rng)
    nz, ny, nx = shape
    index = rng.integers(0, len(mat), size=shape).astype(np.uint8)
    dx, f0, R = 0.5e-3, 5e5, 1e-4
    rc, coef, ts = orc.material_coefs(mat, f0, 1.0, L)
    assert rc == 0
    dt = 0.3 * orc.courant_limit() * dx / 3200.0
    A = orc.Acoustic(nx, ny, nz, dx, dt, index, mat, f0, n_sls=L, n_pml=P, pml_R=R)
    st = rng.standard_normal(A.state.shape)
    st[0][:, :, -1] = 0.0
    st[1][:, -1, :] = 0.0
    st[2][-1, :, :] = 0.0
    A.state[:] = st
    s = st.copy()
    n_steps = 3
    assert A.run(n_steps, peak_from=-1) == 0
    cp = dict(P=P, R=R, cmax=mat[:, 1].max())
    for n in range(n_steps):
        s = so.step(s, index, mat[:, 0], coef, ts, dt, dx, n, cpml=cp)
    for f in range(A.state.shape[0]):
        ref = A.state[f]
        scale = max(np.abs(ref).max(), 1e-300)
        assert np.abs(s[f] - ref).max() <= 1e-12 * scale, f


def test_bhte_array_form_agrees(orc):
    """The C oracle's BHTE against the array-form step on random heterogeneous
    tissue, a random acoustic field and a starting temperature spread over
    37 .. 46 C (both CEM43 bases): T, T_max and CEM43 to 1e-12."""
    rng = np.random.default_rng(17)
    # rho, cL, cS, alphaL, alphaS, k, c_th, perf, heat_frac
    mat = np.array([[1000.0, 1500.0, 0.0, 0.0, 0.0, 0.6, 4180.0, 0.0, 1.0],
                    [1041.0, 1562.0, 0.0, 35.0, 0.0, 0.51, 3630.0, 0.008, 1.0],
                    [1850.0, 2800.0, 1500.0, 85.0, 170.0, 0.32, 1300.0, 0.0005, 0.16],
                    [1116.0, 1537.0, 0.0, 23.0, 0.0, 0.37, 3390.0, 0.002, 1.0]])
    shape = (10, 12, 14)
    index = rng.integers(0, len(mat), size=shape).astype(np.uint8)
    amp = rng.uniform(0.0, 2e6, size=shape)
    T0 = rng.uniform(37.0, 46.0, size=shape)
    dx, dt = 0.5e-3, 0.02
    rc, T, Tmax, cem = orc.bhte_run(index, mat, dx, amp, 1.0, dt, 5, 3, 0.3, T_init=T0)
    assert rc == 0
    T2, Tmax2, cem2 = so.bhte_run(T0, index, mat, dx, amp, 1.0, dt, 5, 3, 0.3)
    for a, b in ((T2, T), (Tmax2, Tmax), (cem2, cem)):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    assert (cem > 0).all() and np.abs(T - T0).max() > 1e-3


def test_capture_array_form_agrees(orc):
    """Peak and FP64 DFT capture: after each step n -> n+1 the pressure
    p = -(sxx + syy + szz)/3 enters max |p| and C += p cos(w t), S += p sin(w t)
    at t = (n+1) dt; the C oracle's maps equal the array-form sums to 1e-12."""
    shape, L = (9, 10, 11), 2
    A, mat, index, coef, ts, dx, dt, f0, s = _setup(orc, shape, L, seed=23)
    n_steps, dft_start = 6, 3
    assert A.run(n_steps, peak_from=2, dft_start=dft_start, dft_steps=n_steps) == 0
    peak = np.zeros(shape)
    C, S = np.zeros(shape), np.zeros(shape)
    w = 2.0 * np.pi * f0
    for n in range(n_steps):
        s = so.step(s, index, mat[:, 0], coef, ts, dt, dx, n)
        stp = n + 1
        p = -(s[3] + s[4] + s[5]) / 3.0
        if stp >= 2:
            peak = np.maximum(peak, np.abs(p))
        if stp >= dft_start:
            C += p * np.cos(w * stp * dt)
            S += p * np.sin(w * stp * dt)
    for a, b in ((peak, A.peak), (C, A.dftC), (S, A.dftS)):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    assert np.abs(A.dftS).max() > 0.0
