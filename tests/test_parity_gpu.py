"""GPU (libbvf, FP32 with FP64 capture) against the FP64 oracle and closed forms.

Tolerance: relative L2 <= 1e-4 on the pressure field (and on the other
outputs unless stated), the bound set for the FP32 stencil.  Every call goes
through the C ABI.
"""
import math

import numpy as np
import pytest

from tests import analytic as an

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module")
def bvf():
    import torch
    assert torch.cuda.is_available()
    from paper_2301_12727_gb300 import build
    build.build()
    from paper_2301_12727_gb300 import bvf as m
    return m


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def mat_row(rho, cL, cS=0.0, aL=0.0, aS=0.0, k=0.5, c=3600.0, perf=0.0, heat=1.0):
    return [rho, cL, cS, aL, aS, k, c, perf, heat]


def make_pair(bvf, orc, c, n_sls=2, storage="f32"):
    s = bvf.Solver(c.nx, c.ny, c.nz, c.dx, c.dt, c.f0, qc=c.qc, n_sls=n_sls, n_pml=c.n_pml,
                   pml_R=c.pml_R, storage=storage)
    s.set_materials(c.index, c.materials)
    A = orc.Acoustic(c.nx, c.ny, c.nz, c.dx, c.dt, c.index, c.materials, c.f0, qc=c.qc,
                     n_sls=n_sls, n_pml=c.n_pml, pml_R=c.pml_R)
    return s, A


# --------------------------------------------------------------------------
def test_gpu_discrete_plane_wave_exact(bvf):
    """Same closed form that pins the oracle: an oblique discrete plane wave in
    a homogeneous solid, now through the GPU kernels (FP32)."""
    n, dx, rho, cL, cS = 48, 1e-3, 1000.0, 2800.0, 1400.0
    dt = 0.3 * dx / cL
    kvec = np.array([2 * np.pi / (7 * dx), 2 * np.pi / (9 * dx), 2 * np.pi / (11 * dx)])
    for mode in ("P", "S"):
        s = bvf.Solver(n, n, n, dx, dt, 5e5, n_sls=2, n_pml=0)
        s.set_materials(np.zeros((n, n, n), np.uint8), [mat_row(rho, cL, cS)])
        om, amp, fields = an.discrete_plane_wave((n, n, n), dx, dt, rho, rho * cL ** 2,
                                                 rho * cS ** 2, kvec, mode)
        f0 = fields(-0.5 * dt, 0.0)
        for name in an.FIELDS:
            s.set_field(name, f0[name])
        steps = 5
        s.run(steps)
        s.synchronize()
        ex = fields((steps - 0.5) * dt, steps * dt)
        m = 3 * steps + 3
        sl = (slice(m, n - m),) * 3
        for name in an.FIELDS:
            got = s.field(name).cpu().numpy()[sl]
            scale = max(abs(amp[f]) for f in an.FIELDS if f[0] == name[0])
            assert np.abs(got - ex[name][sl]).max() / scale < 2e-5, (mode, name)
        s.close()


@pytest.mark.parametrize("nx,ny,nz", [(45, 38, 29), (48, 37, 29)])
def test_gpu_random_state_all_fields(bvf, orc, nx, ny, nz):
    """Random velocities, stresses and memory variables in a heterogeneous
    fluid/solid/SLS medium with CPML on ragged grids, not multiples of the
    32 x 8 tile: 45 x 38 x 29 runs the direct kernels, 48 x 37 x 29 (a
    half x-tile, ragged y and z) the TMA-fed ones.  Every state array after
    12 steps."""
    dx = 0.5e-3
    rng = np.random.default_rng(11)
    mats = [mat_row(1000.0, 1500.0), mat_row(1850.0, 2800.0, 1500.0, 85.0, 170.0),
            mat_row(1700.0, 2300.0, 1200.0, 81.0, 162.0), mat_row(1041.0, 1562.0, 0.0, 3.45)]
    index = rng.integers(0, 4, size=(nz // 3 + 1, ny // 3 + 1, nx // 3 + 1))
    index = np.kron(index, np.ones((3, 3, 3), np.int64))[:nz, :ny, :nx].astype(np.uint8)
    from paper_2301_12727_gb300 import synth
    dt, _ = synth.choose_dt(dx, 2800.0, 5e5)
    s = bvf.Solver(nx, ny, nz, dx, dt, 5e5, n_sls=2, n_pml=5)
    s.set_materials(index, mats)
    A = orc.Acoustic(nx, ny, nz, dx, dt, index, mats, 5e5, n_sls=2, n_pml=5)
    n_state = 9 + 6 * 2
    init = (rng.standard_normal((n_state, nz, ny, nx)) * np.array(
        [1.0] * 3 + [1e6] * 6 + [1e4] * 12)[:, None, None, None]).astype(np.float32)
    d = {f: init[i] for i, f in enumerate(an.FIELDS)}
    an.zero_ghost_half_points(d)
    for i in range(n_state):
        if i < 9:
            init[i] = d[an.FIELDS[i]]
        s.set_field(i, init[i])
        A.state[i] = init[i].astype(np.float64)
    # memory variables of shear components at ghost half points stay zero too
    for l in range(2):
        for c, f in ((3, "sxy"), (4, "sxz"), (5, "syz")):
            m = (d[f] != 0).astype(np.float32)
            init[9 + 6 * l + c] *= m
            s.set_field(9 + 6 * l + c, init[9 + 6 * l + c])
            A.state[9 + 6 * l + c] = init[9 + 6 * l + c].astype(np.float64)
    s.run(12)
    s.synchronize()
    assert A.run(12) == 0
    for i in range(n_state):
        got = s.field(i).cpu().numpy()
        assert rel_l2(got, A.state[i]) < 2e-5, (i, rel_l2(got, A.state[i]))


def test_gpu_soft_source_matches_lattice_green_function(bvf):
    """The GPU path against a closed form directly (no oracle): the captured
    complex amplitude of a CW plane source, 4-12 cells on both sides of it,
    equals the exact far field of the discrete scheme (phase convention,
    half-step source time, whole-step capture, DFT sign and the lattice
    amplitude factor 1.027 at 6 points per wavelength)."""
    from paper_2301_12727_gb300 import synth
    f0, dx = 5e5, 0.5e-3
    n, nz, P, ks = 32, 120, 8, 40
    dt, M = synth.choose_dt(dx, 1500.0, f0)
    s = bvf.Solver(n, n, nz, dx, dt, f0, n_sls=0, n_pml=P)
    s.set_materials(np.zeros((nz, n, n), np.uint8), [mat_row(1000.0, 1500.0)])
    a0, phi = 2.0, 0.7
    s.set_source(np.full((n, n), a0 * np.exp(1j * phi), np.complex64), ks, 1500.0,
                 bvf.BVF_ENV_RAMP_CW)
    nsteps = 10 * M
    s.run(nsteps, dft_start=nsteps - 2 * M + 1, dft_steps=2 * M)
    s.synchronize()
    amp, ph = (t.cpu().numpy() for t in s.amp_phase())
    w = 2 * np.pi * f0
    for d in (-12, -8, -4, 4, 8, 12):
        got = amp[ks + d, n // 2, n // 2] * np.exp(1j * ph[ks + d, n // 2, n // 2])
        ref = an.soft_source_far_field(-1j * a0 * np.exp(1j * phi), d, w, dt, dx, 1500.0)
        assert abs(abs(got) / abs(ref) - 1) < 3e-3, d
        assert abs(np.angle(got / ref)) < 3e-3, d


def test_gpu_slab_config_full(bvf, orc):
    """64^3, dx 0.5 mm, 400 steps, 3-cycle 500 kHz plane burst onto the
    cortical/trabecular/cortical slab, 2 SLS, 8-cell CPML: pressure and peak."""
    from paper_2301_12727_gb300 import synth
    c = synth.slab_case()
    s, A = make_pair(bvf, orc, c)
    s.set_source(c.plane, c.k_src, c.c0, c.envelope, c.n_cycles)
    A.set_source(c.plane, c.k_src, c.c0, c.envelope, c.n_cycles)
    s.run(c.n_steps, peak_from=0)
    s.synchronize()
    assert A.run(c.n_steps, peak_from=0) == 0
    e_p = rel_l2(s.pressure().cpu().numpy(), A.pressure())
    e_pk = rel_l2(s.peak().cpu().numpy(), A.peak)
    assert e_p < TOL and e_pk < TOL, (e_p, e_pk)
    # the wave reached and crossed the slab (the check is not vacuous)
    assert A.peak[40, 32, 32] > 0.1 * A.peak[20, 32, 32]


def test_gpu_rs_plane_matches_oracle(bvf, orc):
    """Rayleigh-Sommerfeld bowl field on a plane (tilted bowl, ragged size)."""
    import torch
    nx, ny, dx, f0 = 77, 61, 0.5e-3, 5e5
    t = math.radians(10.0)
    bowl = dict(aperture=30e-3, roc=32e-3, apex=(19e-3, 15e-3, -6e-3),
                dir=(math.sin(t), 0.0, math.cos(t)), p0=6e4)
    zp = 4e-3
    got = bvf.rs_plane(bowl, nx, ny, dx, zp, f0).cpu().numpy()
    got = got[..., 0] + 1j * got[..., 1]
    ref = orc.rs_plane(bowl["aperture"], bowl["roc"], bowl["apex"], bowl["dir"], nx, ny, dx, zp,
                       f0, 1500.0, bowl["p0"])
    assert rel_l2(np.abs(got), np.abs(ref)) < 2e-5
    assert np.abs(got - ref).max() / np.abs(ref).max() < 5e-5


def test_gpu_skull_bowl_reduced(bvf, orc):
    """Skull-shaped phantom with a focused bowl (scaled to a 64 x 64 x 56 grid),
    ramp + CW source from each side's own Rayleigh-Sommerfeld plane, peak map
    and FP64 amplitude/phase over the last 2 cycles."""
    from paper_2301_12727_gb300 import synth
    c = synth.skull_case(64, 64, 56, dx=0.5e-3, n_steps=8 * 46, aperture=24e-3, roc=22e-3,
                         dft_cycles=2, n_pml=6, seed=5)
    s, A = make_pair(bvf, orc, c)
    b = c.bowl
    z_plane = c.k_src * c.dx
    plane_gpu = bvf.rs_plane(b, c.nx, c.ny, c.dx, z_plane, c.f0)
    s.set_source(plane_gpu, c.k_src, c.c0, c.envelope)
    plane_ref = orc.rs_plane(b["aperture"], b["roc"], b["apex"], b["dir"], c.nx, c.ny, c.dx,
                             z_plane, c.f0, c.c0, b["p0"])
    A.set_source(plane_ref, c.k_src, c.c0, c.envelope)
    s.run(c.n_steps, peak_from=0, dft_start=c.dft_start, dft_steps=c.dft_steps)
    s.synchronize()
    assert A.run(c.n_steps, peak_from=0, dft_start=c.dft_start, dft_steps=c.dft_steps) == 0
    amp_g, ph_g = s.amp_phase()
    amp_r, ph_r = A.amp_phase(c.dft_steps)
    assert rel_l2(s.pressure().cpu().numpy(), A.pressure()) < TOL
    assert rel_l2(s.peak().cpu().numpy(), A.peak) < TOL
    amp_g = amp_g.cpu().numpy()
    assert rel_l2(amp_g, amp_r) < TOL
    # phase where the amplitude is significant
    sig = amp_r > 0.05 * amp_r.max()
    dph = np.angle(np.exp(1j * (ph_g.cpu().numpy()[sig] - ph_r[sig])))
    assert np.abs(dph).max() < 1e-3


def test_gpu_thermal_matches_oracle(bvf, orc):
    """BHTE + CEM43 from an amplitude map on a layered phantom: final T, T_max
    and CEM43 (FP64 accumulation on the GPU)."""
    import torch
    from paper_2301_12727_gb300 import synth
    c = synth.skull_case(40, 36, 30, dx=0.5e-3, n_steps=10, n_pml=4, seed=9)
    z, y, x = np.meshgrid(np.arange(c.nz), np.arange(c.ny), np.arange(c.nx), indexing="ij")
    amp = 4e6 * np.exp(-((z - 20) ** 2 / 30.0 + (y - 18) ** 2 / 12.0 + (x - 20) ** 2 / 12.0))
    dt, n_on, n_off, duty = 0.05, 200, 100, 0.3
    s = bvf.Solver(c.nx, c.ny, c.nz, c.dx, c.dt, c.f0, n_sls=2, n_pml=c.n_pml)
    s.set_materials(c.index, c.materials)
    T, Tmax, cem = s.thermal(torch.from_numpy(amp).cuda(), dt, n_on, n_off, duty)
    torch.cuda.synchronize()
    rc, Tr, Tmr, cr = orc.bhte_run(c.index, c.materials, c.dx, amp, 1.0, dt, n_on, n_off, duty)
    assert rc == 0
    assert Tmr.max() > 40.0        # real heating happened
    assert rel_l2(T.cpu().numpy() - 37.0, Tr - 37.0) < TOL
    assert rel_l2(Tmax.cpu().numpy() - 37.0, Tmr - 37.0) < TOL
    assert rel_l2(cem.cpu().numpy(), cr) < 1e-3


def test_gpu_thermal_tma_matches_oracle_and_direct_kernel(bvf, orc, monkeypatch):
    """The TMA-fed BHTE step (nx % 8 == 0) on a grid with a ragged y tile
    and a ragged last z-chunk: T, T_max and CEM43 against the oracle, and bit
    for bit against the direct kernel on the same inputs (the flush of the
    FP32 dose partial included: 301 steps)."""
    import torch
    from paper_2301_12727_gb300 import synth
    c = synth.skull_case(48, 37, 30, dx=0.5e-3, n_steps=10, n_pml=4, seed=11)
    z, y, x = np.meshgrid(np.arange(c.nz), np.arange(c.ny), np.arange(c.nx), indexing="ij")
    amp = 4e6 * np.exp(-((z - 17) ** 2 / 30.0 + (y - 18) ** 2 / 12.0 + (x - 23) ** 2 / 12.0))
    dt, n_on, n_off, duty = 0.05, 201, 100, 0.3
    out = {}
    for kernel in ("tma", "direct"):
        if kernel == "direct":
            monkeypatch.setenv("BVF_NO_TMA", "1")
        s = bvf.Solver(c.nx, c.ny, c.nz, c.dx, c.dt, c.f0, n_sls=2, n_pml=c.n_pml)
        s.set_materials(c.index, c.materials)
        T, Tmax, cem = s.thermal(torch.from_numpy(amp).cuda(), dt, n_on, n_off, duty)
        torch.cuda.synchronize()
        out[kernel] = (T.cpu().numpy(), Tmax.cpu().numpy(), cem.cpu().numpy())
        s.close()
    monkeypatch.delenv("BVF_NO_TMA", raising=False)
    for a, b in zip(out["tma"], out["direct"]):
        np.testing.assert_array_equal(a, b)
    rc, Tr, Tmr, cr = orc.bhte_run(c.index, c.materials, c.dx, amp, 1.0, dt, n_on, n_off, duty)
    assert rc == 0
    T, Tmax, cem = out["tma"]
    assert Tmr.max() > 40.0
    assert rel_l2(T - 37.0, Tr - 37.0) < TOL
    assert rel_l2(Tmax - 37.0, Tmr - 37.0) < TOL
    assert rel_l2(cem, cr) < 1e-3


def test_gpu_transmission_matches_oracle(bvf, orc):
    """E_L (Eq. 2) and z_m from the same FP64 maps on both sides."""
    import torch
    rng = np.random.default_rng(2)
    nz, ny, nx = 30, 26, 22
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    amp_w = np.exp(-((z - 17) ** 2 / 20.0 + (y - 12) ** 2 / 9.0 + (x - 10) ** 2 / 9.0))
    amp_a = amp_w * (0.3 + 0.4 * rng.random(amp_w.shape))
    idx_a = rng.integers(0, 3, amp_w.shape).astype(np.uint8)
    idx_w = np.zeros_like(idx_a)
    ma = [mat_row(1000.0, 1500.0), mat_row(1041.0, 1562.0), mat_row(1116.0, 1537.0)]
    mw = [mat_row(1000.0, 1500.0)]
    el_r, zm_r = orc.transmission(idx_a, ma, amp_a, idx_w, mw, amp_w)
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    el, ts, zm, iw = bvf.bvf_transmission(cu(idx_a), ma, cu(amp_a), cu(idx_w), mw, cu(amp_w))
    assert zm == zm_r == 17
    assert el == pytest.approx(el_r, rel=1e-12)
    assert ts == pytest.approx(math.sqrt(el_r), rel=1e-12)
    assert iw == pytest.approx((amp_w ** 2).max() / (2 * 1000.0 * 1500.0), rel=1e-14)


# --------------------------------------------------------------------------
# error paths (failures made on the host; nothing faults the GPU)
# --------------------------------------------------------------------------
def test_gpu_error_paths(bvf):
    import torch
    n, dx = 24, 0.5e-3
    mats = [mat_row(1000.0, 1500.0), mat_row(1850.0, 2800.0, 1500.0, 85.0, 170.0)]
    s = bvf.Solver(n, n, n, dx, 0.6 * dx / 2800.0, 5e5, n_sls=2, n_pml=4)
    with pytest.raises(bvf.BvfError) as e:          # CFL: 0.6 > 6/(7 sqrt 3)
        s.set_materials(np.zeros((n, n, n), np.uint8), mats)
    assert e.value.code == bvf.BVF_E_CFL
    s.close()
    s = bvf.Solver(n, n, n, dx, 0.2 * dx / 2800.0, 5e5, n_sls=2, n_pml=4)
    with pytest.raises(bvf.BvfError) as e:          # index beyond the table (device scan)
        s.set_materials(np.full((n, n, n), 2, np.uint8), mats)
    assert e.value.code == bvf.BVF_E_MATERIAL
    with pytest.raises(bvf.BvfError) as e:          # Poisson ratio below -1
        s.set_materials(np.zeros((n, n, n), np.uint8), [mat_row(1000.0, 1500.0, 1400.0)])
    assert e.value.code == bvf.BVF_E_MATERIAL
    with pytest.raises(bvf.BvfError) as e:          # run before materials
        s.run(1)
    assert e.value.code == bvf.BVF_E_ARG
    s.set_materials(np.zeros((n, n, n), np.uint8), mats)
    bad = np.zeros((n, n, n), np.float32)
    bad[12, 12, 12] = np.nan                        # non-finite state made on the host
    s.set_field("sxx", bad)
    s.run(3)
    with pytest.raises(bvf.BvfError) as e:
        s.synchronize()
    assert e.value.code == bvf.BVF_E_UNSTABLE
    s.reset()
    s.run(3)
    s.synchronize()                                 # reset clears the flag
    with pytest.raises(bvf.BvfError):
        s.amp_phase()                               # nothing captured
    s.close()


@pytest.mark.parametrize("shape,n_sls", [((1, 1, 1), 2), ((2, 3, 4), 2), ((16, 1, 5), 2),
                                         ((3, 2, 1), 1), ((32, 9, 7), 0), ((24, 20, 18), 3)])
def test_gpu_degenerate_grids_match_oracle(bvf, orc, shape, n_sls):
    """Grids with single-cell axes (everything a ghost or a boundary), a TMA
    grid one row high, a lossless medium and three SLS mechanisms (direct
    kernels): every state array after 5 steps from a random state equals the
    oracle's to FP32 rounding."""
    nx, ny, nz = shape
    dx = 0.5e-3
    rng = np.random.default_rng(sum(shape) + n_sls)
    mats = [mat_row(1000.0, 1500.0), mat_row(1850.0, 2800.0, 1500.0, 85.0, 170.0)]
    index = rng.integers(0, 2, size=(nz, ny, nx)).astype(np.uint8)
    from paper_2301_12727_gb300 import synth
    dt, _ = synth.choose_dt(dx, 2800.0, 5e5)
    s = bvf.Solver(nx, ny, nz, dx, dt, 5e5, n_sls=n_sls, n_pml=0)
    s.set_materials(index, mats)
    A = orc.Acoustic(nx, ny, nz, dx, dt, index, mats, 5e5, n_sls=n_sls, n_pml=0)
    n_state = 9 + 6 * n_sls
    d = {f: (rng.standard_normal((nz, ny, nx)) * (1.0 if f[0] == "v" else 1e6)).astype(np.float32)
         for f in an.FIELDS}
    an.zero_ghost_half_points(d)
    for i in range(n_state):
        if i < 9:
            v = d[an.FIELDS[i]]
        else:       # memory variables vanish where their stress is a ghost
            c = (i - 9) % 6
            v = (rng.standard_normal((nz, ny, nx)) * 1e4).astype(np.float32)
            if c >= 3:
                v *= (d[an.FIELDS[3 + c]] != 0)
        s.set_field(i, v)
        A.state[i] = v.astype(np.float64)
    s.run(5)
    s.synchronize()
    assert A.run(5) == 0
    for i in range(n_state):
        got = s.field(i).cpu().numpy()
        ref = A.state[i]
        scale = max(np.abs(ref).max(), 1e-30)
        assert np.abs(got - ref).max() <= 2e-5 * scale, (i, np.abs(got - ref).max() / scale)
    s.close()


def test_gpu_zero_steps_change_nothing(bvf):
    n = 16
    s = bvf.Solver(n, n, n, 0.5e-3, 5e-8, 5e5, n_sls=2, n_pml=0)
    s.set_materials(np.zeros((n, n, n), np.uint8), [mat_row(1000.0, 1500.0)])
    v = np.random.default_rng(0).standard_normal((n, n, n)).astype(np.float32)
    s.set_field("sxx", v)
    s.run(0)
    s.synchronize()
    assert np.array_equal(s.field("sxx").cpu().numpy(), v)
    assert s.stats().steps == 0
    s.close()


def test_gpu_run_twice_is_bitwise_identical(bvf):
    """No atomics on field data: two runs from the same state agree bitwise."""
    from paper_2301_12727_gb300 import synth
    c = synth.skull_case(56, 48, 40, dx=0.5e-3, n_steps=150, aperture=20e-3, roc=20e-3, n_pml=6)
    outs = []
    for _ in range(2):
        s = bvf.Solver(c.nx, c.ny, c.nz, c.dx, c.dt, c.f0, n_sls=2, n_pml=c.n_pml)
        s.set_materials(c.index, c.materials)
        s.set_source(bvf.rs_plane(c.bowl, c.nx, c.ny, c.dx, c.k_src * c.dx, c.f0), c.k_src,
                     c.c0, c.envelope)
        s.run(c.n_steps, peak_from=0, dft_start=51, dft_steps=92)
        s.synchronize()
        outs.append((s.pressure().cpu().numpy(), s.peak().cpu().numpy(),
                     s.amp_phase()[0].cpu().numpy()))
        s.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("nx", [50, 64])
def test_gpu_zchunk_invariance(bvf, monkeypatch, nx):
    """The z-marching kernels split z into chunks per block; the per-voxel
    arithmetic does not depend on the split, so any chunk length gives the
    same fields bit for bit (covers queue start-up at every chunk edge), for
    the direct kernels (nx = 50) and the TMA-fed ones (nx = 64)."""
    from paper_2301_12727_gb300 import synth
    c = synth.skull_case(nx, 41, 37, dx=0.5e-3, n_steps=90, aperture=16e-3, roc=16e-3, n_pml=5)
    outs = []
    for kc in ("1", "3", "37", "0"):
        monkeypatch.setenv("BVF_KCHUNK", kc)
        s = bvf.Solver(c.nx, c.ny, c.nz, c.dx, c.dt, c.f0, n_sls=2, n_pml=c.n_pml)
        s.set_materials(c.index, c.materials)
        s.set_source(bvf.rs_plane(c.bowl, c.nx, c.ny, c.dx, c.k_src * c.dx, c.f0), c.k_src,
                     c.c0, c.envelope)
        s.run(c.n_steps, peak_from=0)
        s.synchronize()
        outs.append([s.field(f).cpu().numpy() for f in range(21)] + [s.peak().cpu().numpy()])
        s.close()
    assert np.abs(outs[0][3]).max() > 0
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_gpu_tma_and_direct_paths_agree_bitwise(bvf, monkeypatch, storage):
    """Grids with nx % 8 == 0 run the TMA-fed kernels (tiles, rings and
    in-place stages moved by the tensor-memory accelerator); other shapes, or
    BVF_NO_TMA, run the direct kernels.  Same arithmetic, so every field, the
    peak map and the FP64 DFT agree bit for bit, across z-chunk lengths (chunk
    prologues) and a partial x-tile (nx = 80), in both storage types."""
    from paper_2301_12727_gb300 import synth
    c = synth.skull_case(80, 48, 40, dx=0.5e-3, n_steps=120, aperture=16e-3, roc=16e-3, n_pml=5)
    outs = []
    for no_tma, st_tma, kc in (("", "1", "0"), ("", "1", "3"), ("", "1", "1"), ("", "0", "0"),
                               ("1", "", "0")):
        monkeypatch.setenv("BVF_KCHUNK", kc)
        monkeypatch.setenv("BVF_STRESS_TMA", st_tma)
        if no_tma:
            monkeypatch.setenv("BVF_NO_TMA", "1")
        else:
            monkeypatch.delenv("BVF_NO_TMA", raising=False)
        s = bvf.Solver(c.nx, c.ny, c.nz, c.dx, c.dt, c.f0, n_sls=2, n_pml=c.n_pml,
                       storage=storage)
        s.set_materials(c.index, c.materials)
        s.set_source(bvf.rs_plane(c.bowl, c.nx, c.ny, c.dx, c.k_src * c.dx, c.f0), c.k_src,
                     c.c0, c.envelope)
        s.run(c.n_steps, peak_from=10, dft_start=c.n_steps - 45, dft_steps=46)
        s.synchronize()
        amp, ph = s.amp_phase()
        outs.append([s.field(f).cpu().numpy() for f in range(21)] +
                    [s.peak().cpu().numpy(), amp.cpu().numpy(), ph.cpu().numpy()])
        s.close()
    assert np.abs(outs[0][21]).max() > 0
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_gpu_tile_heights_agree_bitwise(bvf, storage):
    """The TMA-fed kernels cut the grid into x-y tiles 4, 8 or 16 rows high,
    chosen per kernel (bvf_set_tile); the tiling changes no arithmetic, so
    every field, the peak map and the FP64 DFT agree bit for bit with the
    default tiles (stress 8, velocity 16 rows), on a grid whose y extent (45)
    leaves a partial tile at every height, with CPML slabs, a source plane and
    z-chunks of several lengths."""
    from paper_2301_12727_gb300 import synth
    c = synth.skull_case(64, 45, 36, dx=0.5e-3, n_steps=90, aperture=16e-3, roc=16e-3, n_pml=5)
    outs = []
    for sr, vr, kc in ((0, 0, 0), (8, 8, 0), (4, 4, 0), (16, 16, 0), (4, 16, 5), (16, 4, 7),
                       (8, 8, 3)):
        s = bvf.Solver(c.nx, c.ny, c.nz, c.dx, c.dt, c.f0, n_sls=2, n_pml=c.n_pml,
                       storage=storage)
        s.set_tile(sr, vr, kc)
        assert s.tile()[:2] == (sr or 8, vr or 16)
        s.set_materials(c.index, c.materials)
        s.set_source(bvf.rs_plane(c.bowl, c.nx, c.ny, c.dx, c.k_src * c.dx, c.f0), c.k_src,
                     c.c0, c.envelope)
        s.run(c.n_steps, peak_from=10, dft_start=c.n_steps - 45, dft_steps=46)
        s.synchronize()
        amp, ph = s.amp_phase()
        outs.append([s.field(f).cpu().numpy() for f in range(21)] +
                    [s.peak().cpu().numpy(), amp.cpu().numpy(), ph.cpu().numpy()])
        s.close()
    assert np.abs(outs[0][21]).max() > 0
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_gpu_tma_path_on_rows_of_eight_agrees_with_direct_kernels(bvf, monkeypatch, storage):
    """nx = 72 (a multiple of 8, not of 16): the TMA-fed kernels run, their
    index maps reading a copy with rows padded to 16 bytes; every field, the
    peak map and the FP64 DFT equal the direct kernels' bit for bit, and so do
    the BHTE outputs."""
    import torch
    from paper_2301_12727_gb300 import synth
    c = synth.skull_case(72, 41, 30, dx=0.5e-3, n_steps=80, aperture=16e-3, roc=16e-3, n_pml=5)
    z, y, x = np.meshgrid(np.arange(c.nz), np.arange(c.ny), np.arange(c.nx), indexing="ij")
    amp = torch.from_numpy(3e6 * np.exp(-((z - 15) ** 2 + (y - 20) ** 2 + (x - 36) ** 2) / 40.0)).cuda()
    outs = []
    for no_tma in (False, True):
        if no_tma:
            monkeypatch.setenv("BVF_NO_TMA", "1")
        s = bvf.Solver(c.nx, c.ny, c.nz, c.dx, c.dt, c.f0, n_sls=2, n_pml=c.n_pml,
                       storage=storage)
        s.set_materials(c.index, c.materials)
        if not no_tma:      # the hook is accepted only by a context on the TMA kernels
            bvf.bvf_test_withhold_copy(s.ctx, 1, 3, 64)
            bvf.bvf_test_withhold_copy(s.ctx, 0, 0, 0)
        s.set_source(bvf.rs_plane(c.bowl, c.nx, c.ny, c.dx, c.k_src * c.dx, c.f0), c.k_src,
                     c.c0, c.envelope)
        s.run(c.n_steps, peak_from=10, dft_start=c.n_steps - 45, dft_steps=46)
        s.synchronize()
        amp_, ph = s.amp_phase()
        T = s.thermal(amp, 0.05, 40, 20, 0.3)
        s.synchronize()
        outs.append([s.field(f).cpu().numpy() for f in range(21)] +
                    [s.peak().cpu().numpy(), amp_.cpu().numpy(), ph.cpu().numpy()] +
                    [t.cpu().numpy() for t in T])
        s.close()
    monkeypatch.delenv("BVF_NO_TMA", raising=False)
    assert np.abs(outs[0][21]).max() > 0
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)


def test_gpu_set_tile_rejects_bad_heights(bvf):
    s = bvf.Solver(32, 16, 16, 1e-3, 1e-7, 5e5, n_sls=2, n_pml=0)
    for bad in ((3, 8, 0), (8, 32, 0), (8, 8, -1)):
        with pytest.raises(bvf.BvfError):
            s.set_tile(*bad)
    s.close()
    s1 = bvf.Solver(32, 16, 16, 1e-3, 1e-7, 5e5, n_sls=1, n_pml=0)
    s1.set_tile(16, 16, 0)
    assert s1.tile()[:2] == (8, 8)    # heights other than 8 need two SLS mechanisms
    s1.close()


# --------------------------------------------------------------------------
# FP16 storage: the state rounded to FP16 between steps, FP32 arithmetic.
# A stored value carries a relative rounding error of at most 2^-11; the
# steps of a run add such errors in random directions and transport them with
# the wave, so the accepted error is the one the storage format is meant to
# meet: 1 % of the peak pressure (relative L2 of a whole field below 1 %).
F16_TOL = 1e-2


def test_gpu_f16_slab_matches_oracle(bvf, orc):
    """The 64^3 slab burst with FP16 storage against the FP64 oracle."""
    from paper_2301_12727_gb300 import synth
    c = synth.slab_case()
    s, A = make_pair(bvf, orc, c, storage="f16")
    s.set_source(c.plane, c.k_src, c.c0, c.envelope, c.n_cycles)
    A.set_source(c.plane, c.k_src, c.c0, c.envelope, c.n_cycles)
    s.run(c.n_steps, peak_from=0)
    s.synchronize()
    assert A.run(c.n_steps, peak_from=0) == 0
    peak = s.peak().cpu().numpy()
    assert rel_l2(s.pressure().cpu().numpy(), A.pressure()) < F16_TOL
    assert np.abs(peak - A.peak).max() < F16_TOL * A.peak.max()
    assert rel_l2(peak, A.peak) < F16_TOL


def test_gpu_f16_skull_bowl_matches_oracle(bvf, orc):
    """Focused bowl through the reduced skull phantom with FP16 storage: peak
    map and FP64 amplitude within 1 %, phase within 0.01 rad where the beam
    carries at least 10 % of the largest amplitude."""
    from paper_2301_12727_gb300 import synth
    c = synth.skull_case(64, 64, 56, dx=0.5e-3, n_steps=8 * 46, aperture=24e-3, roc=22e-3,
                         dft_cycles=2, n_pml=6, seed=5)
    s, A = make_pair(bvf, orc, c, storage="f16")
    b = c.bowl
    z_plane = c.k_src * c.dx
    s.set_source(bvf.rs_plane(b, c.nx, c.ny, c.dx, z_plane, c.f0), c.k_src, c.c0, c.envelope)
    A.set_source(orc.rs_plane(b["aperture"], b["roc"], b["apex"], b["dir"], c.nx, c.ny, c.dx,
                              z_plane, c.f0, c.c0, b["p0"]), c.k_src, c.c0, c.envelope)
    s.run(c.n_steps, peak_from=0, dft_start=c.dft_start, dft_steps=c.dft_steps)
    s.synchronize()
    assert A.run(c.n_steps, peak_from=0, dft_start=c.dft_start, dft_steps=c.dft_steps) == 0
    amp_g, ph_g = (t.cpu().numpy() for t in s.amp_phase())
    amp_r, ph_r = A.amp_phase(c.dft_steps)
    peak = s.peak().cpu().numpy()
    assert np.abs(peak - A.peak).max() < F16_TOL * A.peak.max()
    assert np.abs(amp_g - amp_r).max() < F16_TOL * amp_r.max()
    beam = amp_r > 0.1 * amp_r.max()
    assert np.abs(np.angle(np.exp(1j * (ph_g - ph_r))))[beam].max() < 1e-2


def test_gpu_f16_fields_round_trip_through_the_storage_scales(bvf):
    """bvf_set_field / bvf_get_field in FP16 storage: physical FP32 values in
    and out, stored as the FP16 rounding of value / scale (scales p_ref for
    stresses, p_ref / 1.5e6 for velocities)."""
    import torch
    p_ref = 2.0 ** 15
    s = bvf.Solver(32, 16, 16, 1e-3, 1e-7, 5e5, n_sls=2, n_pml=0, storage="f16", p_ref=p_ref)
    rng = np.random.default_rng(3)
    for fid, scale in ((0, p_ref / 1.5e6), (3, p_ref), (7, p_ref)):
        v = (rng.standard_normal((16, 16, 32)) * 40.0 * scale).astype(np.float32)
        s.set_field(fid, torch.from_numpy(v).cuda())
        got = s.field(fid).cpu().numpy()
        inv = np.float32(1.0 / scale)
        expect = (v * inv).astype(np.float16).astype(np.float32) * np.float32(scale)
        assert np.array_equal(got, expect), fid
        assert np.abs(got - v).max() <= 2.0 ** -11 * np.abs(v).max() * 1.001
    s.close()


def test_gpu_plan_with_host_buffers_equals_the_device_call(bvf):
    """bvf_plan_host (host index in, host maps out, the copies inside the
    call) gives bvf_plan's maps and scalars bit for bit, on repeated calls."""
    import torch
    from paper_2301_12727_gb300 import plan, synth
    c = synth.skull_case(64, 48, 40, dx=0.5e-3, n_steps=4 * 46, aperture=20e-3, roc=18e-3,
                         dft_cycles=2, n_pml=5, seed=8)
    regime = plan.ThermalRegime(t_on=1.0, t_off=0.5, dt=0.1)
    pl = plan.Planner(c)
    r = pl.run(torch.from_numpy(c.index).cuda(), c.materials, c.bowl, regime=regime)
    want = [r.peak.cpu().numpy(), r.Tmax.cpu().numpy(), r.cem43.cpu().numpy()]
    h_idx = torch.from_numpy(c.index).pin_memory()
    peak = torch.empty(c.index.shape, dtype=torch.float32).pin_memory()
    Tmax = torch.empty_like(peak).pin_memory()
    T = torch.empty_like(peak).pin_memory()
    cem = torch.empty(c.index.shape, dtype=torch.float64).pin_memory()
    for _ in range(2):
        out = pl.run_host(h_idx, c.materials, c.bowl, peak, Tmax, cem, T=T, regime=regime)
        assert out.EL == r.EL and out.z_m == r.z_m and out.p_scale == r.p_scale
        for a, b in zip((peak.numpy(), Tmax.numpy(), cem.numpy()), want):
            assert np.array_equal(a, b)
    assert T.numpy().max() > regime.T_a
    pl.close()


def test_gpu_plan_call_equals_the_step_by_step_sequence(bvf):
    """bvf_plan (one C-ABI call) gives exactly what the separate calls give:
    skull and water runs, E_L, T_S, z_m, I_w,max, the scaling and the BHTE."""
    import torch
    from paper_2301_12727_gb300 import plan, synth
    c = synth.skull_case(64, 64, 56, dx=0.5e-3, n_steps=5 * 46, aperture=24e-3, roc=22e-3,
                         dft_cycles=2, n_pml=6, seed=5)
    regime = plan.ThermalRegime(t_on=2.0, t_off=1.0, dt=0.1)
    idx = torch.from_numpy(c.index).cuda()
    pl = plan.Planner(c)
    r = pl.run(idx, c.materials, c.bowl, regime=regime)
    pl.close()
    # the same steps, one call at a time
    sk = bvf.Solver(c.nx, c.ny, c.nz, c.dx, c.dt, c.f0, n_sls=2, n_pml=c.n_pml)
    wa = bvf.Solver(c.nx, c.ny, c.nz, c.dx, c.dt, c.f0, n_sls=2, n_pml=c.n_pml)
    sk.set_materials(idx, c.materials)
    widx = torch.zeros_like(idx)
    wtab = np.array([synth.water_row(c.f0)])
    wa.set_materials(widx, wtab)
    plane = bvf.rs_plane(c.bowl, c.nx, c.ny, c.dx, c.k_src * c.dx, c.f0)
    for s in (sk, wa):
        s.set_source(plane, c.k_src, 1500.0, bvf.BVF_ENV_RAMP_CW)
        s.run(c.n_steps, peak_from=0, dft_start=c.dft_start, dft_steps=c.dft_steps)
    amp, _ = sk.amp_phase()
    amp_w, _ = wa.amp_phase()
    EL, TS, zm, Iw = bvf.bvf_transmission(idx, c.materials, amp, widx, wtab, amp_w)
    assert (EL, TS, zm, Iw) == (r.EL, r.TS, r.z_m, r.Iw_max)
    p_scale = float(np.sqrt(5.0e4 / (EL * Iw)))
    assert p_scale == r.p_scale
    T, Tmax, cem = sk.thermal(amp, regime.dt, regime.n_on, regime.n_off, regime.duty,
                              T_a=regime.T_a, rhob_cb=regime.rhob_cb, p_scale=p_scale)
    assert torch.equal(sk.peak(), r.peak) and torch.equal(amp, r.amp)
    assert torch.equal(Tmax, r.Tmax) and torch.equal(cem, r.cem43)
    assert float(r.Tmax.max()) > 37.0 and 0.0 < r.EL < 1.0
    sk.close()
    wa.close()
