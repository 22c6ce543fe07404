"""Properties of whole plans at the benchmark's full size and launch
configuration (240 x 240 x 200 skull, 1500 FDTD steps, 10-cycle DFT, BHTE),
where the oracle cannot follow: exact mirror symmetry, bitwise repeatability,
and E_L = 1 when the skull run sees only water."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    assert torch.cuda.is_available()
    from paper_2301_12727_gb300 import build
    build.build()
    from paper_2301_12727_gb300 import bvf, plan, synth
    return bvf, plan, synth


def symmetrise(plane):
    """Average a (ny, nx, 2) source plane over the two lateral mirrors, summed
    pairwise so that the result is exactly symmetric."""
    return 0.25 * ((plane + plane.flip(1)) + (plane.flip(0) + plane.flip(0).flip(1)))


def test_fullsize_mirror_symmetry(mods):
    import torch
    bvf, plan, synth = mods
    c = synth.skull_case(240, 240, 200, n_steps=1500, symmetric=True)
    idx = c.index
    assert np.array_equal(idx, idx[:, :, ::-1]) and np.array_equal(idx, idx[:, ::-1, :])
    s = bvf.Solver(c.nx, c.ny, c.nz, c.dx, c.dt, c.f0, n_sls=2, n_pml=c.n_pml)
    s.set_materials(idx, c.materials)
    pl = symmetrise(bvf.rs_plane(c.bowl, c.nx, c.ny, c.dx, c.k_src * c.dx, c.f0)).contiguous()
    s.set_source(pl, c.k_src, c.c0, c.envelope)
    s.run(c.n_steps, peak_from=0, dft_start=c.dft_start, dft_steps=c.dft_steps)
    s.synchronize()
    peak = s.peak().cpu().numpy()
    p = s.pressure().cpu().numpy()
    amp = s.amp_phase()[0].cpu().numpy()
    s.close()
    assert peak.max() > 0
    for a in (peak, p, amp):
        assert np.array_equal(a, a[:, :, ::-1])
        assert np.array_equal(a, a[:, ::-1, :])


def test_fullsize_plan_is_repeatable_and_focuses(mods):
    import torch
    bvf, plan, synth = mods
    c = synth.skull_case(240, 240, 200, n_steps=1500)
    pl = plan.Planner(c)
    idx = torch.from_numpy(c.index).cuda()
    outs = []
    for _ in range(2):
        r = pl.run(idx, c.materials, c.bowl)
        outs.append((r.peak.cpu().numpy(), r.amp.cpu().numpy(), r.Tmax.cpu().numpy(),
                     r.cem43.cpu().numpy(), r.EL, r.zm if hasattr(r, "zm") else r.z_m))
    pl.close()
    for a, b in zip(outs[0], outs[1]):
        if isinstance(a, np.ndarray):
            assert np.array_equal(a, b)
        else:
            assert a == b
    peak, amp, Tmax, cem, EL, zm = outs[0]
    # the water-run focus lies in the brain, deeper than the skull, and the
    # transmission is a fraction
    assert 0.0 < EL < 1.0
    # plausibility only (parity unpinned: the paper's CT data are not here): the
    # paper's sub-MHz transmission through real skulls, T_S = sqrt(E_L), lies
    # in about 0.2 .. 0.6 (Results, Figs. 5-6); the synthetic skull falls there
    assert 0.2 < EL ** 0.5 < 0.6
    assert zm > c.k_src + 20
    assert np.isfinite(Tmax).all() and Tmax.max() > 37.0 and (cem >= 0).all()


def test_fullsize_transmission_is_one_for_water(mods):
    import torch
    bvf, plan, synth = mods
    c = synth.skull_case(240, 240, 200, n_steps=1500)
    w = synth.water_like(c)
    pl = plan.Planner(w)
    r = pl.run(torch.from_numpy(w.index).cuda(), w.materials, w.bowl)
    pl.close()
    assert r.EL == 1.0 and r.TS == 1.0


def test_fullsize_f16_storage_within_one_percent_of_f32(mods):
    """FP16 storage at the benchmark's workload (skull run, 1500 steps): peak
    map within 1 % of the FP32 run's largest peak everywhere, focal peak and
    FP64 amplitude within 1 %, phase within 0.01 rad in the beam."""
    bvf, plan, synth = mods
    c = synth.skull_case(240, 240, 200, n_steps=1500)
    out = {}
    for st in ("f32", "f16"):
        s = bvf.Solver(c.nx, c.ny, c.nz, c.dx, c.dt, c.f0, n_sls=2, n_pml=c.n_pml, storage=st)
        s.set_materials(c.index, c.materials)
        s.set_source(bvf.rs_plane(c.bowl, c.nx, c.ny, c.dx, c.k_src * c.dx, c.f0), c.k_src,
                     c.c0, c.envelope)
        s.run(c.n_steps, peak_from=0, dft_start=c.dft_start, dft_steps=c.dft_steps)
        s.synchronize()
        amp, ph = s.amp_phase()
        out[st] = (s.peak().cpu().numpy(), amp.cpu().numpy(), ph.cpu().numpy())
        s.close()
    (p32, a32, f32), (p16, a16, f16) = out["f32"], out["f16"]
    assert abs(p16.max() - p32.max()) < 1e-2 * p32.max()
    assert np.abs(p16 - p32).max() < 1e-2 * p32.max()
    assert np.abs(a16 - a32).max() < 1e-2 * a32.max()
    beam = a32 > 0.1 * a32.max()
    assert np.abs(np.angle(np.exp(1j * (f16 - f32))))[beam].max() < 1e-2
