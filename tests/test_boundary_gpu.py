"""Boundary calls beyond the field accessors, through the C ABI on the GPU:

* the bounded TMA waits: a copy held back (the barrier armed, no copy
  issued, so nothing is ever in flight) makes the waiting blocks give up, stop
  and report BVF_E_CUDA through bvf_synchronize; the same context then runs
  exactly like a fresh one;
* snapshots: bvf_state_save / bvf_state_load resume a run bit for bit,
  capture window included, in FP32 and FP16 storage, and refuse a snapshot of
  another grid;
* the per-call wall-clock budget: BVF_E_TIMEOUT after whole chunks of steps,
  leaving a consistent state that a later call continues (acoustic: bit for
  bit; thermal: up to the one FP32 rounding of T at the stop)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    assert torch.cuda.is_available()
    from paper_2301_12727_gb300 import build
    build.build()
    from paper_2301_12727_gb300 import bvf, synth
    return bvf, synth


def small_case(synth, nx=48, ny=48, nz=40):
    # nx % 8 == 0: the TMA-fed kernels run
    return synth.skull_case(nx, ny, nz, dx=0.5e-3, n_steps=90, aperture=20e-3, roc=18e-3,
                            n_pml=4, seed=11, dft_cycles=1)


def make_solver(bvf, c, storage="f32"):
    s = bvf.Solver(c.nx, c.ny, c.nz, c.dx, c.dt, c.f0, n_sls=2, n_pml=c.n_pml, storage=storage)
    s.set_materials(c.index, c.materials)
    s.set_source(bvf.rs_plane(c.bowl, c.nx, c.ny, c.dx, c.k_src * c.dx, c.f0), c.k_src, c.c0,
                 c.envelope)
    return s


def snapshot(bvf, s, with_dft=True):
    out = [s.field(f).cpu().numpy() for f in range(9 + 6 * s.n_sls)]
    out.append(s.peak().cpu().numpy())
    if with_dft:
        a, p = s.amp_phase()
        out += [a.cpu().numpy(), p.cpu().numpy()]
    return out


def assert_same(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("kernel,storage", [(1, "f32"), (2, "f32"), (2, "f16")])
def test_withheld_copy_times_out_and_context_recovers(mods, kernel, storage):
    """Kernel 1 (velocity) or 2 (stress; with FP16 storage the paired stress
    tile) arms the barrier of the copies it would issue at plane 3 of the
    first z-chunk but issues none: every block of that chunk gives up after
    its bounded wait, drains the copies it did issue and stops.
    bvf_synchronize reports BVF_E_CUDA with the time-out message; after
    bvf_reset the context's next 30 steps equal a fresh context's."""
    import torch
    bvf, synth = mods
    c = small_case(synth)
    s = make_solver(bvf, c, storage)
    bvf.bvf_test_withhold_copy(s.ctx, kernel, 3, 4096)
    s.run(2, peak_from=0)
    with pytest.raises(bvf.BvfError) as ei:
        s.synchronize()
    assert ei.value.code == bvf.BVF_E_CUDA
    assert "wait limit" in str(ei.value)
    # the hook applied to one step only; the context is usable after a reset
    s.reset()
    s.run(30, peak_from=0)
    s.synchronize()
    got = snapshot(bvf, s, with_dft=False)
    ref = make_solver(bvf, c, storage)
    ref.run(30, peak_from=0)
    ref.synchronize()
    assert_same(got, snapshot(bvf, ref, with_dft=False))
    s.close()
    ref.close()
    torch.cuda.synchronize()


def test_withheld_copy_of_the_bhte_step_times_out_and_context_recovers(mods):
    """Kernel 3: the first step of the next thermal call arms the ring barrier
    of plane 5 but issues none of its copies; the blocks that wait for it give
    up, drain and flag the time-out, bvf_synchronize reports BVF_E_CUDA, and
    after bvf_reset a thermal call equals a fresh context's bit for bit."""
    import torch
    bvf, synth = mods
    c = small_case(synth)
    z, y, x = np.meshgrid(np.arange(c.nz), np.arange(c.ny), np.arange(c.nx), indexing="ij")
    amp = torch.from_numpy(3e6 * np.exp(-((z - 20) ** 2 + (y - 24) ** 2 + (x - 24) ** 2) / 40.0)).cuda()
    s = make_solver(bvf, c)
    bvf.bvf_test_withhold_copy(s.ctx, 3, 5, 4096)
    s.thermal(amp, 0.05, 10, 5, 0.3)
    with pytest.raises(bvf.BvfError) as ei:
        s.synchronize()
    assert ei.value.code == bvf.BVF_E_CUDA
    assert "wait limit" in str(ei.value)
    s.reset()
    got = [t.cpu().numpy() for t in s.thermal(amp, 0.05, 10, 5, 0.3)]
    s.synchronize()
    ref = make_solver(bvf, c)
    want = [t.cpu().numpy() for t in ref.thermal(amp, 0.05, 10, 5, 0.3)]
    ref.synchronize()
    for a, b in zip(got, want):
        assert np.array_equal(a, b)
    s.close()
    ref.close()
    torch.cuda.synchronize()


def test_withhold_hook_rejects_direct_kernels_and_bad_planes(mods):
    bvf, synth = mods
    c = synth.skull_case(42, 40, 24, dx=0.5e-3, n_steps=10, aperture=16e-3, roc=15e-3, n_pml=3)
    s = make_solver(bvf, c)           # nx % 8 != 0: direct kernels
    for kernel in (1, 3):
        with pytest.raises(bvf.BvfError) as ei:
            bvf.bvf_test_withhold_copy(s.ctx, kernel, 3, 64)
        assert ei.value.code == bvf.BVF_E_ARG
    s.close()
    c = small_case(synth)
    s = make_solver(bvf, c)
    for kernel, plane in ((4, 2), (1, -1), (2, c.nz), (3, c.nz)):
        with pytest.raises(bvf.BvfError):
            bvf.bvf_test_withhold_copy(s.ctx, kernel, plane, 64)
    bvf.bvf_test_withhold_copy(s.ctx, 0, 0, 0)      # disarm is always accepted
    s.close()


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_snapshot_resumes_bit_for_bit(mods, storage):
    """Run 55 steps, save, run 35 more, load, run the 35 again: both endings
    equal the uninterrupted 90-step run bit for bit in every state array, the
    peak map and the FP64 amplitude and phase of a capture window (steps
    46..90) that spans the snapshot."""
    bvf, synth = mods
    c = small_case(synth)
    cap = dict(peak_from=0, dft_start=46, dft_steps=45)
    ref = make_solver(bvf, c, storage)
    ref.run(90, **cap)
    ref.synchronize()
    want = snapshot(bvf, ref)
    ref.close()
    s = make_solver(bvf, c, storage)
    s.run(55, **cap)
    buf = s.save_state()
    s.run(35, **cap)
    s.synchronize()
    assert s.stats().steps == 90
    assert_same(snapshot(bvf, s), want)
    s.load_state(buf)
    assert s.stats().steps == 55
    s.run(35, **cap)
    s.synchronize()
    assert_same(snapshot(bvf, s), want)
    # a fresh context of the same grid resumes from the snapshot as well
    t = make_solver(bvf, c, storage)
    t.load_state(buf)
    t.run(35, **cap)
    t.synchronize()
    assert_same(snapshot(bvf, t), want)
    t.close()
    s.close()


def test_snapshot_of_another_grid_is_refused(mods):
    import torch
    bvf, synth = mods
    a = small_case(synth)
    b = small_case(synth, nz=48)
    sa, sb = make_solver(bvf, a), make_solver(bvf, b)
    sa.run(3)
    buf = sa.save_state()
    with pytest.raises(bvf.BvfError) as ei:
        sb.load_state(torch.zeros(bvf.bvf_state_bytes(sb.ctx), dtype=torch.uint8, device="cuda"))
    assert ei.value.code == bvf.BVF_E_ARG
    with pytest.raises(bvf.BvfError):
        sb.load_state(buf)               # too small for b's layout
    big = torch.zeros(bvf.bvf_state_bytes(sb.ctx), dtype=torch.uint8, device="cuda")
    big[: buf.numel()] = buf
    with pytest.raises(bvf.BvfError):
        sb.load_state(big)               # a's header: another grid
    sa.close()
    sb.close()


def test_time_budget_stops_after_a_chunk_and_the_run_continues(mods):
    """A budget far below one chunk's duration: bvf_run_acoustic returns
    BVF_E_TIMEOUT after the first chunk of 32 steps; with the budget lifted, a
    second call runs the rest, and the result equals the uninterrupted run."""
    bvf, synth = mods
    c = small_case(synth)
    cap = dict(peak_from=0, dft_start=46, dft_steps=45)
    ref = make_solver(bvf, c)
    ref.run(90, **cap)
    ref.synchronize()
    want = snapshot(bvf, ref)
    ref.close()
    s = make_solver(bvf, c)
    s.set_time_budget(1e-9)
    with pytest.raises(bvf.BvfError) as ei:
        s.run(90, **cap)
    assert ei.value.code == bvf.BVF_E_TIMEOUT
    assert s.stats().steps == 32
    s.set_time_budget(0.0)
    s.run(58, **cap)
    s.synchronize()
    assert_same(snapshot(bvf, s), want)
    # a generous budget changes nothing
    s.reset()
    s.set_time_budget(3600.0)
    s.run(90, **cap)
    s.synchronize()
    assert_same(snapshot(bvf, s), want)
    s.close()


def test_time_budget_of_the_thermal_call(mods):
    """BHTE under a spent budget stops after 32 steps with T, T_max and the
    FP64 dose of those steps; continuing with the remaining on/off steps gives
    the uninterrupted result up to the one rounding at the stop.  The kernels
    advance the rise T - T_a; the stopped call hands T back in C, which rounds
    it once to FP32 near 37 C (at most half an ulp, 2^-19 C = 1.9e-6 C), and
    the explicit step is a convex combination of neighbours, so the
    difference stays within that rounding plus the rounding of the later
    steps' arithmetic on the perturbed values: below 1e-5 C in T and T_max
    and 1e-5 relative in the dose (R^(43 - T) moves by 1.39 per C)."""
    import torch
    bvf, synth = mods
    c = small_case(synth)
    s = make_solver(bvf, c)
    s.run(90, dft_start=46, dft_steps=45)
    amp = s.amp_phase()[0]
    s.synchronize()
    p_scale = 2e5 / float(amp.max())
    n_on, n_off = 50, 30
    T, Tmax, cem = s.thermal(amp, 0.05, n_on, n_off, 0.3, p_scale=p_scale)
    want = [T.cpu().numpy(), Tmax.cpu().numpy(), cem.cpu().numpy()]
    assert want[1].max() > 37.0
    s.set_time_budget(1e-9)
    shape = amp.shape
    T = torch.full(shape, 37.0, dtype=torch.float32, device="cuda")
    Tmax, cem = T.clone(), torch.zeros(shape, dtype=torch.float64, device="cuda")
    with pytest.raises(bvf.BvfError) as ei:
        s.thermal(amp, 0.05, n_on, n_off, 0.3, p_scale=p_scale, T=T, Tmax=Tmax, cem=cem)
    assert ei.value.code == bvf.BVF_E_TIMEOUT
    assert s.stats().thermal_steps == 80 + 32
    s.set_time_budget(0.0)
    s.thermal(amp, 0.05, n_on - 32, n_off, 0.3, p_scale=p_scale, T=T, Tmax=Tmax, cem=cem)
    got = [T.cpu().numpy(), Tmax.cpu().numpy(), cem.cpu().numpy()]
    assert np.abs(got[0] - want[0]).max() < 1e-5
    assert np.abs(got[1] - want[1]).max() < 1e-5
    assert np.abs(got[2] - want[2]).max() <= 1e-5 * np.abs(want[2]).max()
    s.close()
