"""Batched sweeps (persistent kernels over a work list spanning several
domains, optionally replayed from a CUDA graph) against the same contexts run
one by one: identical results, bit for bit."""
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


def make(bvf, synth, spec, n_steps, storage="f32"):
    c = synth.sweep_case(spec, n_steps=n_steps, dft_cycles=2)
    s = bvf.Solver(c.nx, c.ny, c.nz, c.dx, c.dt, c.f0, n_sls=2, n_pml=c.n_pml, storage=storage)
    s.set_materials(c.index, c.materials)
    s.set_source(bvf.rs_plane(c.bowl, c.nx, c.ny, c.dx, c.k_src * c.dx, c.f0), c.k_src, c.c0,
                 c.envelope)
    M = c.steps_per_period
    cap = (5, n_steps - M + 1, M)            # peak from step 5, DFT over the last period
    return c, s, cap


def outputs(s):
    amp, ph = s.amp_phase()
    return ([s.field(f).cpu().numpy() for f in range(21)] +
            [s.peak().cpu().numpy(), amp.cpu().numpy(), ph.cpu().numpy()])


@pytest.mark.parametrize("kchunk,graph_steps,storage", [(0, 0, "f32"), (5, 16, "f32"),
                                                         (13, 7, "f32"), (6, 9, "f16")])
def test_gpu_batch_matches_single_runs_bitwise(mods, kchunk, graph_steps, storage):
    """Four domains of different sizes (ragged y and z, two x-tiles or one),
    frequencies, tilts and step counts: every state array, the peak map and
    the FP64 amplitude and phase equal those of single-context runs (FP32 and
    FP16 storage)."""
    bvf, synth = mods
    specs = synth.sweep_specs(n=4, seed=7, n_min=40, n_max=72)
    n_steps = [60, 90, 75, 40]
    ref = []
    for spec, n in zip(specs, n_steps):
        c, s, cap = make(bvf, synth, spec, n, storage)
        s.run(n, peak_from=cap[0], dft_start=cap[1], dft_steps=cap[2])
        s.synchronize()
        ref.append(outputs(s))
        s.close()
    made = [make(bvf, synth, spec, n, storage) for spec, n in zip(specs, n_steps)]
    solvers = [m[1] for m in made]
    b = bvf.Batch(solvers)
    b.run(n_steps, caps=[m[2] for m in made], kchunk=kchunk, graph_steps=graph_steps)
    for s in solvers:
        s.synchronize()
    assert b.launches() >= 3 * max(n_steps)
    for d, s in enumerate(solvers):
        assert s.stats().steps == n_steps[d]
        got = outputs(s)
        assert np.abs(got[21]).max() > 0
        for a, r in zip(got, ref[d]):
            assert np.array_equal(a, r), d
    b.close()
    for s in solvers:
        s.close()


def test_gpu_batch_streams_match_single_runs_bitwise(mods):
    """The stream-level alternative (per-context launches on 2 side streams)
    gives the single-run results too."""
    bvf, synth = mods
    specs = synth.sweep_specs(n=3, seed=9, n_min=40, n_max=64)
    n_steps = [50, 30, 40]
    ref = []
    for spec, n in zip(specs, n_steps):
        c, s, cap = make(bvf, synth, spec, n)
        s.run(n, peak_from=cap[0], dft_start=cap[1], dft_steps=cap[2])
        s.synchronize()
        ref.append(outputs(s))
        s.close()
    made = [make(bvf, synth, spec, n) for spec, n in zip(specs, n_steps)]
    solvers = [m[1] for m in made]
    b = bvf.Batch(solvers)
    b.run_streams(n_steps, caps=[m[2] for m in made], n_streams=2)
    for d, s in enumerate(solvers):
        s.synchronize()
        for a, r in zip(outputs(s), ref[d]):
            assert np.array_equal(a, r), d
    b.close()
    for s in solvers:
        s.close()


def test_gpu_batch_tune_picks_a_candidate_and_resets(mods):
    bvf, synth = mods
    specs = synth.sweep_specs(n=3, seed=11, n_min=40, n_max=64)
    made = [make(bvf, synth, spec, 30) for spec in specs]
    solvers = [m[1] for m in made]
    b = bvf.Batch(solvers)
    best, ms = b.tune(trial_steps=8, candidates=(4, 8))
    assert best in (4, 8) and ms > 0
    for s in solvers:
        s.synchronize()
        assert s.stats().steps == 0
        assert float(s.field(3).abs().max()) == 0.0
    b.close()
    for s in solvers:
        s.close()


def test_gpu_batch_rejects_grids_off_the_tma_path(mods):
    bvf, synth = mods
    c = synth.skull_case(50, 40, 36, n_steps=10, aperture=16e-3, roc=16e-3, n_pml=5)
    s = bvf.Solver(c.nx, c.ny, c.nz, c.dx, c.dt, c.f0, n_sls=2, n_pml=c.n_pml)
    s.set_materials(c.index, c.materials)
    with pytest.raises(bvf.BvfError):
        bvf.Batch([s])
    s.close()


def test_gpu_batch_graph_matches_single_runs_bitwise(mods):
    """The sweep recorded as one CUDA graph of per-domain launches on three
    branches: the first call records and replays, a second call after
    bvf_reset replays the same recording; both give the single-run results
    bit for bit (state, peak, FP64 amplitude and phase), and a call from
    other step counts records anew."""
    bvf, synth = mods
    specs = synth.sweep_specs(n=4, seed=11, n_min=40, n_max=72)
    n_steps = [45, 70, 30, 55]
    ref = []
    for spec, n in zip(specs, n_steps):
        c, s, cap = make(bvf, synth, spec, n)
        s.run(n, peak_from=cap[0], dft_start=cap[1], dft_steps=cap[2])
        s.synchronize()
        ref.append(outputs(s))
        s.close()
    made = [make(bvf, synth, spec, n) for spec, n in zip(specs, n_steps)]
    solvers = [m[1] for m in made]
    caps = [m[2] for m in made]
    b = bvf.Batch(solvers)
    for rep in range(2):
        for s in solvers:
            s.reset()
        b.run_graph(n_steps, caps=caps, n_branches=3)
        for d, s in enumerate(solvers):
            s.synchronize()
            assert s.stats().steps == n_steps[d]
            for a, r in zip(outputs(s), ref[d]):
                assert np.array_equal(a, r), (rep, d)
    # continuing from the reached steps records a new graph (no capture window)
    b.run_graph(5, n_branches=2)
    for d, s in enumerate(solvers):
        s.synchronize()
        assert s.stats().steps == n_steps[d] + 5
    b.close()
    for s in solvers:
        s.close()


def test_gpu_batch_tune_domains_picks_a_candidate_and_keeps_results(mods):
    """The per-domain tile tuner returns one of the candidate (rows, z-chunk)
    pairs for every domain and keeps it in the context, leaves the contexts
    reset, and runs after it equal single runs with the default tile."""
    bvf, synth = mods
    specs = synth.sweep_specs(n=2, seed=3, n_min=48, n_max=64)
    made = [make(bvf, synth, spec, 40) for spec in specs]
    solvers = [m[1] for m in made]
    b = bvf.Batch(solvers)
    cand = ((8, 16, 6), (4, 8, 9), (16, 16, 16), (8, 4, 5))
    best = b.tune_domains(trial_steps=4, candidates=cand)
    for (sr, vr, k), s in zip(best, solvers):
        assert (sr, vr, k) in [(a, v, min(c, s.shape[0])) for a, v, c in cand]
        assert s.tile() == (sr, vr, k)
    for s in solvers:
        assert s.stats().steps == 0
    b.run_streams(40, caps=[m[2] for m in made], n_streams=2)
    for s, spec in zip(solvers, specs):
        s.synchronize()
        c, r, cap = make(bvf, synth, spec, 40)
        r.run(40, peak_from=cap[0], dft_start=cap[1], dft_steps=cap[2])
        r.synchronize()
        for a, x in zip(outputs(s), outputs(r)):
            assert np.array_equal(a, x)
        r.close()
    b.close()
    for s in solvers:
        s.close()


def test_gpu_batch_tune_graph_picks_a_candidate_and_keeps_results(mods):
    """The graph-mode tuner gives every context the same candidate tile, leaves
    them reset, and the graph run after it equals single runs with the
    default tiles bit for bit."""
    bvf, synth = mods
    specs = synth.sweep_specs(n=3, seed=5, n_min=48, n_max=64)
    made = [make(bvf, synth, spec, 30) for spec in specs]
    solvers = [m[1] for m in made]
    b = bvf.Batch(solvers)
    cand = ((8, 16, 6), (8, 8, 12), (16, 16, 0))
    tile, ms = b.tune_graph(trial_steps=4, candidates=cand, n_branches=2)
    assert tile in cand and ms > 0
    for s in solvers:
        assert s.stats().steps == 0
        assert s.tile()[:2] == tile[:2]
    b.run_graph(30, caps=[m[2] for m in made], n_branches=2)
    for s, spec in zip(solvers, specs):
        s.synchronize()
        c, r, cap = make(bvf, synth, spec, 30)
        r.run(30, peak_from=cap[0], dft_start=cap[1], dft_steps=cap[2])
        r.synchronize()
        for a, x in zip(outputs(s), outputs(r)):
            assert np.array_equal(a, x)
        r.close()
    b.close()
    for s in solvers:
        s.close()
