"""Surrogate inference on the GPU against the FP64 oracle (oracle/fno.py):
element-by-element parity on ragged grids across the width templates, the
feature volume of a placement, and, at the benchmark's full size, properties
that hold at any size (circular-shift equivariance; the constant-field
reduction to a plain MLP)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# FP32 sums (DFT over up to nx, ny, nz terms; channel sums over width) against
# FP64: the bound is a multiple of the FP32 unit roundoff times the largest
# output and the sum lengths, rounded up to 2e-5 relative to max |ref|.
TOL = 2e-5


@pytest.fixture(scope="module")
def mods():
    import torch
    assert torch.cuda.is_available()
    from paper_2301_12727_gb300 import build
    build.build()
    from paper_2301_12727_gb300 import fno, synth
    return torch, fno, synth


def _run(mods, dims, grid, seed):
    torch, fno, synth = mods
    nx, ny, nz = grid
    w = synth.fno_weights(dims, seed)
    a = synth.fno_inputs(dims["c_in"], nx, ny, nz, seed + 1)
    net = fno.Surrogate(dims, w)
    out = net(torch.from_numpy(a).cuda())
    net.synchronize()
    got = out.cpu().numpy()
    net.close()
    return w, a, got


@pytest.mark.parametrize("dims,grid", [
    (dict(c_in=8, width=16, modes=4, n_layers=3, hidden=32, c_out=2), (20, 11, 9)),
    (dict(c_in=8, width=32, modes=12, n_layers=4, hidden=128, c_out=1), (40, 30, 27)),
    (dict(c_in=3, width=16, modes=3, n_layers=2, hidden=5, c_out=3), (7, 6, 13)),
    (dict(c_in=5, width=64, modes=6, n_layers=2, hidden=96, c_out=1), (37, 13, 12)),
    (dict(c_in=16, width=48, modes=1, n_layers=1, hidden=256, c_out=8), (2, 2, 2)),
    (dict(c_in=8, width=32, modes=16, n_layers=2, hidden=64, c_out=1), (33, 32, 40)),
    # rows too long for the fused row pass (unfused kernels)
    (dict(c_in=4, width=64, modes=16, n_layers=2, hidden=32, c_out=1), (600, 32, 33)),
])
def test_gpu_surrogate_matches_oracle(mods, dims, grid):
    from oracle import fno as ofno
    w, a, got = _run(mods, dims, grid, seed=sum(grid) + dims["width"])
    ref = ofno.forward(a.astype(np.float64), w.astype(np.float64), **dims)
    assert got.shape == ref.shape
    err = np.abs(got - ref).max()
    assert err <= TOL * np.abs(ref).max(), (err, np.abs(ref).max())


def test_gpu_features_match_oracle(mods):
    torch, fno, synth = mods
    from oracle import fno as ofno
    rng = np.random.default_rng(4)
    nz, ny, nx = 9, 14, 23
    table = [(1000.0, 1500.0, 0, 0.0, 0, 0.6, 4180, 0, 0),
             (1900.0, 2800.0, 1400, 210.0, 300, 0.32, 1300, 0, 0),
             (1050.0, 1560.0, 0, 35.0, 0, 0.5, 3600, 0.008, 0)]
    idx = rng.integers(0, 3, size=(nz, ny, nx)).astype(np.uint8)
    src = (rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))) * 1e4
    out = torch.empty((8, nz, ny, nx), dtype=torch.float32, device="cuda")
    fno.bvf_fno_features(torch.from_numpy(idx).cuda(), table, table[0], 5e5, 3,
                         torch.from_numpy(src.astype(np.complex64)).cuda(), 2.5e4, out)
    torch.cuda.synchronize()
    ref = ofno.features(idx, np.array(table), table[0], 5e5, 3, src.astype(np.complex64), 2.5e4)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=2e-7, atol=1e-7)


def test_gpu_surrogate_rejects_small_grids(mods):
    torch, fno, synth = mods
    from paper_2301_12727_gb300 import bvf
    dims = dict(c_in=2, width=16, modes=4, n_layers=1, hidden=8, c_out=1)
    net = fno.Surrogate(dims, synth.fno_weights(dims, 1))
    for grid in ((7, 8, 8), (8, 7, 8), (8, 8, 7)):          # m > nx/2 or 2m > ny, nz
        a = torch.zeros((2, grid[2], grid[1], grid[0]), device="cuda")
        with pytest.raises(bvf.BvfError):
            net(a)
    a = torch.zeros((2, 8, 8, 8), device="cuda")
    out = net(a)
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
    net.close()


FULL = dict(c_in=8, width=32, modes=12, n_layers=4, hidden=128, c_out=1)
FULL_GRID = (240, 240, 200)     # the benchmark's skull domain (nx, ny, nz)


def test_gpu_full_size_shift_equivariance(mods):
    """Every stage is pointwise or a circular convolution, so a circular shift
    of the input shifts the output; at 240 x 240 x 200 the two runs agree to
    FP32 rounding."""
    torch, fno, synth = mods
    nx, ny, nz = FULL_GRID
    net = fno.Surrogate(FULL, synth.fno_weights(FULL, 77))
    a = torch.from_numpy(synth.fno_inputs(8, nx, ny, nz, 78)).cuda()
    u = net(a).clone()
    sh = (5, -17, 31)
    us = net(torch.roll(a, sh, dims=(1, 2, 3)).contiguous())
    net.synchronize()
    d = (us - torch.roll(u, sh, dims=(1, 2, 3))).abs().max().item()
    assert d <= 5 * TOL * u.abs().max().item()
    net.close()


def test_gpu_full_size_constant_field_is_the_mlp(mods):
    """On a constant field only the DC mode is non-zero: the network is then
    the MLP with W_l + Re R_l(0,0,0)^T per layer, evaluated here in FP64."""
    torch, fno, synth = mods
    from oracle import fno as ofno
    nx, ny, nz = FULL_GRID
    w = synth.fno_weights(FULL, 91)
    a0 = np.random.default_rng(92).standard_normal(8)
    net = fno.Surrogate(FULL, w)
    a = torch.from_numpy(np.broadcast_to(a0[:, None, None, None].astype(np.float32),
                                         (8, nz, ny, nx)).copy()).cuda()
    u = net(a)
    net.synchronize()
    p = ofno.unpack(w.astype(np.float64), **FULL)
    v = p["Wp"] @ a0.astype(np.float32).astype(np.float64) + p["bp"]
    for l, lay in enumerate(p["layers"]):
        s = (lay["W"] + np.real(lay["R"][0, 0, 0]).T) @ v + lay["b"]
        v = ofno.gelu(s) if l < FULL["n_layers"] - 1 else s
    ref = p["Q2"] @ ofno.gelu(p["Q1"] @ v + p["q1"]) + p["q2"]
    got = u.cpu().numpy()
    assert np.abs(got - ref[:, None, None, None]).max() <= 10 * TOL * max(1.0, abs(ref).max())
    net.close()


def test_gpu_one_context_across_grid_changes_is_bit_identical(mods):
    """A context reused on another grid regrows its workspace and rebuilds its
    twiddle tables: every call equals a fresh context's, bit for bit."""
    torch, fno, synth = mods
    dims = dict(c_in=8, width=32, modes=6, n_layers=2, hidden=32, c_out=1)
    w = synth.fno_weights(dims, 13)
    grids = [(24, 20, 16), (40, 36, 30), (24, 20, 16)]
    ins = [torch.from_numpy(synth.fno_inputs(8, *g, seed=20 + i)).cuda() for i, g in enumerate(grids)]
    shared = fno.Surrogate(dims, w)
    got = [shared(a).clone() for a in ins]
    shared.synchronize()
    shared.close()
    for a, u in zip(ins, got):
        fresh = fno.Surrogate(dims, w)
        ref = fresh(a)
        fresh.synchronize()
        fresh.close()
        assert torch.equal(u, ref)


def test_gpu_stage_times_cover_the_inference(mods):
    torch, fno, synth = mods
    dims = dict(c_in=8, width=32, modes=12, n_layers=4, hidden=128, c_out=1)
    net = fno.Surrogate(dims, synth.fno_weights(dims, 3))
    a = torch.from_numpy(synth.fno_inputs(8, 64, 48, 40, 4)).cuda()
    net(a)
    net.timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    net(a)
    e1.record()
    net.synchronize()
    st = net.stage_times()
    total = e0.elapsed_time(e1)
    assert set(st) == set(fno.STAGES)
    assert all(v >= 0.0 for v in st.values())
    assert 0.5 * total <= sum(st.values()) <= 1.05 * total
    net.timing(False)
    net.close()


def test_gpu_prediction_falls_back_to_the_fdtd(mods):
    """predict_amplitude keeps an in-range prediction and calls the FDTD for
    one whose maximum leaves the trained range."""
    torch, fno, synth = mods
    from paper_2301_12727_gb300 import bvf
    c = synth.slab_case(n=32, n_steps=10, n_pml=4, k_src=6)
    dims = dict(c_in=8, width=16, modes=4, n_layers=2, hidden=16, c_out=1)
    net = fno.Surrogate(dims, synth.fno_weights(dims, 31))
    idx = torch.from_numpy(c.index).cuda()
    src = torch.zeros((c.ny, c.nx, 2), dtype=torch.float32, device="cuda")
    src[..., 0] = 1e4
    water = synth.water_row(c.f0)
    calls = []

    def fdtd():
        calls.append(1)
        return torch.full(c.index.shape, 7.0, dtype=torch.float32, device="cuda")

    amp, how = fno.predict_amplitude(net, idx, c.materials, water, c.f0, c.k_src, src, 1e4,
                                     (-1e30, 1e30), fdtd)
    assert how == "surrogate" and not calls and torch.isfinite(amp).all()
    amp2, how2 = fno.predict_amplitude(net, idx, c.materials, water, c.f0, c.k_src, src, 1e4,
                                       (1e29, 1e30), fdtd)
    assert how2 == "fdtd" and calls == [1] and float(amp2.max()) == 7.0
    with pytest.raises(RuntimeError):
        fno.predict_amplitude(net, idx, c.materials, water, c.f0, c.k_src, src, 1e4,
                              (1e29, 1e30), None)
    net.close()
