"""The surrogate's BF16 path (bvf_fno_bf16_*) against the FP64 oracle
(oracle/fno.py):

* inference: output of seeded networks on ragged grids, relative L2 error
  below 3e-2 (BF16 operands round to 8 significant bits, relative 2^-9, in
  every product of a chain of about ten transforms and mixes; the observed
  errors are printed);
* training: the gradient of the loss (relative L2 of channel 0 against a
  target, plus the transmission term on channel 1's spatial mean) against
  central finite differences of the oracle's loss, on parameters drawn from
  every group (lift, spectral weights R real and imaginary, W, biases,
  projection): per group the relative L2 difference below 5e-2 of the
  finite-difference vector's norm;
* an Adam step lowers the loss of the batch."""
import json

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    assert torch.cuda.is_available()
    from paper_2301_12727_gb300 import build
    build.build()
    from paper_2301_12727_gb300 import fno, synth
    from oracle import fno as ofno
    return fno, synth, ofno


def groups(dims):
    """(name, start, length) of every parameter group in the blob."""
    ci, W, m, L, H, co = (dims[k] for k in ("c_in", "width", "modes", "n_layers", "hidden", "c_out"))
    out, pos = [], 0

    def add(name, n):
        nonlocal pos
        out.append((name, pos, n))
        pos += n
    add("Wp", W * ci)
    add("bp", W)
    for l in range(L):
        add("R%d" % l, (2 * m) * (2 * m) * m * W * W * 2)
        add("W%d" % l, W * W)
        add("b%d" % l, W)
    add("Q1", H * W)
    add("q1", H)
    add("Q2", co * H)
    add("q2", co)
    return out


def oracle_loss(ofno, a, w, dims, y, el, el_weight):
    loss = 0.0
    for b in range(a.shape[0]):
        o = ofno.forward(a[b], w, **dims)
        loss += np.linalg.norm(o[0] - y[b]) / np.linalg.norm(y[b])
        if dims["c_out"] > 1:
            loss += el_weight * (o[1].mean() - el[b]) ** 2
    return loss / a.shape[0]


@pytest.mark.parametrize("dims,grid,batch", [
    (dict(c_in=8, width=32, modes=4, n_layers=2, hidden=64, c_out=1), (16, 12, 10), 2),
    (dict(c_in=5, width=16, modes=3, n_layers=3, hidden=32, c_out=2), (12, 14, 9), 1),
    (dict(c_in=8, width=32, modes=12, n_layers=4, hidden=128, c_out=2), (36, 26, 28), 1),
])
def test_bf16_inference_matches_oracle(mods, dims, grid, batch):
    import torch
    fno, synth, ofno = mods
    nx, ny, nz = grid
    w = synth.fno_weights(dims, 11)
    a = np.stack([synth.fno_inputs(dims["c_in"], nx, ny, nz, 3 + b) for b in range(batch)])
    net = fno.Bf16Net(dims, w, grid, max_batch=batch)
    out = net.forward(torch.from_numpy(a.astype(np.float32)).cuda()).cpu().numpy()
    net.synchronize()
    net.close()
    errs = []
    for b in range(batch):
        ref = ofno.forward(a[b].astype(np.float64), w.astype(np.float64), **dims)
        errs.append(float(np.linalg.norm(out[b] - ref) / np.linalg.norm(ref)))
    print("bf16 inference vs FP64 oracle, rel L2:", errs)
    assert max(errs) < 3e-2


def test_bf16_gradient_matches_oracle_finite_differences(mods):
    import torch
    fno, synth, ofno = mods
    dims = dict(c_in=4, width=16, modes=2, n_layers=2, hidden=16, c_out=2)
    nx, ny, nz = 8, 6, 6
    batch, el_weight = 2, 3.0
    w = synth.fno_weights(dims, 21).astype(np.float64)
    rng = np.random.default_rng(5)
    a = np.stack([synth.fno_inputs(dims["c_in"], nx, ny, nz, 30 + b) for b in range(batch)])
    y = rng.standard_normal((batch, nz, ny, nx))
    el = rng.uniform(0.2, 0.8, batch)
    net = fno.Bf16Net(dims, w.astype(np.float32), (nx, ny, nz), max_batch=batch)
    loss, g = net.gradient(torch.from_numpy(a.astype(np.float32)).cuda(),
                           torch.from_numpy(y.astype(np.float32)).cuda(),
                           torch.from_numpy(el.astype(np.float32)).cuda(), el_weight)
    net.synchronize()
    g = g.cpu().numpy().astype(np.float64)
    net.close()
    L0 = oracle_loss(ofno, a, w, dims, y, el, el_weight)
    assert abs(loss - L0) < 3e-2 * abs(L0)
    eps = 1e-4
    report = {}
    for name, start, n in groups(dims):
        pick = rng.choice(n, size=min(n, 10), replace=False) + start
        fd = []
        for i in pick:
            wp, wm = w.copy(), w.copy()
            wp[i] += eps
            wm[i] -= eps
            fd.append((oracle_loss(ofno, a, wp, dims, y, el, el_weight)
                       - oracle_loss(ofno, a, wm, dims, y, el, el_weight)) / (2 * eps))
        fd = np.array(fd)
        err = float(np.linalg.norm(g[pick] - fd) / max(np.linalg.norm(fd), 1e-12))
        report[name] = err
    print("bf16 gradient vs oracle finite differences:", json.dumps(report))
    assert max(report.values()) < 5e-2, report


def test_bf16_adam_step_lowers_the_loss(mods):
    import torch
    fno, synth, ofno = mods
    dims = dict(c_in=8, width=16, modes=4, n_layers=2, hidden=32, c_out=1)
    nx, ny, nz = 16, 16, 12
    w = synth.fno_weights(dims, 2)
    rng = np.random.default_rng(1)
    a = torch.from_numpy(np.stack([synth.fno_inputs(8, nx, ny, nz, 40 + b)
                                   for b in range(2)]).astype(np.float32)).cuda()
    y = torch.from_numpy(rng.standard_normal((2, nz, ny, nx)).astype(np.float32)).cuda()
    net = fno.Bf16Net(dims, w, (nx, ny, nz), max_batch=2)
    l0 = net.adam(a, y, 1e-3)
    losses = [net.adam(a, y, 1e-3) for _ in range(5)]
    net.synchronize()
    net.close()
    assert losses[-1] < l0
