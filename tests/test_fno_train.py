"""Host logic of the surrogate's training tool (the training itself runs in
the library's BF16 kernels, checked in tests/test_fno_bf16_gpu.py): the
initial weights scale exactly the spectral blocks of the blob layout, and the
learning-rate schedule warms up, peaks at lr_max and decays."""
import numpy as np


def test_initial_weights_scale_only_the_spectral_blocks():
    from oracle import fno as ofno
    from paper_2301_12727_gb300 import synth
    from paper_2301_12727_gb300.fno_train import initial_weights
    d = dict(c_in=3, width=16, modes=2, n_layers=3, hidden=8, c_out=2)
    w0 = synth.fno_weights(d, 4).astype(np.float64)
    w1 = initial_weights(d, 4).astype(np.float64)
    assert w1.size == ofno.weight_count(**d)
    p0 = ofno.unpack(w0, **d)
    p1 = ofno.unpack(w1, **d)
    for key in ("Wp", "bp", "Q1", "q1", "Q2", "q2"):
        np.testing.assert_array_equal(p0[key], p1[key])
    for l0, l1 in zip(p0["layers"], p1["layers"]):
        np.testing.assert_allclose(l1["R"], l0["R"] / d["width"], rtol=1e-6)
        np.testing.assert_array_equal(l0["W"], l1["W"])
        np.testing.assert_array_equal(l0["b"], l1["b"])


def test_one_cycle_schedule():
    from paper_2301_12727_gb300.fno_train import one_cycle
    total, lr = 1000, 2e-3
    lrs = np.array([one_cycle(s, total, lr) for s in range(total)])
    assert lrs.max() <= lr * (1 + 1e-12)
    peak = int(np.argmax(lrs))
    assert abs(peak - 300) <= 1
    assert np.all(np.diff(lrs[:peak]) > 0) and np.all(np.diff(lrs[peak + 1:]) <= 0)
    assert lrs[0] < 0.1 * lr and lrs[-1] < 0.05 * lr
