"""The training model of the surrogate (PyTorch, offline tool) computes the
network of the FP64 oracle, and exports its weights in the oracle's blob
layout: its forward on CPU matches oracle/fno.py with the exported blob."""
import numpy as np
import pytest


def test_training_model_matches_the_oracle_on_cpu():
    torch = pytest.importorskip("torch")
    from oracle import fno as ofno
    from paper_2301_12727_gb300.fno_train import TorchFNO
    d = dict(c_in=3, width=16, modes=2, n_layers=3, hidden=8, c_out=2)
    model = TorchFNO(d, seed=3, device="cpu")
    for t in model.params():        # double precision for the comparison
        t.data = t.data.double()
    rng = np.random.default_rng(1)
    a = rng.standard_normal((1, 3, 6, 5, 8))
    with torch.no_grad():
        got = model(torch.from_numpy(a))[0].numpy()
    blob = np.concatenate([t.detach().numpy().ravel() for t in model.params()])
    assert blob.size == ofno.weight_count(**d)
    ref = ofno.forward(a[0], blob, **d)
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-10)
