"""bvf_transmission_noalloc: the energy-loss reduction for callers that cannot
allocate device memory (their pool already holds the GPU's memory, or an
allocation would stall a latency-bound loop).  Its temporaries live in a fixed
array inside the library; this checks, through the C ABI, that it returns what
bvf_transmission returns, on two calls in a row with different inputs (so a
value left over in the shared array from the first call would show)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_transmission_matches_allocating_one_twice():
    import torch
    assert torch.cuda.is_available()
    from paper_2301_12727_gb300 import build
    build.build()
    from paper_2301_12727_gb300 import bvf
    rng = np.random.default_rng(17)
    water = [[1000.0, 1500.0, 0.0, 0.0, 0.0, 0.6, 4178.0, 0.0, 1.0]]
    tissue = [[1000.0, 1500.0, 0.0, 0.0, 0.0, 0.6, 4178.0, 0.0, 1.0],
              [1041.0, 1562.0, 0.0, 3.45, 0.0, 0.51, 3630.0, 0.008, 1.0],
              [1850.0, 2800.0, 1500.0, 85.0, 170.0, 0.32, 1313.0, 0.008, 0.16]]
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    results = []
    for call, (shape, peak) in enumerate((((30, 26, 22), (17, 12, 10)),
                                          ((24, 40, 36), (5, 30, 20)))):
        nz, ny, nx = shape
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        amp_w = np.exp(-((z - peak[0]) ** 2 / 20.0 + (y - peak[1]) ** 2 / 9.0
                         + (x - peak[2]) ** 2 / 9.0))
        amp_a = amp_w * (0.3 + 0.4 * rng.random(amp_w.shape))
        idx_a = rng.integers(0, 3, amp_w.shape).astype(np.uint8)
        idx_w = np.zeros_like(idx_a)
        args = (cu(idx_a), tissue, cu(amp_a), cu(idx_w), water, cu(amp_w))
        ref = bvf.bvf_transmission(*args)
        got = bvf.bvf_transmission_noalloc(*args)
        assert got[2] == ref[2] == peak[0]
        np.testing.assert_allclose(got[0], ref[0], rtol=1e-12)
        np.testing.assert_allclose(got[1], ref[1], rtol=1e-12)
        np.testing.assert_allclose(got[3], ref[3], rtol=1e-12)
        results.append(got)
    assert results[0][0] != results[1][0]
