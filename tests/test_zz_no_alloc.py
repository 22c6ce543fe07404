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


def test_noalloc_limits_and_cleared_rows():
    """The edges of the fixed array: a table of 257 rows is refused
    (BVF_E_ARG) while 256 are accepted; an all-zero water field is refused like
    bvf_transmission refuses it; and rows beyond a call's table read as zero
    even after a longer table filled them in the previous call (a 3-row call,
    then a 1-row call whose index volume holds the value 2 gives what
    bvf_transmission gives)."""
    import ctypes
    import torch
    assert torch.cuda.is_available()
    from paper_2301_12727_gb300 import build
    build.build()
    from paper_2301_12727_gb300 import bvf
    rng = np.random.default_rng(5)
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    nz, ny, nx = 12, 10, 9
    amp_w = rng.random((nz, ny, nx)) + 0.1
    amp_a = amp_w * rng.random((nz, ny, nx))
    idx0 = np.zeros((nz, ny, nx), np.uint8)
    row = [1000.0, 1500.0, 0.0, 0.0, 0.0, 0.6, 4178.0, 0.0, 1.0]
    # 256 rows accepted, 257 refused
    for n_rows, ok in ((256, True), (257, False)):
        table = [row] * n_rows
        args = (cu(idx0), table, cu(amp_a), cu(idx0), [row], cu(amp_w))
        if ok:
            assert bvf.bvf_transmission_noalloc(*args)[2] >= 0
        else:
            arr = bvf.material_array(table)
            el = ctypes.c_double()
            rc = bvf.lib().bvf_transmission_noalloc(
                nx, ny, nz, bvf._ptr(args[0]), arr, n_rows, bvf._ptr(args[2]), bvf._ptr(args[3]),
                bvf.material_array([row]), 1, bvf._ptr(args[5]), ctypes.byref(el), None, None,
                None, None)
            assert rc == bvf.BVF_E_ARG
    # zero water intensity: refused by both
    zero = np.zeros_like(amp_w)
    for fn in (bvf.bvf_transmission, bvf.bvf_transmission_noalloc):
        with pytest.raises(bvf.BvfError) as ei:
            fn(cu(idx0), [row], cu(amp_a), cu(idx0), [row], cu(zero))
        assert ei.value.code == bvf.BVF_E_ARG
    # a 3-row call leaves rows 1 and 2 of the array filled ...
    tissue = [row, [1041.0, 1562.0, 0.0, 3.45, 0.0, 0.51, 3630.0, 0.008, 1.0],
              [1850.0, 2800.0, 1500.0, 85.0, 170.0, 0.32, 1313.0, 0.008, 0.16]]
    idx3 = rng.integers(0, 3, (nz, ny, nx)).astype(np.uint8)
    bvf.bvf_transmission_noalloc(cu(idx3), tissue, cu(amp_a), cu(idx3), tissue, cu(amp_w))
    # ... and a 1-row call whose index holds 2 must read them as zero
    args = (cu(idx3), [row], cu(amp_a), cu(idx3), [row], cu(amp_w))
    ref = bvf.bvf_transmission(*args)
    got = bvf.bvf_transmission_noalloc(*args)
    assert got[2] == ref[2]
    np.testing.assert_allclose(got[0], ref[0], rtol=1e-12)
    np.testing.assert_allclose(got[3], ref[3], rtol=1e-12)
