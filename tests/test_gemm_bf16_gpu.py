"""The BF16 tensor-core product (bvf_gemm_bf16) against a host product of the
same BF16-rounded operands in FP64: row- and column-major views, ragged M, N
and K (several 128-row tiles, several K chunks and a partial one), batches,
split K, bias per column and per row, beta, and GELU with the pre-activation
kept.  The operands are exact in BF16 once rounded, so the only differences
are FP32 accumulation order: bounded by 1e-5 of sum |a||b| per element."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    assert torch.cuda.is_available()
    from paper_2301_12727_gb300 import build
    build.build()
    from paper_2301_12727_gb300 import fno
    return fno


def bf16(x):
    """Round FP32 values to BF16 (nearest, ties to even) and back, in numpy."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def gelu(x):
    from scipy.special import erf
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


@pytest.mark.parametrize("M,N,K,a_cm,b_nm,c_cm,batch", [
    (200, 24, 64, False, True, False, 1),      # x-stage shape: rows x nx -> 2m
    (300, 48, 150, False, True, True, 2),      # ragged K over three chunks
    (1000, 32, 32, True, False, True, 3),      # channel mix: voxels x channels
    (130, 130, 70, True, True, False, 1),      # N beyond 128: the 256-wide tile
    (129, 300, 20, False, False, True, 1),     # N over two 256-wide tiles
])
def test_gemm_matches_host_product(mods, M, N, K, a_cm, b_nm, c_cm, batch):
    import torch
    fno = mods
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((batch, M, K)).astype(np.float32)
    B = rng.standard_normal((batch, K, N)).astype(np.float32)
    C0 = rng.standard_normal((batch, M, N)).astype(np.float32)
    bias = rng.standard_normal(N).astype(np.float32)
    # device layouts
    Ad = torch.from_numpy(np.ascontiguousarray(A.transpose(0, 2, 1) if a_cm else A)).cuda()
    a_str = (1, M, M * K) if a_cm else (K, 1, M * K)
    Bd = torch.from_numpy(np.ascontiguousarray(B if b_nm else B.transpose(0, 2, 1))).cuda()
    b_str = (N, 1, K * N) if b_nm else (1, K, K * N)
    Cn = C0.transpose(0, 2, 1) if c_cm else C0
    c_str = (1, M, M * N) if c_cm else (N, 1, M * N)
    ref = np.einsum("bmk,bkn->bmn", bf16(A).astype(np.float64), bf16(B).astype(np.float64))
    bound = np.einsum("bmk,bkn->bmn", np.abs(bf16(A)).astype(np.float64),
                      np.abs(bf16(B)).astype(np.float64))

    def run(alpha, beta, bias_mode, act, pre, ksplit=1):
        Cd = torch.from_numpy(np.ascontiguousarray(Cn)).cuda()
        Pd = torch.zeros_like(Cd) if pre else None
        bd = torch.from_numpy(bias if bias_mode == 1 else
                              rng.standard_normal(M).astype(np.float32)).cuda()
        flag = fno.bvf_gemm_bf16(Ad, a_str, Bd, b_str, Cd, c_str, M, N, K, batch, ksplit, alpha,
                                 beta, bd if bias_mode else None, bias_mode, act, Pd)
        torch.cuda.synchronize()
        assert int(flag.item()) == 0
        back = lambda t: (t.cpu().numpy().transpose(0, 2, 1) if c_cm else t.cpu().numpy())
        return back(Cd), (back(Pd) if pre else None), bd.cpu().numpy()

    got, _, _ = run(1.0, 0.0, 0, 0, False)
    assert np.all(np.abs(got - ref) <= 1e-5 * bound + 1e-30)
    got, _, bd = run(0.5, -2.0, 1, 0, False)
    want = 0.5 * ref - 2.0 * C0 + bd[None, None, :]
    assert np.all(np.abs(got - want) <= 1e-5 * (0.5 * bound + 2 * np.abs(C0) + np.abs(bd)) + 1e-6)
    got, pre, bd = run(1.0, 0.0, 2, 1, True)
    s = ref + bd[None, :, None]
    assert np.all(np.abs(pre - s) <= 1e-5 * (bound + np.abs(bd)[None, :, None]) + 1e-6)
    assert np.allclose(got, gelu(pre.astype(np.float64)), rtol=1e-5, atol=1e-6)
    got, _, _ = run(1.0, 1.0, 0, 0, False, ksplit=3)
    assert np.all(np.abs(got - (ref + C0)) <= 1e-5 * (bound + np.abs(C0)) + 1e-6)


def test_gemm_rejects_bad_arguments(mods):
    import torch
    fno = mods
    x = torch.zeros(64, device="cuda")
    with pytest.raises(Exception):
        fno.bvf_gemm_bf16(x, (1, 1, 0), x, (1, 1, 0), x, (1, 1, 0), 0, 4, 4)
    with pytest.raises(Exception):       # split K with an activation
        fno.bvf_gemm_bf16(x, (1, 1, 0), x, (1, 1, 0), x, (1, 1, 0), 4, 4, 4, ksplit=2, beta=1.0,
                          act=1)
