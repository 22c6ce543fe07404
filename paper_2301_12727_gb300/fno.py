"""Python binding of the surrogate's C ABI (include/bvf_fno.h), ctypes over
libbvf.so.  Argument marshalling only: the inference runs in the CUDA library.

    dims = FnoDims(c_in=8, width=32, modes=12, n_layers=4, hidden=128, c_out=1)
    net = Surrogate(dims, weights)            # weights: flat float32 blob
    out = net(features)                       # [c_in, nz, ny, nx] CUDA float32
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import bvf

EXPORTS = ("bvf_fno_weight_count", "bvf_fno_create", "bvf_fno_destroy", "bvf_fno_forward",
           "bvf_fno_features", "bvf_fno_timing", "bvf_fno_stage_times", "bvf_fno_synchronize",
           "bvf_gemm_bf16", "bvf_fno_bf16_create", "bvf_fno_bf16_destroy", "bvf_fno_bf16_forward",
           "bvf_fno_bf16_gradient", "bvf_fno_bf16_adam", "bvf_fno_bf16_weights",
           "bvf_fno_bf16_synchronize", "bvf_fno_mean")
N_FEATURES = 8
N_STAGES = 9
STAGES = ("lift", "dft_x", "dft_y", "dft_z", "mix", "idft_z", "idft_y", "out_x_pointwise",
          "project")


class FnoDims(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in
                ("c_in", "width", "modes", "n_layers", "hidden", "c_out")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class Gemm(ctypes.Structure):
    """bvf_gemm (include/bvf_fno.h): strided views of FP32 device arrays."""
    _fields_ = [("A", ctypes.c_void_p), ("sam", ctypes.c_longlong), ("sak", ctypes.c_longlong),
                ("sab", ctypes.c_longlong), ("B", ctypes.c_void_p), ("sbk", ctypes.c_longlong),
                ("sbn", ctypes.c_longlong), ("sbb", ctypes.c_longlong), ("C", ctypes.c_void_p),
                ("scm", ctypes.c_longlong), ("scn", ctypes.c_longlong), ("scb", ctypes.c_longlong),
                ("C_pre", ctypes.c_void_p), ("bias", ctypes.c_void_p), ("bias_mode", ctypes.c_int),
                ("M", ctypes.c_int), ("N", ctypes.c_int), ("K", ctypes.c_int),
                ("batch", ctypes.c_int), ("ksplit", ctypes.c_int), ("alpha", ctypes.c_float),
                ("beta", ctypes.c_float), ("act", ctypes.c_int)]


_declared = False


def lib():
    global _declared
    L = bvf.lib()
    if not _declared:
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.bvf_fno_weight_count.restype = ctypes.c_size_t
        L.bvf_fno_weight_count.argtypes = [ctypes.POINTER(FnoDims)]
        L.bvf_fno_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(FnoDims), vp,
                                     ctypes.c_size_t]
        L.bvf_fno_destroy.argtypes = [vp]
        L.bvf_fno_forward.argtypes = [vp, i, i, i, vp, vp, vp]
        L.bvf_fno_features.argtypes = [vp, ctypes.POINTER(bvf.Material), i,
                                       ctypes.POINTER(bvf.Material), i, i, i, d, i, vp, d, vp, vp]
        L.bvf_fno_timing.argtypes = [vp, i]
        L.bvf_fno_stage_times.argtypes = [vp, ctypes.POINTER(d)]
        L.bvf_fno_synchronize.argtypes = [vp, vp]
        L.bvf_gemm_bf16.argtypes = [ctypes.POINTER(Gemm), vp, vp]
        L.bvf_fno_bf16_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(FnoDims), vp,
                                          ctypes.c_size_t, i, i, i, i]
        L.bvf_fno_bf16_destroy.argtypes = [vp]
        L.bvf_fno_bf16_forward.argtypes = [vp, i, vp, vp, vp]
        L.bvf_fno_bf16_gradient.argtypes = [vp, i, vp, vp, vp, d, vp, ctypes.POINTER(d), vp]
        L.bvf_fno_bf16_adam.argtypes = [vp, i, vp, vp, vp, d, d, ctypes.POINTER(d), vp]
        L.bvf_fno_bf16_weights.argtypes = [vp, vp]
        L.bvf_fno_bf16_synchronize.argtypes = [vp, vp]
        L.bvf_fno_mean.argtypes = [vp, ctypes.c_size_t, ctypes.POINTER(d), vp]
        _declared = True
    return L


def bvf_gemm_bf16(A, a_strides, B, b_strides, C, c_strides, M, N, K, batch=1, ksplit=1,
                  alpha=1.0, beta=0.0, bias=None, bias_mode=0, act=0, C_pre=None, flag=None,
                  stream=None):
    """C = alpha A B + beta C (+ bias) (-> GELU) with BF16 operands on the tensor
    cores; strides in elements as (m, k, batch), (k, n, batch), (m, n, batch).
    flag: a one-element int32 CUDA tensor receiving bit 2 on a timed-out wait."""
    import torch
    ptr = lambda t: t.data_ptr() if t is not None else None
    g = Gemm(ptr(A), *a_strides, ptr(B), *b_strides, ptr(C), *c_strides, ptr(C_pre), ptr(bias),
             bias_mode, M, N, K, batch, ksplit, alpha, beta, act)
    if flag is None:
        flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    bvf._check(lib().bvf_gemm_bf16(ctypes.byref(g), ctypes.c_void_p(flag.data_ptr()),
                                   bvf._stream(stream)))
    return flag


def bvf_fno_weight_count(dims: FnoDims) -> int:
    return int(lib().bvf_fno_weight_count(ctypes.byref(dims)))


def bvf_fno_create(dims: FnoDims, weights):
    w = np.ascontiguousarray(weights, dtype=np.float32)
    h = ctypes.c_void_p()
    bvf._check(lib().bvf_fno_create(ctypes.byref(h), ctypes.byref(dims),
                                    w.ctypes.data_as(ctypes.c_void_p), w.size))
    return h


def bvf_fno_destroy(h):
    lib().bvf_fno_destroy(h)


def bvf_fno_forward(h, inp, out, stream=None):
    import torch
    c, nz, ny, nx = inp.shape
    bvf._check(lib().bvf_fno_forward(h, nx, ny, nz, bvf._ptr(inp, torch.float32),
                                     bvf._ptr(out, torch.float32), bvf._stream(stream)))


def bvf_fno_features(index, table, water_row, f0, k_src, src, p_norm, out, stream=None):
    """index: [nz, ny, nx] uint8 CUDA tensor; table, water_row: material rows
    (sequences of the nine bvf.Material fields); src: [ny, nx] complex64 CUDA
    tensor; out: [8, nz, ny, nx] float32 CUDA tensor."""
    import torch
    nz, ny, nx = index.shape
    tab = bvf.material_array(table)
    water = bvf.material_array([water_row])
    srcf = torch.view_as_real(src).contiguous() if src.is_complex() else src
    bvf._check(lib().bvf_fno_features(bvf._ptr(index, torch.uint8), tab, len(tab), water, nx, ny,
                                      nz, float(f0), int(k_src), bvf._ptr(srcf, torch.float32),
                                      float(p_norm), bvf._ptr(out, torch.float32),
                                      bvf._stream(stream)))


def bvf_fno_synchronize(h, stream=None):
    bvf._check(lib().bvf_fno_synchronize(h, bvf._stream(stream)))


def bvf_fno_timing(h, enable: bool):
    bvf._check(lib().bvf_fno_timing(h, 1 if enable else 0))


def bvf_fno_stage_times(h) -> dict:
    arr = (ctypes.c_double * N_STAGES)()
    bvf._check(lib().bvf_fno_stage_times(h, arr))
    return dict(zip(STAGES, list(arr)))


class Surrogate:
    """One surrogate context; call it on a [c_in, nz, ny, nx] CUDA tensor."""

    def __init__(self, dims: FnoDims | dict, weights):
        self.dims = dims if isinstance(dims, FnoDims) else FnoDims(**dims)
        self.h = bvf_fno_create(self.dims, weights)

    def __call__(self, inp, out=None, stream=None):
        import torch
        c, nz, ny, nx = inp.shape
        if out is None:
            out = torch.empty((self.dims.c_out, nz, ny, nx), dtype=torch.float32,
                              device=inp.device)
        bvf_fno_forward(self.h, inp, out, stream)
        return out

    def synchronize(self, stream=None):
        bvf_fno_synchronize(self.h, stream)

    def timing(self, enable: bool):
        bvf_fno_timing(self.h, enable)

    def stage_times(self) -> dict:
        return bvf_fno_stage_times(self.h)

    def close(self):
        if self.h:
            bvf_fno_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def predict_amplitude(net: Surrogate, index, table, water_row, f0, k_src, src, p0, amp_range,
                      fdtd=None, stream=None):
    """Amplitude field (Pa, [nz, ny, nx]) of one placement from the surrogate,
    with the FDTD as fallback.

    The features of the placement (bvf_fno_features) go through the network,
    whose output is the amplitude divided by the bowl's surface pressure p0.
    The prediction is kept when it is finite everywhere and its maximum lies
    inside amp_range = (lo, hi), the focal amplitudes (in units of p0) that the
    training data covered; otherwise `fdtd()` (a callable returning the FDTD
    amplitude field) is called instead, and if it is None a RuntimeError is
    raised.  Returns (amp, "surrogate" | "fdtd")."""
    import torch
    nz, ny, nx = index.shape
    feats = torch.empty((N_FEATURES, nz, ny, nx), dtype=torch.float32, device=index.device)
    bvf_fno_features(index, table, water_row, f0, k_src, src, p0, feats, stream)
    out = net(feats, stream=stream)
    net.synchronize(stream)
    u = out[0]
    ok = bool(torch.isfinite(u).all())
    if ok:
        mx = float(u.max())
        ok = amp_range[0] <= mx <= amp_range[1]
    if ok:
        return u * float(p0), "surrogate"
    if fdtd is None:
        raise RuntimeError("surrogate prediction outside its trained range and no FDTD fallback")
    return fdtd(), "fdtd"


def bvf_fno_mean(x, stream=None) -> float:
    """Mean of a float32 CUDA tensor (e.g. the transmission channel of an output)."""
    import torch
    v = ctypes.c_double()
    bvf._check(lib().bvf_fno_mean(bvf._ptr(x, torch.float32), x.numel(), ctypes.byref(v),
                                  bvf._stream(stream)))
    return v.value


class Bf16Net:
    """The surrogate with BF16 tensor-core products (bvf_fno_bf16_*): inference
    of batches of feature volumes and training (loss gradient, Adam steps) on
    one grid.  Argument marshalling only."""

    def __init__(self, dims, weights, grid, max_batch=1):
        self.dims = dims if isinstance(dims, FnoDims) else FnoDims(**dims)
        self.nx, self.ny, self.nz = grid
        self.max_batch = max_batch
        w = np.ascontiguousarray(weights, dtype=np.float32)
        h = ctypes.c_void_p()
        bvf._check(lib().bvf_fno_bf16_create(ctypes.byref(h), ctypes.byref(self.dims),
                                             w.ctypes.data_as(ctypes.c_void_p), w.size, self.nx,
                                             self.ny, self.nz, max_batch))
        self.h = h
        self.n_w = w.size

    def close(self):
        if self.h:
            lib().bvf_fno_bf16_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, x, out=None, stream=None):
        """x: [batch, c_in, nz, ny, nx] float32 CUDA tensor."""
        import torch
        b = x.shape[0]
        if out is None:
            out = torch.empty((b, self.dims.c_out, self.nz, self.ny, self.nx), dtype=torch.float32,
                              device="cuda")
        bvf._check(lib().bvf_fno_bf16_forward(self.h, b, bvf._ptr(x, torch.float32),
                                              bvf._ptr(out, torch.float32), bvf._stream(stream)))
        return out

    def gradient(self, x, target, el=None, el_weight=0.0, stream=None):
        """(loss, gradient as a float32 CUDA tensor in the blob layout)."""
        import torch
        g = torch.empty(self.n_w, dtype=torch.float32, device="cuda")
        loss = ctypes.c_double()
        bvf._check(lib().bvf_fno_bf16_gradient(
            self.h, x.shape[0], bvf._ptr(x, torch.float32), bvf._ptr(target, torch.float32),
            bvf._ptr(el, torch.float32) if el is not None else None, float(el_weight),
            bvf._ptr(g, torch.float32), ctypes.byref(loss), bvf._stream(stream)))
        return loss.value, g

    def adam(self, x, target, lr, el=None, el_weight=0.0, stream=None):
        """One Adam step on a batch; returns the batch loss before the step."""
        import torch
        loss = ctypes.c_double()
        bvf._check(lib().bvf_fno_bf16_adam(
            self.h, x.shape[0], bvf._ptr(x, torch.float32), bvf._ptr(target, torch.float32),
            bvf._ptr(el, torch.float32) if el is not None else None, float(el_weight), float(lr),
            ctypes.byref(loss), bvf._stream(stream)))
        return loss.value

    def weights(self):
        w = np.empty(self.n_w, dtype=np.float32)
        bvf._check(lib().bvf_fno_bf16_weights(self.h, w.ctypes.data_as(ctypes.c_void_p)))
        return w

    def synchronize(self, stream=None):
        bvf._check(lib().bvf_fno_bf16_synchronize(self.h, bvf._stream(stream)))
