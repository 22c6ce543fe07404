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
           "bvf_fno_features", "bvf_fno_timing", "bvf_fno_stage_times", "bvf_fno_synchronize")
N_FEATURES = 8
N_STAGES = 9
STAGES = ("lift", "dft_x", "dft_y", "dft_z", "mix", "idft_z", "idft_y", "out_x_pointwise",
          "project")


class FnoDims(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in
                ("c_in", "width", "modes", "n_layers", "hidden", "c_out")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


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
        _declared = True
    return L


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
