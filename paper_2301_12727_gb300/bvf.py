"""Python binding of libbvf (ctypes).  Argument marshalling only: every step of
the hot path runs in the CUDA library; this module never computes a field.

Functions carry the C ABI's names (include/bvf.h) and take torch CUDA tensors
for device pointers; the stream is torch's current stream unless given.
`Solver` bundles one context with the buffers a caller usually wants.

The library must have been built (``__graft_entry__.build()`` or
``python -m paper_2301_12727_gb300.build``); importing without it raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbvf.so")

BVF_OK, BVF_E_ARG, BVF_E_CFL, BVF_E_MATERIAL = 0, -1, -2, -3
BVF_E_NOMEM, BVF_E_CUDA, BVF_E_UNSTABLE, BVF_E_TIMEOUT = -4, -5, -6, -7
BVF_ENV_NONE, BVF_ENV_BURST, BVF_ENV_RAMP_CW = 0, 1, 2
FIELDS = ("vx", "vy", "vz", "sxx", "syy", "szz", "sxy", "sxz", "syz")
EXPORTS = ("bvf_version", "bvf_courant_limit", "bvf_strerror", "bvf_create", "bvf_destroy",
           "bvf_last_error", "bvf_set_materials", "bvf_rs_plane", "bvf_set_source", "bvf_reset",
           "bvf_run_acoustic", "bvf_synchronize", "bvf_get_field", "bvf_set_field",
           "bvf_get_pressure", "bvf_get_peak", "bvf_get_amp_phase", "bvf_run_thermal",
           "bvf_transmission", "bvf_get_stats", "bvf_kernel_timing", "bvf_get_kernel_times",
           "bvf_transmission_noalloc", "bvf_batch_create", "bvf_batch_destroy", "bvf_batch_run",
           "bvf_batch_tune", "bvf_batch_launches", "bvf_batch_run_streams", "bvf_plan",
           "bvf_rs_elements", "bvf_set_time_budget", "bvf_state_bytes", "bvf_state_save",
           "bvf_state_load", "bvf_test_withhold_copy", "bvf_bowl_array", "bvf_steer_weights",
           "bvf_time_reversal_plane", "bvf_batch_run_graph", "bvf_batch_tune_domains",
           "bvf_set_tile", "bvf_get_tile", "bvf_batch_tune_graph", "bvf_plan_host")


class BvfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libbvf error %d: %s" % (code, msg))
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("n_pml", ctypes.c_int),
                ("pml_R", ctypes.c_double)]


class Material(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("rho", "cL", "cS", "alphaL", "alphaS", "k_th", "c_th", "perf", "heat_frac")]


BVF_STORAGE_F32, BVF_STORAGE_F16 = 0, 1
STORAGE = {"f32": BVF_STORAGE_F32, "f16": BVF_STORAGE_F16}


class Physics(ctypes.Structure):
    _fields_ = [("f0", ctypes.c_double), ("qc", ctypes.c_double), ("n_sls", ctypes.c_int),
                ("storage", ctypes.c_int), ("p_ref", ctypes.c_double)]


class Bowl(ctypes.Structure):
    _fields_ = [("aperture", ctypes.c_double), ("roc", ctypes.c_double),
                ("apex", ctypes.c_double * 3), ("dir", ctypes.c_double * 3),
                ("p0", ctypes.c_double), ("c0", ctypes.c_double),
                ("ds_over_lambda", ctypes.c_double)]


class Capture(ctypes.Structure):
    _fields_ = [("peak_from", ctypes.c_int), ("dft_start", ctypes.c_int),
                ("dft_steps", ctypes.c_int)]


class Thermal(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("n_on", ctypes.c_int), ("n_off", ctypes.c_int),
                ("duty", ctypes.c_double), ("T_a", ctypes.c_double), ("rhob_cb", ctypes.c_double),
                ("p_scale", ctypes.c_double)]


class PlanParams(ctypes.Structure):
    _fields_ = [("n_steps", ctypes.c_int), ("dft_start", ctypes.c_int), ("dft_steps", ctypes.c_int),
                ("i_sppa", ctypes.c_double), ("thermal", Thermal), ("serial", ctypes.c_int)]


class PlanOut(ctypes.Structure):
    _fields_ = [("EL", ctypes.c_double), ("TS", ctypes.c_double), ("Iw_max", ctypes.c_double),
                ("p_scale", ctypes.c_double), ("z_m", ctypes.c_int)]


class Tile(ctypes.Structure):
    _fields_ = [("stress_rows", ctypes.c_int), ("velocity_rows", ctypes.c_int),
                ("kchunk", ctypes.c_int)]


# candidates of the per-domain tile autotuner: (stress rows, velocity rows, z-planes per block)
TILE_CANDIDATES = tuple((s, v, k) for s, v in ((8, 16), (8, 8), (16, 16))
                        for k in (6, 8, 10, 13, 16))


class Stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_longlong), ("kernel_launches", ctypes.c_longlong),
                ("thermal_steps", ctypes.c_longlong), ("courant", ctypes.c_double),
                ("bytes_per_voxel_step", ctypes.c_double)]


class KernelTimes(ctypes.Structure):
    _fields_ = [("velocity_launches", ctypes.c_longlong), ("stress_launches", ctypes.c_longlong),
                ("velocity_ms", ctypes.c_double), ("stress_ms", ctypes.c_double)]


_lib = None


def lib():
    """Load libbvf.so (fails loudly when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libbvf.so is not built: run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.bvf_version.restype = i
        L.bvf_courant_limit.restype = d
        L.bvf_strerror.restype = ctypes.c_char_p
        L.bvf_strerror.argtypes = [i]
        L.bvf_last_error.restype = ctypes.c_char_p
        L.bvf_last_error.argtypes = [vp]
        L.bvf_create.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Physics), ctypes.POINTER(vp)]
        L.bvf_destroy.argtypes = [vp]
        L.bvf_destroy.restype = None
        L.bvf_set_materials.argtypes = [vp, vp, ctypes.POINTER(Material), i]
        L.bvf_rs_plane.argtypes = [ctypes.POINTER(Bowl), i, i, d, d, d, vp, vp]
        L.bvf_set_source.argtypes = [vp, i, vp, d, i, i, vp]
        L.bvf_reset.argtypes = [vp, vp]
        L.bvf_run_acoustic.argtypes = [vp, i, ctypes.POINTER(Capture), vp]
        L.bvf_synchronize.argtypes = [vp, vp]
        L.bvf_get_field.argtypes = [vp, i, vp, vp]
        L.bvf_set_field.argtypes = [vp, i, vp, vp]
        L.bvf_get_pressure.argtypes = [vp, vp, vp]
        L.bvf_get_peak.argtypes = [vp, vp, vp]
        L.bvf_get_amp_phase.argtypes = [vp, vp, vp, vp]
        L.bvf_run_thermal.argtypes = [vp, ctypes.POINTER(Thermal), vp, vp, vp, vp, vp]
        L.bvf_transmission.argtypes = [i, i, i, vp, ctypes.POINTER(Material), i, vp, vp,
                                       ctypes.POINTER(Material), i, vp,
                                       ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(i),
                                       ctypes.POINTER(d), vp]
        L.bvf_transmission_noalloc.argtypes = L.bvf_transmission.argtypes
        L.bvf_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
        L.bvf_kernel_timing.argtypes = [vp, i]
        L.bvf_get_kernel_times.argtypes = [vp, ctypes.POINTER(KernelTimes)]
        L.bvf_batch_create.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(vp)]
        L.bvf_batch_destroy.argtypes = [vp]
        L.bvf_batch_destroy.restype = None
        L.bvf_batch_run.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(Capture), i, i, vp]
        L.bvf_batch_tune.argtypes = [vp, i, ctypes.POINTER(i), i, ctypes.POINTER(i),
                                     ctypes.POINTER(d), vp]
        L.bvf_batch_launches.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
        L.bvf_batch_run_streams.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(Capture), i, vp]
        L.bvf_rs_elements.argtypes = [vp, i, d, d, i, i, d, d, d, vp, vp]
        L.bvf_plan.argtypes = [vp, vp, vp, ctypes.POINTER(Material), i, ctypes.POINTER(Material),
                               ctypes.POINTER(Bowl), i, ctypes.POINTER(PlanParams), vp, vp, vp, vp,
                               vp, ctypes.POINTER(PlanOut), vp]
        L.bvf_plan_host.argtypes = [vp, vp, vp, ctypes.POINTER(Material), i,
                                    ctypes.POINTER(Material), ctypes.POINTER(Bowl), i,
                                    ctypes.POINTER(PlanParams), vp, vp, vp, vp,
                                    ctypes.POINTER(PlanOut), vp]
        L.bvf_set_time_budget.argtypes = [vp, d]
        L.bvf_batch_run_graph.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(Capture), i, vp]
        L.bvf_batch_tune_domains.argtypes = [vp, i, ctypes.POINTER(Tile), i, ctypes.POINTER(Tile),
                                             vp]
        L.bvf_set_tile.argtypes = [vp, ctypes.POINTER(Tile)]
        L.bvf_batch_tune_graph.argtypes = [vp, i, ctypes.POINTER(Tile), i, i, ctypes.POINTER(Tile),
                                           ctypes.POINTER(ctypes.c_double), vp]
        L.bvf_get_tile.argtypes = [vp, ctypes.POINTER(Tile)]
        L.bvf_state_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
        L.bvf_state_save.argtypes = [vp, vp, ctypes.c_size_t, vp]
        L.bvf_state_load.argtypes = [vp, vp, ctypes.c_size_t, vp]
        L.bvf_test_withhold_copy.argtypes = [vp, i, i, ctypes.c_uint]
        L.bvf_bowl_array.argtypes = [ctypes.POINTER(Bowl), i, i, vp, ctypes.POINTER(i)]
        L.bvf_steer_weights.argtypes = [vp, i, vp, d, d]
        L.bvf_time_reversal_plane.argtypes = [vp, i, i, i, i, i, d, vp, vp]
        _lib = L
    return _lib


def _check(rc, ctx=None):
    if rc != BVF_OK:
        msg = lib().bvf_last_error(ctx)
        raise BvfError(rc, msg.decode() if msg else "")
    return rc


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t, dtype=None):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError("expected dtype %s, got %s" % (dtype, t.dtype))
    return ctypes.c_void_p(t.data_ptr())


def material_array(rows) -> "ctypes.Array":
    rows = np.asarray(rows, dtype=np.float64).reshape(-1, 9)
    arr = (Material * rows.shape[0])()
    for m, r in enumerate(rows):
        arr[m] = Material(*[float(v) for v in r])
    return arr


# ---- C ABI, one wrapper per entry point ----------------------------------
def bvf_version():
    return lib().bvf_version()


def bvf_courant_limit():
    return lib().bvf_courant_limit()


def bvf_create(grid: Grid, phys: Physics):
    ctx = ctypes.c_void_p()
    _check(lib().bvf_create(ctypes.byref(grid), ctypes.byref(phys), ctypes.byref(ctx)))
    return ctx


def bvf_destroy(ctx):
    lib().bvf_destroy(ctx)


def bvf_set_materials(ctx, index, table):
    import torch
    arr = material_array(table)
    _check(lib().bvf_set_materials(ctx, _ptr(index, torch.uint8), arr, len(arr)), ctx)


def bvf_rs_plane(bowl: Bowl, nx, ny, dx, z_plane, f0, out, stream=None):
    import torch
    _check(lib().bvf_rs_plane(ctypes.byref(bowl), nx, ny, dx, z_plane, f0,
                              _ptr(out, torch.float32), _stream(stream)))


def bvf_set_source(ctx, k_plane, plane, c0, envelope, n_cycles=0, stream=None):
    import torch
    _check(lib().bvf_set_source(ctx, k_plane, _ptr(plane, torch.float32), c0, envelope, n_cycles,
                                _stream(stream)), ctx)


def bvf_reset(ctx, stream=None):
    _check(lib().bvf_reset(ctx, _stream(stream)), ctx)


def bvf_run_acoustic(ctx, n_steps, capture: Capture | None = None, stream=None):
    cap = ctypes.byref(capture) if capture is not None else None
    _check(lib().bvf_run_acoustic(ctx, n_steps, cap, _stream(stream)), ctx)


def bvf_synchronize(ctx, stream=None):
    return _check(lib().bvf_synchronize(ctx, _stream(stream)), ctx)


def bvf_get_field(ctx, which, out, stream=None):
    import torch
    _check(lib().bvf_get_field(ctx, which, _ptr(out, torch.float32), _stream(stream)), ctx)


def bvf_set_field(ctx, which, src, stream=None):
    import torch
    _check(lib().bvf_set_field(ctx, which, _ptr(src, torch.float32), _stream(stream)), ctx)


def bvf_get_pressure(ctx, out, stream=None):
    import torch
    _check(lib().bvf_get_pressure(ctx, _ptr(out, torch.float32), _stream(stream)), ctx)


def bvf_get_peak(ctx, out, stream=None):
    import torch
    _check(lib().bvf_get_peak(ctx, _ptr(out, torch.float32), _stream(stream)), ctx)


def bvf_get_amp_phase(ctx, amp, phase, stream=None):
    import torch
    _check(lib().bvf_get_amp_phase(ctx, _ptr(amp, torch.float64), _ptr(phase, torch.float64),
                                   _stream(stream)), ctx)


def bvf_run_thermal(ctx, th: Thermal, amp, T, Tmax, cem, stream=None):
    import torch
    _check(lib().bvf_run_thermal(ctx, ctypes.byref(th), _ptr(amp, torch.float64),
                                 _ptr(T, torch.float32), _ptr(Tmax, torch.float32),
                                 _ptr(cem, torch.float64), _stream(stream)), ctx)


def bvf_transmission(idx_a, table_a, amp_a, idx_w, table_w, amp_w, stream=None):
    import torch
    nz, ny, nx = idx_a.shape
    ma, mw = material_array(table_a), material_array(table_w)
    el, ts, zm, iw = ctypes.c_double(), ctypes.c_double(), ctypes.c_int(), ctypes.c_double()
    _check(lib().bvf_transmission(nx, ny, nz, _ptr(idx_a, torch.uint8), ma, len(ma),
                                  _ptr(amp_a, torch.float64), _ptr(idx_w, torch.uint8), mw,
                                  len(mw), _ptr(amp_w, torch.float64), ctypes.byref(el),
                                  ctypes.byref(ts), ctypes.byref(zm), ctypes.byref(iw),
                                  _stream(stream)))
    return el.value, ts.value, zm.value, iw.value


def bvf_transmission_noalloc(idx_a, table_a, amp_a, idx_w, table_w, amp_w, stream=None):
    """bvf_transmission for callers that cannot allocate device memory: the
    library keeps the reduction's temporaries in a fixed array (see bvf.h)."""
    import torch
    nz, ny, nx = idx_a.shape
    ma, mw = material_array(table_a), material_array(table_w)
    el, ts, zm, iw = ctypes.c_double(), ctypes.c_double(), ctypes.c_int(), ctypes.c_double()
    _check(lib().bvf_transmission_noalloc(nx, ny, nz, _ptr(idx_a, torch.uint8), ma, len(ma),
                                          _ptr(amp_a, torch.float64), _ptr(idx_w, torch.uint8),
                                          mw, len(mw), _ptr(amp_w, torch.float64),
                                          ctypes.byref(el), ctypes.byref(ts), ctypes.byref(zm),
                                          ctypes.byref(iw), _stream(stream)))
    return el.value, ts.value, zm.value, iw.value


def bvf_get_stats(ctx) -> Stats:
    s = Stats()
    _check(lib().bvf_get_stats(ctx, ctypes.byref(s)), ctx)
    return s


def bvf_kernel_timing(ctx, enable: bool):
    _check(lib().bvf_kernel_timing(ctx, 1 if enable else 0), ctx)


def bvf_get_kernel_times(ctx) -> KernelTimes:
    t = KernelTimes()
    _check(lib().bvf_get_kernel_times(ctx, ctypes.byref(t)), ctx)
    return t


def bvf_set_time_budget(ctx, seconds):
    _check(lib().bvf_set_time_budget(ctx, float(seconds)), ctx)


def bvf_state_bytes(ctx) -> int:
    n = ctypes.c_size_t()
    _check(lib().bvf_state_bytes(ctx, ctypes.byref(n)), ctx)
    return n.value


def bvf_state_save(ctx, buf, stream=None):
    import torch
    _check(lib().bvf_state_save(ctx, _ptr(buf, torch.uint8), buf.numel(), _stream(stream)), ctx)


def bvf_state_load(ctx, buf, stream=None):
    import torch
    _check(lib().bvf_state_load(ctx, _ptr(buf, torch.uint8), buf.numel(), _stream(stream)), ctx)


def bvf_test_withhold_copy(ctx, kernel, plane, wait_limit=0):
    _check(lib().bvf_test_withhold_copy(ctx, kernel, plane, wait_limit), ctx)


def bvf_bowl_array(bowl: Bowl, n_rings, n_inner) -> np.ndarray:
    """Rows (x, y, z, area, 1, 0) of a spherical cap's elements."""
    n = ctypes.c_int()
    _check(lib().bvf_bowl_array(ctypes.byref(bowl), n_rings, n_inner, None, ctypes.byref(n)))
    out = np.zeros((n.value, 6))
    _check(lib().bvf_bowl_array(ctypes.byref(bowl), n_rings, n_inner,
                                out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n)))
    return out


def bvf_steer_weights(elements, target, f0, c0=1500.0) -> np.ndarray:
    """A copy of the element rows with steering weights exp(+i k r) towards target."""
    el = np.array(elements, dtype=np.float64).reshape(-1, 6)
    tg = np.ascontiguousarray(np.asarray(target, dtype=np.float64).reshape(3))
    _check(lib().bvf_steer_weights(el.ctypes.data_as(ctypes.c_void_p), el.shape[0],
                                   tg.ctypes.data_as(ctypes.c_void_p), f0, c0))
    return el


def bvf_time_reversal_plane(ctx, target_ijk, k_src, n_steps, c0, out, stream=None):
    import torch
    i, j, k = (int(v) for v in target_ijk)
    _check(lib().bvf_time_reversal_plane(ctx, i, j, k, k_src, n_steps, c0,
                                         _ptr(out, torch.float32), _stream(stream)), ctx)


# ---- convenience ---------------------------------------------------------
class Solver:
    """One libbvf context on the current CUDA device."""

    def __init__(self, nx, ny, nz, dx, dt, f0, qc=1.0, n_sls=2, n_pml=8, pml_R=1e-4,
                 storage="f32", p_ref=0.0):
        """storage "f32", or "f16" (scaled FP16 state, FP32 arithmetic; p_ref in Pa
        near the largest expected pressure, 0 = 1e5)."""
        self.shape = (nz, ny, nx)
        self.grid = Grid(nx, ny, nz, dx, dt, n_pml, pml_R)
        self.phys = Physics(f0, qc, n_sls, STORAGE[storage], p_ref)
        self.storage = storage
        self.n_sls = n_sls
        self.ctx = bvf_create(self.grid, self.phys)

    def close(self):
        if self.ctx:
            bvf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_materials(self, index, table):
        import torch
        idx = torch.as_tensor(np.asarray(index, dtype=np.uint8) if not torch.is_tensor(index)
                              else index).to("cuda", torch.uint8).contiguous()
        bvf_set_materials(self.ctx, idx, table)
        self.table = np.asarray(table, dtype=np.float64).reshape(-1, 9)

    def set_source(self, plane, k_plane, c0, envelope, n_cycles=0, stream=None):
        """plane: complex (ny, nx) array/tensor, or a float32 CUDA tensor (ny, nx, 2)."""
        import torch
        if torch.is_tensor(plane) and plane.dtype == torch.float32:
            pl = plane.contiguous()
        else:
            p = np.asarray(plane.cpu() if torch.is_tensor(plane) else plane).astype(np.complex128)
            pl = torch.from_numpy(np.stack([p.real, p.imag], -1).astype(np.float32)).cuda()
        bvf_set_source(self.ctx, k_plane, pl, c0, envelope, n_cycles, stream)
        self._plane = pl

    def run(self, n_steps, peak_from=-1, dft_start=0, dft_steps=0, stream=None):
        bvf_run_acoustic(self.ctx, n_steps, Capture(peak_from, dft_start, dft_steps), stream)

    def reset(self, stream=None):
        bvf_reset(self.ctx, stream)

    def synchronize(self, stream=None):
        bvf_synchronize(self.ctx, stream)

    def _empty(self, dtype):
        import torch
        return torch.empty(self.shape, dtype=dtype, device="cuda")

    def field(self, name_or_id, stream=None):
        import torch
        which = FIELDS.index(name_or_id) if isinstance(name_or_id, str) else name_or_id
        out = self._empty(torch.float32)
        bvf_get_field(self.ctx, which, out, stream)
        return out

    def set_field(self, name_or_id, value, stream=None):
        import torch
        which = FIELDS.index(name_or_id) if isinstance(name_or_id, str) else name_or_id
        t = torch.as_tensor(value, dtype=torch.float32).cuda().contiguous()
        bvf_set_field(self.ctx, which, t, stream)
        self._keep = t

    def memory_id(self, l, c):
        return 9 + 6 * l + c

    def pressure(self, stream=None):
        import torch
        out = self._empty(torch.float32)
        bvf_get_pressure(self.ctx, out, stream)
        return out

    def peak(self, stream=None):
        import torch
        out = self._empty(torch.float32)
        bvf_get_peak(self.ctx, out, stream)
        return out

    def amp_phase(self, stream=None):
        import torch
        amp, ph = self._empty(torch.float64), self._empty(torch.float64)
        bvf_get_amp_phase(self.ctx, amp, ph, stream)
        return amp, ph

    def thermal(self, amp, dt, n_on, n_off, duty, T_a=37.0, rhob_cb=1050.0 * 3617.0,
                p_scale=1.0, T=None, Tmax=None, cem=None, stream=None):
        import torch
        T = torch.full(self.shape, T_a, dtype=torch.float32, device="cuda") if T is None else T
        Tmax = T.clone() if Tmax is None else Tmax
        cem = torch.zeros(self.shape, dtype=torch.float64, device="cuda") if cem is None else cem
        bvf_run_thermal(self.ctx, Thermal(dt, n_on, n_off, duty, T_a, rhob_cb, p_scale), amp, T,
                        Tmax, cem, stream)
        return T, Tmax, cem

    def stats(self) -> Stats:
        return bvf_get_stats(self.ctx)

    def set_time_budget(self, seconds):
        bvf_set_time_budget(self.ctx, seconds)

    def set_tile(self, stress_rows=0, velocity_rows=0, kchunk=0):
        """Rows of the stress and velocity kernels' x-y tiles (0 = default, 4,
        8, 16) and z-planes per block (0 = default)."""
        t = Tile(int(stress_rows), int(velocity_rows), int(kchunk))
        _check(lib().bvf_set_tile(self.ctx, ctypes.byref(t)), self.ctx)

    def tile(self):
        """(stress rows, velocity rows, z-chunk) the kernels use."""
        t = Tile()
        _check(lib().bvf_get_tile(self.ctx, ctypes.byref(t)), self.ctx)
        return t.stress_rows, t.velocity_rows, t.kchunk

    def save_state(self, stream=None):
        """Snapshot of the acoustic state in a fresh uint8 CUDA tensor."""
        import torch
        buf = torch.empty(bvf_state_bytes(self.ctx), dtype=torch.uint8, device="cuda")
        bvf_state_save(self.ctx, buf, stream)
        return buf

    def load_state(self, buf, stream=None):
        bvf_state_load(self.ctx, buf, stream)

    def kernel_timing(self, enable: bool):
        bvf_kernel_timing(self.ctx, enable)

    def kernel_times(self) -> KernelTimes:
        return bvf_get_kernel_times(self.ctx)


def make_bowl(bowl: dict, c0=1500.0, ds_over_lambda=0.25) -> Bowl:
    return Bowl(bowl["aperture"], bowl["roc"], (ctypes.c_double * 3)(*bowl["apex"]),
                (ctypes.c_double * 3)(*bowl["dir"]), bowl["p0"], c0, ds_over_lambda)


def rs_plane(bowl: dict, nx, ny, dx, z_plane, f0, c0=1500.0, ds_over_lambda=0.25, stream=None):
    """Rayleigh-Sommerfeld plane as a (ny, nx, 2) float32 CUDA tensor."""
    import torch
    b = make_bowl(bowl, c0, ds_over_lambda)
    out = torch.empty((ny, nx, 2), dtype=torch.float32, device="cuda")
    bvf_rs_plane(b, nx, ny, dx, z_plane, f0, out, stream)
    return out


def bvf_rs_elements(elements, p0, c0, nx, ny, dx, z_plane, f0, stream=None):
    """Field of weighted elements (rows x, y, z, area, w_re, w_im) as a
    (ny, nx, 2) float32 CUDA tensor."""
    import torch
    el = np.ascontiguousarray(np.asarray(elements, dtype=np.float64).reshape(-1, 6))
    out = torch.empty((ny, nx, 2), dtype=torch.float32, device="cuda")
    _check(lib().bvf_rs_elements(el.ctypes.data_as(ctypes.c_void_p), el.shape[0], float(p0),
                                 float(c0), int(nx), int(ny), float(dx), float(z_plane), float(f0),
                                 _ptr(out, torch.float32), _stream(stream)))
    return out


# ---- batched sweeps ---------------------------------------------------------
def bvf_batch_create(ctxs):
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value if isinstance(c, ctypes.c_void_p) else c
                                          for c in ctxs])
    out = ctypes.c_void_p()
    _check(lib().bvf_batch_create(arr, len(ctxs), ctypes.byref(out)))
    return out


def bvf_batch_run(batch, n_steps, caps=None, kchunk=0, graph_steps=0, stream=None):
    n = len(n_steps)
    steps = (ctypes.c_int * n)(*[int(v) for v in n_steps])
    cp = None
    if caps is not None:
        cp = (Capture * n)(*[c if isinstance(c, Capture) else Capture(*c) for c in caps])
    _check(lib().bvf_batch_run(batch, steps, cp, int(kchunk), int(graph_steps), _stream(stream)))


def bvf_batch_tune(batch, trial_steps, candidates, stream=None):
    cand = (ctypes.c_int * len(candidates))(*[int(v) for v in candidates])
    best, ms = ctypes.c_int(), ctypes.c_double()
    _check(lib().bvf_batch_tune(batch, int(trial_steps), cand, len(candidates), ctypes.byref(best),
                                ctypes.byref(ms), _stream(stream)))
    return best.value, ms.value


class Batch:
    """Several Solvers advanced in lockstep by the persistent batch kernels
    (optionally replayed from a CUDA graph)."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        self.handle = bvf_batch_create([s.ctx for s in self.solvers])

    def run(self, n_steps, caps=None, kchunk=0, graph_steps=0, stream=None):
        if isinstance(n_steps, int):
            n_steps = [n_steps] * len(self.solvers)
        bvf_batch_run(self.handle, n_steps, caps, kchunk, graph_steps, stream)

    def run_streams(self, n_steps, caps=None, n_streams=4, stream=None):
        n = len(self.solvers)
        if isinstance(n_steps, int):
            n_steps = [n_steps] * n
        steps = (ctypes.c_int * n)(*[int(v) for v in n_steps])
        cp = None
        if caps is not None:
            cp = (Capture * n)(*[c if isinstance(c, Capture) else Capture(*c) for c in caps])
        _check(lib().bvf_batch_run_streams(self.handle, steps, cp, int(n_streams),
                                           _stream(stream)))

    def run_graph(self, n_steps, caps=None, n_branches=8, stream=None):
        """The sweep as one recorded CUDA graph of per-domain launches on
        n_branches parallel branches (bvf_batch_run_graph)."""
        n = len(self.solvers)
        if isinstance(n_steps, int):
            n_steps = [n_steps] * n
        steps = (ctypes.c_int * n)(*[int(v) for v in n_steps])
        cp = None
        if caps is not None:
            cp = (Capture * n)(*[c if isinstance(c, Capture) else Capture(*c) for c in caps])
        _check(lib().bvf_batch_run_graph(self.handle, steps, cp, int(n_branches), _stream(stream)))

    def tune(self, trial_steps=20, candidates=(6, 8, 10, 13, 16, 24), stream=None):
        return bvf_batch_tune(self.handle, trial_steps, candidates, stream)

    def tune_domains(self, trial_steps=10, candidates=TILE_CANDIDATES, stream=None):
        """Per-domain tile autotuner over (stress rows, velocity rows, z-chunk)
        candidates; returns the chosen triple of each domain."""
        n = len(self.solvers)
        cand = (Tile * len(candidates))(*[Tile(int(a), int(b), int(k)) for a, b, k in candidates])
        best = (Tile * n)()
        _check(lib().bvf_batch_tune_domains(self.handle, trial_steps, cand, len(candidates), best,
                                            _stream(stream)))
        return [(b.stress_rows, b.velocity_rows, b.kchunk) for b in best]

    def tune_graph(self, trial_steps=20, candidates=TILE_CANDIDATES, n_branches=8, stream=None):
        """Graph-mode tile autotuner (one tile for all domains, timed under
        concurrency); returns ((stress rows, velocity rows, z-chunk), ms per step)."""
        cand = (Tile * len(candidates))(*[Tile(int(a), int(b), int(k)) for a, b, k in candidates])
        best, ms = Tile(), ctypes.c_double()
        _check(lib().bvf_batch_tune_graph(self.handle, trial_steps, cand, len(candidates),
                                          int(n_branches), ctypes.byref(best), ctypes.byref(ms),
                                          _stream(stream)))
        return (best.stress_rows, best.velocity_rows, best.kchunk), ms.value

    def launches(self):
        out = ctypes.c_longlong()
        _check(lib().bvf_batch_launches(self.handle, ctypes.byref(out)))
        return out.value

    def close(self):
        if self.handle:
            lib().bvf_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- one placement end to end ----------------------------------------------
def _host_ptr(a, dtype):
    """Address of a contiguous host array (numpy, or a CPU torch tensor)."""
    import numpy as np
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("expected a C-contiguous %s array" % np.dtype(dtype).name)
        return ctypes.c_void_p(a.ctypes.data)
    if a.is_cuda or not a.is_contiguous():
        raise ValueError("expected a contiguous host tensor")
    return ctypes.c_void_p(a.data_ptr())


def bvf_plan_host(skull, water, h_index, table, water_row, bowl, k_src, params, h_peak, h_T,
                  h_Tmax, h_cem, stream=None):
    """bvf_plan with host buffers (numpy arrays or pinned CPU tensors);
    returns a PlanOut."""
    import numpy as np
    tab = material_array(table)
    wat = material_array([water_row])
    b = bowl if isinstance(bowl, Bowl) else make_bowl(bowl)
    out = PlanOut()
    _check(lib().bvf_plan_host(skull.ctx, water.ctx, _host_ptr(h_index, np.uint8), tab, len(tab),
                               wat, ctypes.byref(b), int(k_src), ctypes.byref(params),
                               _host_ptr(h_peak, np.float32),
                               _host_ptr(h_T, np.float32) if h_T is not None else None,
                               _host_ptr(h_Tmax, np.float32), _host_ptr(h_cem, np.float64),
                               ctypes.byref(out), _stream(stream)))
    return out


def bvf_plan(skull, water, index, table, water_row, bowl, k_src, params, peak, amp, T, Tmax, cem,
             stream=None):
    """Returns a PlanOut; outputs land in the given CUDA tensors."""
    import torch
    tab = material_array(table)
    wat = material_array([water_row])
    b = bowl if isinstance(bowl, Bowl) else make_bowl(bowl)
    out = PlanOut()
    _check(lib().bvf_plan(skull.ctx, water.ctx, _ptr(index, torch.uint8), tab, len(tab), wat,
                          ctypes.byref(b), int(k_src), ctypes.byref(params),
                          _ptr(peak, torch.float32), _ptr(amp, torch.float64),
                          _ptr(T, torch.float32), _ptr(Tmax, torch.float32),
                          _ptr(cem, torch.float64), ctypes.byref(out), _stream(stream)))
    return out
