"""FP64 CPU oracle for the transcranial FDTD + BHTE hot path (arXiv 2301.12727).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package; the product library never does.  It wraps ``bvf_oracle.c`` (plain C,
double precision) through ctypes and shares no code with the CUDA path.

Parity status per function (pins live in tests/test_oracle_pins.py):
  material_coefs   pinned (Q(w0) and phase speed from the complex modulus)
  acoustic_run     pinned (exact discrete plane waves, energy conservation,
                   SLS relaxation vs the continuum ODE, attenuation of a point
                   source, normal-incidence reflection, CFL, mirror symmetry;
                   index conventions against a second, array-form FP64
                   implementation on small random media, tests/second_oracle.py)
  rs_plane         pinned (O'Neil on-axis field of a spherical bowl)
  rs_elements      pinned (single-element magnitude; coherent sum of a steered
                   array at its target)
  bhte_run         pinned (Gaussian diffusion with perfusion; constant-T CEM43)
  transmission     pinned (constructed maps with known E_L; identical runs)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bvf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_bvf.so")

E_ARG, E_CFL, E_MATERIAL = -1, -2, -3
ENV_NONE, ENV_BURST, ENV_RAMP_CW = 0, 1, 2

# material row layout
MAT_COLS = ("rho", "cL", "cS", "alphaL", "alphaS", "k_th", "c_th", "perf", "heat_frac")
N_PSI = 18


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dt", ctypes.c_double),
                ("n_pml", ctypes.c_int), ("pml_R", ctypes.c_double),
                ("f0", ctypes.c_double), ("qc", ctypes.c_double), ("n_sls", ctypes.c_int)]


_lib = None


def lib():
    """The oracle library; BVF_ORACLE_LIB names another build of bvf_oracle.c
    (used to check that the pins catch planted mistakes)."""
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(os.environ.get("BVF_ORACLE_LIB") or build())
        d = ctypes.c_double
        _lib.orc_courant_limit.restype = d
        _lib.orc_bowl_elements.restype = ctypes.c_long
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def n_fields(n_sls: int) -> int:
    return 9 + 6 * n_sls + N_PSI


def courant_limit() -> float:
    return lib().orc_courant_limit()


def materials(rows) -> np.ndarray:
    """Material table as a contiguous (n, 9) float64 array."""
    m = np.ascontiguousarray(np.asarray(rows, dtype=np.float64).reshape(-1, len(MAT_COLS)))
    return m


def relaxation_times(f0: float, n_sls: int) -> np.ndarray:
    ts = np.zeros(max(n_sls, 1))
    lib().orc_relaxation_times(ctypes.c_double(f0), ctypes.c_int(n_sls), _p(ts))
    return ts[:n_sls]


def material_coefs(mat, f0, qc, n_sls):
    """(rc, coef[n,4] = pi_R, mu_R, tau_P, tau_S, tau_sigma[L])."""
    mat = materials(mat)
    coef = np.zeros((mat.shape[0], 4))
    ts = np.zeros(4)
    rc = lib().orc_material_coefs(_p(mat), ctypes.c_int(mat.shape[0]), ctypes.c_double(f0),
                                  ctypes.c_double(qc), ctypes.c_int(n_sls), _p(coef), _p(ts))
    return rc, coef, ts[:n_sls]


class Acoustic:
    """FP64 acoustic state plus capture buffers; steps with ``run``."""

    def __init__(self, nx, ny, nz, dx, dt, index, mat, f0, qc=1.0, n_sls=2,
                 n_pml=0, pml_R=1e-4):
        self.g = _Grid(nx, ny, nz, dx, dt, n_pml, pml_R, f0, qc, n_sls)
        self.shape = (nz, ny, nx)
        self.index = np.ascontiguousarray(np.asarray(index, dtype=np.uint8).reshape(self.shape))
        self.mat = materials(mat)
        self.n_sls = n_sls
        self.state = np.zeros((n_fields(n_sls),) + self.shape)
        self.peak = np.zeros(self.shape)
        self.dftC = np.zeros(self.shape)
        self.dftS = np.zeros(self.shape)
        self.step = 0
        self.src = None
        self.k_src, self.c0, self.envelope, self.n_cycles = 0, 1500.0, ENV_NONE, 0

    # named views of the state
    FIELDS = ("vx", "vy", "vz", "sxx", "syy", "szz", "sxy", "sxz", "syz")

    def field(self, name):
        return self.state[self.FIELDS.index(name)]

    def memory(self, l, c):
        return self.state[9 + 6 * l + c]

    def pressure(self):
        return -(self.state[3] + self.state[4] + self.state[5]) / 3.0

    def set_source(self, plane, k_src, c0, envelope, n_cycles=0):
        """plane: complex (ny, nx) incident amplitude A e^{i phi}."""
        pl = np.asarray(plane, dtype=np.complex128).reshape(self.shape[1:])
        self.src = np.ascontiguousarray(np.stack([pl.real, pl.imag], axis=-1))
        self.k_src, self.c0, self.envelope, self.n_cycles = k_src, c0, envelope, n_cycles

    def run(self, n_steps, peak_from=0, dft_start=0, dft_steps=0, check_cfl=True):
        L = lib()
        src = _p(self.src) if self.src is not None else None
        rc = L.orc_acoustic_run(ctypes.byref(self.g), _p(self.index), _p(self.mat),
                                ctypes.c_int(self.mat.shape[0]), src, ctypes.c_int(self.k_src),
                                ctypes.c_double(self.c0), ctypes.c_int(self.envelope),
                                ctypes.c_int(self.n_cycles), ctypes.c_int(self.step),
                                ctypes.c_int(n_steps), ctypes.c_int(peak_from),
                                ctypes.c_int(dft_start), ctypes.c_int(dft_steps),
                                ctypes.c_int(1 if check_cfl else 0), _p(self.state),
                                _p(self.peak), _p(self.dftC), _p(self.dftS))
        if rc == 0:
            self.step += n_steps
        return rc

    def amp_phase(self, n_samples):
        amp = np.zeros(self.shape)
        ph = np.zeros(self.shape)
        lib().orc_amp_phase(_p(self.dftC), _p(self.dftS), ctypes.c_size_t(amp.size),
                            ctypes.c_int(n_samples), _p(amp), _p(ph))
        return amp, ph


def bowl_elements(aperture, roc, apex, direction, lam, ds_over_lambda=0.25):
    apex = np.asarray(apex, dtype=np.float64)
    d = np.asarray(direction, dtype=np.float64)
    n = lib().orc_bowl_elements(ctypes.c_double(aperture), ctypes.c_double(roc), _p(apex), _p(d),
                                ctypes.c_double(lam), ctypes.c_double(ds_over_lambda), None)
    out = np.zeros((n, 4))
    lib().orc_bowl_elements(ctypes.c_double(aperture), ctypes.c_double(roc), _p(apex), _p(d),
                            ctypes.c_double(lam), ctypes.c_double(ds_over_lambda), _p(out))
    return out


def rs_plane(aperture, roc, apex, direction, nx, ny, dx, z_plane, f0, c0, p0,
             ds_over_lambda=0.25):
    """Complex (ny, nx) Rayleigh-Sommerfeld pressure on the plane z = z_plane."""
    apex = np.asarray(apex, dtype=np.float64)
    d = np.asarray(direction, dtype=np.float64)
    out = np.zeros((ny, nx, 2))
    rc = lib().orc_rs_plane(ctypes.c_double(aperture), ctypes.c_double(roc), _p(apex), _p(d),
                            ctypes.c_double(ds_over_lambda), ctypes.c_int(nx), ctypes.c_int(ny),
                            ctypes.c_double(dx), ctypes.c_double(z_plane), ctypes.c_double(f0),
                            ctypes.c_double(c0), ctypes.c_double(p0), _p(out))
    if rc:
        raise ValueError("orc_rs_plane failed: %d" % rc)
    return out[..., 0] + 1j * out[..., 1]


def rs_elements(elements, p0, c0, nx, ny, dx, z_plane, f0):
    """Complex (ny, nx) field of weighted elements, rows (x, y, z, area, w_re, w_im)."""
    el = np.ascontiguousarray(np.asarray(elements, dtype=np.float64).reshape(-1, 6))
    out = np.zeros((ny, nx, 2))
    rc = lib().orc_rs_elements(_p(el), ctypes.c_long(el.shape[0]), ctypes.c_double(p0),
                               ctypes.c_double(c0), ctypes.c_int(nx), ctypes.c_int(ny),
                               ctypes.c_double(dx), ctypes.c_double(z_plane), ctypes.c_double(f0),
                               _p(out))
    if rc:
        raise ValueError("orc_rs_elements failed: %d" % rc)
    return out[..., 0] + 1j * out[..., 1]


def bhte_run(index, mat, dx, amp, p_scale, dt, n_on, n_off, duty, T_a=37.0,
             rhob_cb=1050.0 * 3617.0, T_init=None):
    """Returns (rc, T, Tmax, cem43) as float64 arrays shaped like ``index``."""
    index = np.ascontiguousarray(np.asarray(index, dtype=np.uint8))
    nz, ny, nx = index.shape
    mat = materials(mat)
    T = np.full(index.shape, T_a) if T_init is None else np.array(T_init, dtype=np.float64)
    Tmax = T.copy()
    cem = np.zeros(index.shape)
    a = None if amp is None else np.ascontiguousarray(np.asarray(amp, dtype=np.float64))
    rc = lib().orc_bhte_run(ctypes.c_int(nx), ctypes.c_int(ny), ctypes.c_int(nz),
                            ctypes.c_double(dx), _p(index), _p(mat), ctypes.c_int(mat.shape[0]),
                            _p(a) if a is not None else None, ctypes.c_double(p_scale),
                            ctypes.c_double(dt), ctypes.c_int(n_on), ctypes.c_int(n_off),
                            ctypes.c_double(duty), ctypes.c_double(T_a), ctypes.c_double(rhob_cb),
                            _p(T), _p(Tmax), _p(cem))
    return rc, T, Tmax, cem


def transmission(idx_a, mat_a, amp_a, idx_w, mat_w, amp_w):
    """(E_L, z_m) from Eq. 2."""
    idx_a = np.ascontiguousarray(idx_a, dtype=np.uint8)
    idx_w = np.ascontiguousarray(idx_w, dtype=np.uint8)
    amp_a = np.ascontiguousarray(amp_a, dtype=np.float64)
    amp_w = np.ascontiguousarray(amp_w, dtype=np.float64)
    mat_a, mat_w = materials(mat_a), materials(mat_w)
    nz, ny, nx = idx_a.shape
    el = ctypes.c_double(0)
    zm = ctypes.c_int(0)
    rc = lib().orc_transmission(ctypes.c_int(nx), ctypes.c_int(ny), ctypes.c_int(nz),
                                _p(idx_a), _p(mat_a), _p(amp_a), _p(idx_w), _p(mat_w), _p(amp_w),
                                ctypes.byref(el), ctypes.byref(zm))
    if rc:
        raise ValueError("orc_transmission failed: %d" % rc)
    return el.value, zm.value
