"""FP64 oracle of the Fourier-neural-operator surrogate of the acoustic solve.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``): the product
library never imports it, and it shares no code with the CUDA path.

The surrogate replaces the FDTD field of one placement by a learned operator
(the paper's Discussion names machine-learned models as the way to make
planning interactive).  The network is the Fourier neural operator of Li et
al. (ICLR 2021, Sec. 4): a pointwise lift P, L Fourier layers
    v <- sigma(W v + b + K(v)),  K(v) = IFFT(R . FFT(v)) on the kept modes,
with sigma = GELU on all but the last layer, and a two-layer pointwise
projection Q.  Everything here is written from that definition with numpy's
FFT as the only library step; tests/test_fno_pins.py pins it against brute
force sums and closed forms.

Conventions (shared with the CUDA path only through this written definition):
  * fields are channel-major arrays [c][z][y][x] (x fastest);
  * the FFT runs over (z, y, x) with the real-input half spectrum along x;
  * kept modes: kx = 0 .. m-1, and ky, kz in {0 .. m-1} U {-m .. -1}; the
    mode slot j in [0, 2m) of the y or z axis has the signed frequency j for
    j < m and j - 2m otherwise;
  * the inverse is the real inverse FFT of that half spectrum (numpy irfftn):
    the kx = 0 terms contribute their real part once, kx >= 1 twice, all over
    N = nx ny nz; this needs m <= nx/2, 2m <= ny and 2m <= nz.

Flat weight layout (float32 on the product side, float64 here), in order:
  lift      Wp[width][c_in], bp[width]
  layer l   R_l[2m][2m][m][width_in][width_out][2] (re, im),
            W_l[width_out][width_in], b_l[width]
  project   Q1[hidden][width], q1[hidden], Q2[c_out][hidden], q2[c_out]

Feature channels of a placement (c_in = 8), per voxel of material row r and
water row w: c_L/c_L,w - 1, rho/rho_w - 1, alpha_L c_L,w / f0 (nepers per water
wavelength), Re and Im of the source plane / p_norm on plane k_src (zero
elsewhere), and the cell-centre coordinates (i+1/2)/nx, (j+1/2)/ny, (k+1/2)/nz.

Parity status: pinned (brute-force DFT sums on small grids, single-mode
pass-through, circular-shift equivariance, the constant-field reduction to a
plain MLP, GELU identities and the tabulated normal CDF).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

N_FEATURES = 8


def dims_ok(c_in, width, modes, n_layers, hidden, c_out) -> bool:
    return (c_in >= 1 and width >= 1 and modes >= 1 and n_layers >= 1 and hidden >= 1
            and c_out >= 1)


def weight_count(c_in, width, modes, n_layers, hidden, c_out) -> int:
    """Length of the flat weight blob for the layout in the module header."""
    m3 = (2 * modes) * (2 * modes) * modes
    per_layer = m3 * width * width * 2 + width * width + width
    return (width * c_in + width + n_layers * per_layer + hidden * width + hidden
            + c_out * hidden + c_out)


def unpack(w, c_in, width, modes, n_layers, hidden, c_out) -> dict:
    """Split the flat blob into named FP64 arrays (layout of the module header)."""
    w = np.asarray(w, dtype=np.float64)
    if w.size != weight_count(c_in, width, modes, n_layers, hidden, c_out):
        raise ValueError("weight blob has %d values, layout needs %d"
                         % (w.size, weight_count(c_in, width, modes, n_layers, hidden, c_out)))
    pos = 0

    def take(*shape):
        nonlocal pos
        n = int(np.prod(shape))
        a = w[pos:pos + n].reshape(shape)
        pos += n
        return a

    out = {"Wp": take(width, c_in), "bp": take(width), "layers": []}
    m2 = 2 * modes
    for _ in range(n_layers):
        r = take(m2, m2, modes, width, width, 2)
        out["layers"].append({"R": r[..., 0] + 1j * r[..., 1],
                              "W": take(width, width), "b": take(width)})
    out["Q1"] = take(hidden, width)
    out["q1"] = take(hidden)
    out["Q2"] = take(c_out, hidden)
    out["q2"] = take(c_out)
    return out


def gelu(x):
    """GELU(x) = x Phi(x) with the exact normal CDF Phi(x) = (1 + erf(x/sqrt 2))/2."""
    x = np.asarray(x, dtype=np.float64)
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def mode_index(n: int, modes: int) -> np.ndarray:
    """FFT bin of each mode slot j in [0, 2m) of a y or z axis of length n."""
    j = np.arange(2 * modes)
    f = np.where(j < modes, j, j - 2 * modes)
    return np.mod(f, n)


def spectral_conv(v, R, modes):
    """K(v) of one Fourier layer.

    v: [C, nz, ny, nx] real; R: [2m, 2m, m, C_in, C_out] complex.
    Returns [C_out, nz, ny, nx]."""
    v = np.asarray(v, dtype=np.float64)
    c, nz, ny, nx = v.shape
    if not (modes <= nx // 2 and 2 * modes <= ny and 2 * modes <= nz):
        raise ValueError("grid too small for %d modes" % modes)
    vh = np.fft.rfftn(v, axes=(1, 2, 3))                       # [C, nz, ny, nx//2+1]
    iz, iy = mode_index(nz, modes), mode_index(ny, modes)
    kept = vh[:, iz][:, :, iy][:, :, :, :modes]                 # [C, 2m, 2m, m]
    out_k = np.einsum("zykco,czyk->ozyk", R, kept)
    full = np.zeros((R.shape[4], nz, ny, nx // 2 + 1), dtype=np.complex128)
    full[:, iz[:, None], iy[None, :], :modes] = out_k
    return np.fft.irfftn(full, s=(nz, ny, nx), axes=(1, 2, 3))


def forward(a, w, c_in, width, modes, n_layers, hidden, c_out):
    """The surrogate on one feature volume a [c_in, nz, ny, nx] -> [c_out, nz, ny, nx]."""
    a = np.asarray(a, dtype=np.float64)
    p = unpack(w, c_in, width, modes, n_layers, hidden, c_out)
    v = np.einsum("oi,izyx->ozyx", p["Wp"], a) + p["bp"][:, None, None, None]
    for l, lay in enumerate(p["layers"]):
        s = (spectral_conv(v, lay["R"], modes) + np.einsum("oc,czyx->ozyx", lay["W"], v)
             + lay["b"][:, None, None, None])
        v = gelu(s) if l < n_layers - 1 else s
    h = gelu(np.einsum("hc,czyx->hzyx", p["Q1"], v) + p["q1"][:, None, None, None])
    return np.einsum("oh,hzyx->ozyx", p["Q2"], h) + p["q2"][:, None, None, None]


def features(index, table, water_row, f0, k_src, src, p_norm):
    """Feature channels of one placement (definition in the module header).

    index: [nz, ny, nx] material numbers; table: rows (rho, cL, ...) as in the
    solver's material table; water_row: the coupling medium's row; src:
    [ny, nx] complex source plane (Pa)."""
    index = np.asarray(index)
    nz, ny, nx = index.shape
    t = np.asarray(table, dtype=np.float64)
    w = np.asarray(water_row, dtype=np.float64)
    rho, cl, al = t[:, 0][index], t[:, 1][index], t[:, 3][index]
    out = np.zeros((N_FEATURES, nz, ny, nx))
    out[0] = cl / w[1] - 1.0
    out[1] = rho / w[0] - 1.0
    out[2] = al * w[1] / f0
    s = np.asarray(src, dtype=np.complex128) / p_norm
    out[3, k_src] = s.real
    out[4, k_src] = s.imag
    out[5] = ((np.arange(nx) + 0.5) / nx)[None, None, :]
    out[6] = ((np.arange(ny) + 0.5) / ny)[None, :, None]
    out[7] = ((np.arange(nz) + 0.5) / nz)[:, None, None]
    return out
