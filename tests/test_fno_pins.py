"""Pins of the FP64 surrogate oracle (oracle/fno.py) against brute force sums
and closed forms that do not go through numpy's FFT: the truncated spectral
convolution of a Fourier layer, the pass-through of single Fourier modes, the
circular-shift equivariance of the whole network, its reduction to a plain MLP
on constant fields, and the GELU activation against the tabulated normal CDF."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import fno


def _signed(j, m):
    return j if j < m else j - 2 * m


def brute_spectral_conv(v, R, m):
    """Truncated forward DFT, mode mixing and the real inverse written as
    explicit sums over the grid and the kept modes."""
    c, nz, ny, nx = v.shape
    z = np.arange(nz)[:, None, None]
    y = np.arange(ny)[None, :, None]
    x = np.arange(nx)[None, None, :]
    n = nz * ny * nx
    out = np.zeros((R.shape[4], nz, ny, nx))
    for jz in range(2 * m):
        for jy in range(2 * m):
            for kx in range(m):
                ph = 2 * np.pi * (_signed(jz, m) * z / nz + _signed(jy, m) * y / ny + kx * x / nx)
                e = np.exp(-1j * ph)
                F = np.array([(v[ci] * e).sum() for ci in range(c)])
                G = R[jz, jy, kx].T @ F                      # sum over c of R[.., c, o] F[c]
                weight = 1.0 if kx == 0 else 2.0
                for o in range(R.shape[4]):
                    out[o] += weight * np.real(G[o] * np.exp(1j * ph)) / n
    return out


def _rand_R(rng, m, ci, co):
    return rng.standard_normal((2 * m, 2 * m, m, ci, co)) + 1j * rng.standard_normal(
        (2 * m, 2 * m, m, ci, co))


@pytest.mark.parametrize("shape,m", [((5, 6, 7), 2), ((4, 4, 6), 2), ((6, 8, 4), 1)])
def test_spectral_conv_matches_brute_force_sums(shape, m):
    rng = np.random.default_rng(11)
    v = rng.standard_normal((3,) + shape)
    R = _rand_R(rng, m, 3, 2)
    got = fno.spectral_conv(v, R, m)
    ref = brute_spectral_conv(v, R, m)
    assert got.shape == ref.shape
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def _cos_mode(shape, a, b, c):
    nz, ny, nx = shape
    z = np.arange(nz)[:, None, None]
    y = np.arange(ny)[None, :, None]
    x = np.arange(nx)[None, None, :]
    th = 2 * np.pi * (a * z / nz + b * y / ny + c * x / nx)
    return np.cos(th), np.sin(th)


@pytest.mark.parametrize("abc,frac", [((1, -1, 1), 1.0), ((0, 1, 0), 1.0), ((-2, 0, 1), 1.0),
                                      ((0, 0, 3), 0.0), ((4, 0, 0), 0.0), ((1, 3, 1), 0.0),
                                      ((3, 0, 0), 0.5), ((0, -3, 0), 0.5), ((-3, 2, 2), 1.0)])
def test_single_mode_passes_through_identity_weights(abc, frac):
    """Kept slots have signed frequencies -m .. m-1 on y and z.  A kx >= 1 mode
    is one half-spectrum bin (kept or not); on the kx = 0 plane cos carries
    the bins k and -k, and with |k| = m only -m is kept, so half passes."""
    shape, m = (8, 8, 8), 3
    cth, sth = _cos_mode(shape, *abc)
    v = cth[None]
    one = np.ones((2 * m, 2 * m, m, 1, 1), dtype=complex)
    got = fno.spectral_conv(v, one, m)[0]
    np.testing.assert_allclose(got, frac * cth, atol=1e-12)
    # R = i: a kx >= 1 mode turns cos into -sin; on the kx = 0 plane each bin
    # pair contributes Re(i e^{i th}) + Re(i e^{-i th}) = 0, a lone -m bin
    # Re(i e^{-i th})/2 = sin(th)/2 with th the phase of +k
    got_i = fno.spectral_conv(v, 1j * one, m)[0]
    if frac == 0.0:
        expect = 0.0 * sth
    elif abc[2] != 0:
        expect = -sth
    elif frac == 1.0:
        expect = 0.0 * sth
    else:
        # the kept bin is the negative one of the pair (+m is not a slot)
        sgn = 1.0 if (abc[0] == m or abc[1] == m) else -1.0
        expect = 0.5 * sgn * sth
    np.testing.assert_allclose(got_i, expect, atol=1e-12)


DIMS = dict(c_in=3, width=4, modes=2, n_layers=3, hidden=6, c_out=2)


def _weights(rng, scale=0.5):
    return scale * rng.standard_normal(fno.weight_count(**DIMS))


def test_network_is_equivariant_to_circular_shifts():
    rng = np.random.default_rng(5)
    w = _weights(rng)
    a = rng.standard_normal((DIMS["c_in"], 6, 5, 8))
    u = fno.forward(a, w, **DIMS)
    shift = (2, -1, 3)
    u_s = fno.forward(np.roll(a, shift, axis=(1, 2, 3)), w, **DIMS)
    np.testing.assert_allclose(u_s, np.roll(u, shift, axis=(1, 2, 3)), atol=1e-12)


def test_constant_field_reduces_to_mlp():
    """On a constant field only the DC mode is non-zero: each Fourier layer is
    then sigma((W + Re R_000^T) v + b)."""
    rng = np.random.default_rng(8)
    w = _weights(rng)
    p = fno.unpack(w, **DIMS)
    a0 = rng.standard_normal(DIMS["c_in"])
    a = np.broadcast_to(a0[:, None, None, None], (DIMS["c_in"], 4, 6, 4)).copy()
    got = fno.forward(a, w, **DIMS)

    def phi(t):  # normal CDF from its series-free closed form via erfc
        from math import erfc, sqrt
        return np.array([0.5 * erfc(-ti / sqrt(2.0)) for ti in np.atleast_1d(t)])

    def act(t):
        return t * phi(t)

    v = p["Wp"] @ a0 + p["bp"]
    for l, lay in enumerate(p["layers"]):
        s = (lay["W"] + np.real(lay["R"][0, 0, 0]).T) @ v + lay["b"]
        v = act(s) if l < DIMS["n_layers"] - 1 else s
    u = p["Q2"] @ act(p["Q1"] @ v + p["q1"]) + p["q2"]
    np.testing.assert_allclose(got, np.broadcast_to(u[:, None, None, None], got.shape),
                               rtol=1e-12, atol=1e-12)


def test_gelu_identities_and_table_values():
    x = np.linspace(-4, 4, 33)
    np.testing.assert_allclose(fno.gelu(x) - fno.gelu(-x), x, atol=1e-15)
    assert fno.gelu(0.0) == 0.0
    # standard normal CDF table: Phi(1) = 0.8413447461, Phi(2) = 0.9772498681
    np.testing.assert_allclose(fno.gelu(1.0), 0.8413447460685429, rtol=1e-13)
    np.testing.assert_allclose(fno.gelu(2.0), 2 * 0.9772498680518208, rtol=1e-13)
    np.testing.assert_allclose(fno.gelu(-1.0), -(1 - 0.8413447460685429), rtol=1e-12)


def test_weight_layout_round_trip():
    n = fno.weight_count(**DIMS)
    m3 = (2 * DIMS["modes"]) ** 2 * DIMS["modes"]
    w_, c_in, h, co = DIMS["width"], DIMS["c_in"], DIMS["hidden"], DIMS["c_out"]
    assert n == w_ * c_in + w_ + DIMS["n_layers"] * (2 * m3 * w_ * w_ + w_ * w_ + w_) \
        + h * w_ + h + co * h + co
    blob = np.arange(n, dtype=np.float64)
    p = fno.unpack(blob, **DIMS)
    assert p["Wp"][1, 2] == 1 * c_in + 2
    lay0 = p["layers"][0]
    base = w_ * c_in + w_
    # R_0[jz=1][jy=0][kx=1][ci=2][co=3] = (re, im) at consecutive positions
    off = base + ((((1 * 2 * DIMS["modes"] + 0) * DIMS["modes"] + 1) * w_ + 2) * w_ + 3) * 2
    assert lay0["R"][1, 0, 1, 2, 3] == off + 1j * (off + 1)
    assert p["q2"][-1] == n - 1
    with pytest.raises(ValueError):
        fno.unpack(blob[:-1], **DIMS)


def test_features_of_a_water_voxel_and_the_source_plane():
    table = np.array([[1000.0, 1500.0, 0, 0.0, 0, 0.6, 4180, 0, 0],
                      [1900.0, 2800.0, 0, 200.0, 0, 0.3, 1300, 0, 0]])
    idx = np.zeros((5, 4, 6), dtype=np.int32)
    idx[2, 1, 3] = 1
    src = np.zeros((4, 6), complex)
    src[1, 2] = 3.0 - 4.0j
    f = fno.features(idx, table, table[0], 5e5, 1, src, 2.0)
    assert f.shape == (fno.N_FEATURES, 5, 4, 6)
    assert f[0, 0, 0, 0] == 0.0 and f[1, 0, 0, 0] == 0.0 and f[2, 0, 0, 0] == 0.0
    np.testing.assert_allclose(f[:3, 2, 1, 3], [2800 / 1500 - 1, 0.9, 200 * 1500 / 5e5])
    assert f[3, 1, 1, 2] == 1.5 and f[4, 1, 1, 2] == -2.0
    assert np.count_nonzero(f[3]) == 1 and np.count_nonzero(f[4]) == 1
    np.testing.assert_allclose(f[5, 0, 0, :], (np.arange(6) + 0.5) / 6)
    np.testing.assert_allclose(f[7, :, 0, 0], (np.arange(5) + 0.5) / 5)


def test_identity_weights_give_a_symmetric_band_filter():
    """With R = 1 on every kept mode the spectral convolution passes a field
    band-limited to |ky|, |kz| < m, kx < m unchanged, and its kernel
    sum cos(k.(x - x')) / N is symmetric: <K n, u> = <n, K u> for any fields.
    The lone -m bins of the kx = 0 plane pass half their pair, so K is a
    contraction but not a projection there."""
    rng = np.random.default_rng(12)
    m = 2
    shape = (9, 10, 12)
    # a field band-limited to |kz|, |ky| < m, 0 <= kx < m: no content at |k| = m
    nz, ny, nx = shape
    z = np.arange(nz)[:, None, None] / nz
    y = np.arange(ny)[None, :, None] / ny
    x = np.arange(nx)[None, None, :] / nx
    u = np.zeros(shape)
    for a in range(-(m - 1), m):
        for b in range(-(m - 1), m):
            for c in range(m):
                u += rng.standard_normal() * np.cos(2 * np.pi * (a * z + b * y + c * x)
                                                    + rng.uniform(0, 2 * np.pi))
    noise = rng.standard_normal(shape)
    one = np.ones((2 * m, 2 * m, m, 1, 1), dtype=complex)
    Kn = fno.spectral_conv(noise[None], one, m)[0]
    Ku = fno.spectral_conv(u[None], one, m)[0]
    np.testing.assert_allclose(Ku, u, atol=1e-12 * np.abs(u).max())     # band passes unchanged
    KKn = fno.spectral_conv(Kn[None], one, m)[0]
    # idempotent on the part of the band without the lone -m bins
    w = rng.standard_normal(shape)
    Kw = fno.spectral_conv(w[None], one, m)[0]
    np.testing.assert_allclose(np.sum(Kn * u), np.sum(noise * Ku), rtol=1e-10)   # <Kn, u> = <n, Ku>
    np.testing.assert_allclose(np.sum(Kn * w), np.sum(noise * Kw), rtol=1e-10)   # self-adjoint
    assert np.linalg.norm(KKn - Kn) <= np.linalg.norm(Kn)                        # contraction
