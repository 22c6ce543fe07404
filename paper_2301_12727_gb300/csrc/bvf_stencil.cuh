// Arithmetic shared by the acoustic kernels: O(4) staggered differences
// (Sec. 2.3), CPML recursion, and the Crank-Nicolson update of the SLS
// memory variables (Sec. 3.2).
#pragma once

#include <cuda_fp16.h>

#include "bvf_internal.cuh"

namespace bvf {
namespace st {

// State storage: float, or scaled FP16 converted to FP32 on load and rounded
// to nearest on store.
__device__ __forceinline__ float tof(float v) { return v; }
__device__ __forceinline__ float tof(__half v) { return __half2float(v); }
__device__ __forceinline__ void stv(float *p, float v) { *p = v; }
__device__ __forceinline__ void stv(__half *p, float v) { *p = __float2half_rn(v); }
// two neighbouring elements (x, x+1) at an even element offset
__device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ float2 ld2(const __half *p)
{
    return __half22float2(*reinterpret_cast<const __half2 *>(p));
}
__device__ __forceinline__ void st2(float *p, float a, float b)
{
    *reinterpret_cast<float2 *>(p) = make_float2(a, b);
}
__device__ __forceinline__ void st2(__half *p, float a, float b)
{
    *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(a, b);
}

constexpr float kC1 = 1.125f;            // 9/8
constexpr float kC2 = -1.0f / 24.0f;     // -1/24

// Difference coefficients with 1/dx folded in.
struct Dx {
    float c1, c2;
};
__device__ __forceinline__ Dx make_dx(float inv_dx) { return Dx{kC1 * inv_dx, kC2 * inv_dx}; }

// D+ : integer-point field -> derivative at s + 1/2
__device__ __forceinline__ float dfw(float fm1, float f0, float f1, float f2, Dx d)
{
    return fmaf(d.c2, f2 - fm1, d.c1 * (f1 - f0));
}
// D- : half-point field -> derivative at s
__device__ __forceinline__ float dbw(float fm2, float fm1, float f0, float f1, Dx d)
{
    return fmaf(d.c2, f1 - fm2, d.c1 * (f0 - fm1));
}

// position of coordinate c in its axis' CPML slab (-1 outside):
// [0, P) on the low side, [n-P-1, n) on the high side.
__device__ __forceinline__ int slab_pos(int c, int n, int P)
{
    if (P <= 0) return -1;
    if (c < P) return c;
    if (c >= n - P - 1) return c - (n - P - 1) + P;
    return -1;
}

// CPML recursion psi <- b psi + a d; the derivative used is d + psi.
__device__ __forceinline__ float cpml(float *__restrict__ psi, float2 ab, float d)
{
    const float v = fmaf(ab.x, d, ab.y * *psi);
    *psi = v;
    return d + v;
}

// The same recursion with psi already loaded (old): lets a kernel issue the
// loads of all its CPML memories at once, ahead of the derivatives.
__device__ __forceinline__ float cpml_pre(float *__restrict__ psi, float old, float2 ab, float d)
{
    const float v = fmaf(ab.x, d, ab.y * old);
    *psi = v;
    return d + v;
}

// Memory variables of one stress component, on registers:
// r_l <- ca_l r_l - cb_l Theta ; returns sum_l (r_l^{n+1} + r_l^n).
template <int L>
__device__ __forceinline__ float sls_update(const AcParams &p, float (&rv)[L > 0 ? L : 1][6],
                                            int c, float The)
{
    float sum = 0.0f;
#pragma unroll
    for (int l = 0; l < L; ++l) {
        const float r0 = rv[l][c];
        const float rn = p.ca[l] * r0 - p.cb[l] * The;
        sum += rn + r0;
        rv[l][c] = rn;
    }
    return sum;
}

// ---- per-voxel updates shared by the direct and the TMA-fed kernels -------

// velocity increment dt b (d1 + d2 + d3) with the buoyancy b of the two
// cells' materials from the pair table (FP64-derived, one load)
__device__ __forceinline__ float vel_increment(float dt, const float *buoy, int n_mat, int ma,
                                               int mb, float d1, float d2, float d3)
{
    return dt * __ldg(buoy + ma * n_mat + mb) * (d1 + d2 + d3);
}

// Per-material coefficients as the stress kernels hold them in shared memory.
// psiS/theS are the shear coefficients of a shear point whose four cells are
// all this material, computed with exactly the operations of the general
// four-cell path below, so taking them is bit-identical to that path.
struct alignas(16) StressCoef {
    float piU, piT, mu2U, mu2T;
    float inv_mu, tauS;    // adjacent: one 8-byte load
    float psiS, theS;
};

__device__ __forceinline__ float shear_mu(float2 a, float2 b, float2 d, float2 f)
{
    return 4.0f * __frcp_rn((a.x + b.x) + (d.x + f.x));
}
__device__ __forceinline__ float shear_tau(float2 a, float2 b, float2 d, float2 f)
{
    return 0.25f * ((a.y + b.y) + (d.y + f.y));
}

__device__ __forceinline__ StressCoef make_stress_coef(const MatCoef &m, float Lf)
{
    StressCoef c;
    c.piU = m.piU;
    c.piT = m.piT;
    c.mu2U = m.mu2U;
    c.mu2T = m.mu2T;
    c.inv_mu = m.inv_mu;
    c.tauS = m.tauS;
    const float2 q = make_float2(m.inv_mu, m.tauS);
    const float muh = shear_mu(q, q, q, q), tsh = shear_tau(q, q, q, q);
    c.psiS = muh * fmaf(Lf, tsh, 1.0f);
    c.theS = muh * tsh;
    return c;
}

// (inv_mu, tauS) of a table entry as one 8-byte load
__device__ __forceinline__ float2 shear_pair(const StressCoef *lut, int m)
{
    return *reinterpret_cast<const float2 *>(&lut[m].inv_mu);
}

// normal stresses + their memory variables at one voxel (the source, already
// scaled, is subtracted from each normal stress)
template <int L>
__device__ __forceinline__ void normal_update(const AcParams &p, const StressCoef &c0, float exx,
                                              float eyy, float ezz, float srcv, float (&sv)[6],
                                              float (&rv)[L > 0 ? L : 1][6])
{
    const float th = exx + eyy + ezz;
    const float ev[3] = {exx, eyy, ezz};
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
        const float dev = th - ev[cc];
        const float Psi = c0.piU * th - c0.mu2U * dev;
        const float The = c0.piT * th - c0.mu2T * dev;
        const float sum = sls_update<L>(p, rv, cc, The);
        float v = sv[cc] + p.dt * (Psi + p.rh * sum);
        v -= srcv;
        sv[cc] = v;
    }
}

// p = -(sxx + syy + szz) / 3
__device__ __forceinline__ float pressure(const float (&sv)[6])
{
    return -(sv[0] + sv[1] + sv[2]) * (1.0f / 3.0f);
}

// shear stress cc at a shear point with cells m00, mb (first-axis pair) and
// md, mf (second): harmonic-mean mu, mean tau_S, pairs along the first axis
// summed first (mirror symmetry).  One material in all four cells takes the
// per-material constants.
template <int L>
__device__ __forceinline__ void shear_update(const AcParams &p, const StressCoef *lut,
                                             const StressCoef &c0, int m00, int mb, int md, int mf,
                                             float e, int cc, float (&sv)[6],
                                             float (&rv)[L > 0 ? L : 1][6])
{
    float psic, thec;
    if (mb == m00 && md == m00 && mf == m00) {
        psic = c0.psiS;
        thec = c0.theS;
    } else {
        const float2 a = make_float2(c0.inv_mu, c0.tauS), b = shear_pair(lut, mb);
        const float2 d = shear_pair(lut, md), f = shear_pair(lut, mf);
        const float muh = shear_mu(a, b, d, f), tsh = shear_tau(a, b, d, f);
        psic = muh * fmaf(p.Lf, tsh, 1.0f);
        thec = muh * tsh;
    }
    const float Psi = psic * e;
    const float The = thec * e;
    const float sum = sls_update<L>(p, rv, cc, The);
    sv[cc] += p.dt * (Psi + p.rh * sum);
}

}  // namespace st
}  // namespace bvf
