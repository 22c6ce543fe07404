// Arithmetic shared by the acoustic kernels: O(4) staggered differences
// (Sec. 2.3), CPML recursion, and the Crank-Nicolson update of the SLS
// memory variables (Sec. 3.2).
#pragma once

#include "bvf_internal.cuh"

namespace bvf {
namespace st {

constexpr float kC1 = 1.125f;            // 9/8
constexpr float kC2 = -1.0f / 24.0f;     // -1/24

// D+ : integer-point field -> derivative at s + 1/2
__device__ __forceinline__ float dfw(float fm1, float f0, float f1, float f2, float ix)
{
    return fmaf(kC2, f2 - fm1, kC1 * (f1 - f0)) * ix;
}
// D- : half-point field -> derivative at s
__device__ __forceinline__ float dbw(float fm2, float fm1, float f0, float f1, float ix)
{
    return fmaf(kC2, f1 - fm2, kC1 * (f0 - fm1)) * ix;
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

// velocity increment dt b (d1 + d2 + d3), buoyancy b = 2 / (rho_a + rho_b)
__device__ __forceinline__ float vel_increment(float dt, float rho_a, float rho_b, float d1,
                                               float d2, float d3)
{
    return dt * (2.0f * __frcp_rn(rho_a + rho_b)) * (d1 + d2 + d3);
}

// normal stresses + their memory variables at one voxel (the source, already
// scaled, is subtracted from each normal stress)
template <int L>
__device__ __forceinline__ void normal_update(const AcParams &p, const MatCoef &c0, float exx,
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
        float v = sv[cc] + p.dt * (Psi + 0.5f * sum);
        v -= srcv;
        sv[cc] = v;
    }
}

// p = -(sxx + syy + szz) / 3
__device__ __forceinline__ float pressure(const float (&sv)[6])
{
    return -(sv[0] + sv[1] + sv[2]) * (1.0f / 3.0f);
}

// shear stress cc at a shear point whose four cells carry (inv_mu, tauS) in
// a, b (first axis pair) and d, f (second); harmonic-mean mu, mean tau_S,
// pairs along the first axis summed first (mirror symmetry)
template <int L>
__device__ __forceinline__ void shear_update(const AcParams &p, float2 a, float2 b, float2 d,
                                             float2 f, float e, int cc, float (&sv)[6],
                                             float (&rv)[L > 0 ? L : 1][6])
{
    const float muh = 4.0f * __frcp_rn((a.x + b.x) + (d.x + f.x));
    const float tsh = 0.25f * ((a.y + b.y) + (d.y + f.y));
    const float Psi = muh * (1.0f + p.Lf * tsh) * e;
    const float The = muh * tsh * e;
    const float sum = sls_update<L>(p, rv, cc, The);
    sv[cc] += p.dt * (Psi + 0.5f * sum);
}

// (inv_mu, tauS) of a table entry as one 8-byte load
__device__ __forceinline__ float2 shear_pair(const MatCoef *lut, int m)
{
    return *reinterpret_cast<const float2 *>(&lut[m].inv_mu);
}

}  // namespace st
}  // namespace bvf
