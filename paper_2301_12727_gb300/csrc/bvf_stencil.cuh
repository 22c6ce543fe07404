// Arithmetic shared by the acoustic kernels: O(4) staggered differences
// (Sec. 2.3), CPML recursion, and the Crank-Nicolson update of the SLS
// memory variables (Sec. 3.2).
//
// Every per-voxel operation is written once, for V = float (one voxel) and
// V = float2 (two x-adjacent voxels, on the packed FP32x2 add / multiply /
// fused multiply-add of sm_100 and later).  Each operation rounds to nearest
// exactly once and nothing is left for the compiler to contract, so the
// paired TMA kernels and the single-voxel direct kernels produce the same
// bits.
#pragma once

#include <cuda_fp16.h>

#include "bvf_internal.cuh"

namespace bvf {
namespace st {

// ---- explicitly rounded FP32 arithmetic, one voxel or a pair ---------------
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b)
{
    const unsigned long long ra = *reinterpret_cast<const unsigned long long *>(&a);
    const unsigned long long rb = *reinterpret_cast<const unsigned long long *>(&b);
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(ra), "l"(rb));
    return *reinterpret_cast<const float2 *>(&r);
}
template <class V>
__device__ __forceinline__ V splat(float s);
template <>
__device__ __forceinline__ float splat<float>(float s) { return s; }
template <>
__device__ __forceinline__ float2 splat<float2>(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 pair(float a, float b) { return make_float2(a, b); }

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
__device__ __forceinline__ void st2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
__device__ __forceinline__ void st2(__half *p, float2 v)
{
    *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(v.x, v.y);
}
// a pair whose second element is the ghost of its axis: only the first is stored
template <typename T>
__device__ __forceinline__ void st2_or_1(T *p, float2 v, bool both)
{
    if (both)
        st2(p, v);
    else
        stv(p, v.x);
}

constexpr float kC1 = 1.125f;            // 9/8
constexpr float kC2 = -1.0f / 24.0f;     // -1/24

// Difference coefficients with 1/dx folded in.
struct Dx {
    float c1, c2;
};
__device__ __forceinline__ Dx make_dx(float inv_dx) { return Dx{kC1 * inv_dx, kC2 * inv_dx}; }

// D+ : integer-point field -> derivative at s + 1/2
template <class V>
__device__ __forceinline__ V dfw(V fm1, V f0, V f1, V f2, Dx d)
{
    return vfma(splat<V>(d.c2), vsub(f2, fm1), vmul(splat<V>(d.c1), vsub(f1, f0)));
}
// D- : half-point field -> derivative at s
template <class V>
__device__ __forceinline__ V dbw(V fm2, V fm1, V f0, V f1, Dx d)
{
    return vfma(splat<V>(d.c2), vsub(f1, fm2), vmul(splat<V>(d.c1), vsub(f0, fm1)));
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

// CPML recursion psi <- b psi + a d on the old memory `old`; `neu` receives
// the new memory and the derivative used, d + psi, is returned.
template <class V>
__device__ __forceinline__ V cpml_v(V old, V a, V b, V d, V &neu)
{
    neu = vfma(a, d, vmul(b, old));
    return vadd(d, neu);
}
// the same with the memory in global memory (direct kernels)
__device__ __forceinline__ float cpml(float *__restrict__ psi, float2 ab, float d)
{
    float neu;
    const float r = cpml_v(*psi, ab.x, ab.y, d, neu);
    *psi = neu;
    return r;
}
__device__ __forceinline__ float cpml_pre(float *__restrict__ psi, float old, float2 ab, float d)
{
    float neu;
    const float r = cpml_v(old, ab.x, ab.y, d, neu);
    *psi = neu;
    return r;
}

// Memory variables of one stress component:
// r_l <- ca_l r_l + ncb_l Theta (ncb_l = -cb_l); returns sum_l (r_l^{n+1} + r_l^n).
template <int L, class V>
__device__ __forceinline__ V sls_update(const AcParams &p, V (&rv)[L > 0 ? L : 1][6], int c, V The)
{
    V sum = splat<V>(0.0f);
#pragma unroll
    for (int l = 0; l < L; ++l) {
        const V r0 = rv[l][c];
        const V rn = vfma(splat<V>(p.ca[l]), r0, vmul(splat<V>(p.ncb[l]), The));
        const V s = vadd(rn, r0);
        sum = (l == 0) ? s : vadd(sum, s);
        rv[l][c] = rn;
    }
    return sum;
}

// stress increment of one component: sigma + dt (Psi + rh sum_l(...))
template <int L, class V>
__device__ __forceinline__ V stress_step(const AcParams &p, V sv, V Psi, V The,
                                         V (&rv)[L > 0 ? L : 1][6], int c)
{
    V upd = Psi;
    if constexpr (L > 0) upd = vfma(splat<V>(p.rh), sls_update<L, V>(p, rv, c, The), Psi);
    return vfma(splat<V>(p.dt), upd, sv);
}

// ---- per-voxel updates shared by the direct and the TMA-fed kernels -------

// velocity u + dt b (d1 + d2 + d3) with the buoyancy b of the two cells'
// materials from the pair table (FP64-derived)
template <class V>
__device__ __forceinline__ V vel_step(float dt, V b, V u, V d1, V d2, V d3)
{
    return vfma(vmul(splat<V>(dt), b), vadd(vadd(d1, d2), d3), u);
}
__device__ __forceinline__ float buoyancy(const float *buoy, int n_mat, int ma, int mb)
{
    return __ldg(buoy + ma * n_mat + mb);
}

// Per-material coefficients as the stress kernels hold them in shared memory.
// Normal stress: Psi = piU th - mu2U (th - e_ii), Theta = piT th - mu2T (th - e_ii),
// held with the negated shear terms nmu2U = -mu2U, nmu2T = -mu2T.
// psiS/theS are the shear coefficients of a shear point whose four cells are
// all this material, computed with exactly the operations of the general
// four-cell path below, so taking them is bit-identical to that path.
struct alignas(16) StressCoef {
    float piU, piT, nmu2U, nmu2T;
    float inv_mu, tauS;    // adjacent: one 8-byte load
    float psiS, theS;
};

__device__ __forceinline__ float shear_mu(float2 a, float2 b, float2 d, float2 f)
{
    return __fmul_rn(4.0f, __frcp_rn(__fadd_rn(__fadd_rn(a.x, b.x), __fadd_rn(d.x, f.x))));
}
__device__ __forceinline__ float shear_tau(float2 a, float2 b, float2 d, float2 f)
{
    return __fmul_rn(0.25f, __fadd_rn(__fadd_rn(a.y, b.y), __fadd_rn(d.y, f.y)));
}

__device__ __forceinline__ StressCoef make_stress_coef(const MatCoef &m, float Lf)
{
    StressCoef c;
    c.piU = m.piU;
    c.piT = m.piT;
    c.nmu2U = -m.mu2U;
    c.nmu2T = -m.mu2T;
    c.inv_mu = m.inv_mu;
    c.tauS = m.tauS;
    const float2 q = make_float2(m.inv_mu, m.tauS);
    const float muh = shear_mu(q, q, q, q), tsh = shear_tau(q, q, q, q);
    c.psiS = __fmul_rn(muh, __fmaf_rn(Lf, tsh, 1.0f));
    c.theS = __fmul_rn(muh, tsh);
    return c;
}

// (inv_mu, tauS) of a table entry as one 8-byte load
__device__ __forceinline__ float2 shear_pair(const StressCoef *lut, int m)
{
    return *reinterpret_cast<const float2 *>(&lut[m].inv_mu);
}

// Shear coefficients (Psi / strain, Theta / strain) at a shear point with
// cells m00, mb (first-axis pair) and md, mf (second): harmonic-mean mu, mean
// tau_S, pairs along the first axis summed first (mirror symmetry).  One
// material in all four cells takes the per-material constants.
__device__ __forceinline__ void shear_coef(const StressCoef *lut, const StressCoef &c0, int m00,
                                           int mb, int md, int mf, float Lf, float &psic,
                                           float &thec)
{
    if (mb == m00 && md == m00 && mf == m00) {
        psic = c0.psiS;
        thec = c0.theS;
    } else {
        const float2 a = make_float2(c0.inv_mu, c0.tauS), b = shear_pair(lut, mb);
        const float2 d = shear_pair(lut, md), f = shear_pair(lut, mf);
        const float muh = shear_mu(a, b, d, f), tsh = shear_tau(a, b, d, f);
        psic = __fmul_rn(muh, __fmaf_rn(Lf, tsh, 1.0f));
        thec = __fmul_rn(muh, tsh);
    }
}

// normal stresses + their memory variables at one voxel or pair (the source,
// already scaled, is subtracted from each normal stress); coefficients per
// lane: piU, piT, nmu2U, nmu2T
template <int L, class V>
__device__ __forceinline__ void normal_update(const AcParams &p, V piU, V piT, V nmu2U, V nmu2T,
                                              V exx, V eyy, V ezz, V srcv, V (&sv)[6],
                                              V (&rv)[L > 0 ? L : 1][6])
{
    const V th = vadd(vadd(exx, eyy), ezz);
    const V ev[3] = {exx, eyy, ezz};
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
        const V dev = vsub(th, ev[cc]);
        const V Psi = vfma(piU, th, vmul(nmu2U, dev));
        const V The = vfma(piT, th, vmul(nmu2T, dev));
        sv[cc] = vsub(stress_step<L, V>(p, sv[cc], Psi, The, rv, cc), srcv);
    }
}
template <int L>
__device__ __forceinline__ void normal_update(const AcParams &p, const StressCoef &c0, float exx,
                                              float eyy, float ezz, float srcv, float (&sv)[6],
                                              float (&rv)[L > 0 ? L : 1][6])
{
    normal_update<L, float>(p, c0.piU, c0.piT, c0.nmu2U, c0.nmu2T, exx, eyy, ezz, srcv, sv, rv);
}

// scaled source value of a voxel: src_scale (A_re ws + A_im wc)
template <class V>
__device__ __forceinline__ V source_value(float scale, V re, V im, float ws, float wc)
{
    return vmul(splat<V>(scale), vfma(re, splat<V>(ws), vmul(im, splat<V>(wc))));
}

// p = -(sxx + syy + szz) / 3
template <class V>
__device__ __forceinline__ V pressure(const V (&sv)[6])
{
    return vmul(vadd(vadd(sv[0], sv[1]), sv[2]), splat<V>(-1.0f / 3.0f));
}

// shear stress cc from its strain e and the point's coefficients
template <int L, class V>
__device__ __forceinline__ void shear_update(const AcParams &p, V psic, V thec, V e, int cc,
                                             V (&sv)[6], V (&rv)[L > 0 ? L : 1][6])
{
    sv[cc] = stress_step<L, V>(p, sv[cc], vmul(psic, e), vmul(thec, e), rv, cc);
}
template <int L>
__device__ __forceinline__ void shear_update(const AcParams &p, const StressCoef *lut,
                                             const StressCoef &c0, int m00, int mb, int md, int mf,
                                             float e, int cc, float (&sv)[6],
                                             float (&rv)[L > 0 ? L : 1][6])
{
    float psic, thec;
    shear_coef(lut, c0, m00, mb, md, mf, p.Lf, psic, thec);
    shear_update<L, float>(p, psic, thec, e, cc, sv, rv);
}

}  // namespace st
}  // namespace bvf
