// Auxiliary kernels: index-range scan, pressure / amplitude-phase read-out,
// Rayleigh-Sommerfeld bowl field (Sec. 2.3), BHTE + CEM43 step (Sec. 2.4),
// and the E_L reductions (Sec. 2.4, Eq. 2).
#include <cuda_fp16.h>

#include "bvf_stencil.cuh"
#include "bvf_tma.cuh"

namespace bvf {

namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(size_t n, int per_block = kThreads, unsigned cap = 152u * 16u)
{
    size_t b = (n + per_block - 1) / per_block;
    return (unsigned)(b < cap ? (b ? b : 1) : cap);
}

__global__ void k_index_max(const uint8_t *__restrict__ idx, size_t n, unsigned *out)
{
    unsigned m = 0;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned)idx[q]);
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

template <typename T>
__global__ void k_pressure(const T *__restrict__ a, const T *__restrict__ b,
                           const T *__restrict__ c, float scale, float *__restrict__ out, size_t n)
{
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x)
        out[q] = -(st::tof(a[q]) + st::tof(b[q]) + st::tof(c[q])) / 3.0f * scale;
}

// state array (element q at f[q * stride]) <-> FP32 values in physical units
// (scale = the storage scale)
template <typename T>
__global__ void k_field_out(const T *__restrict__ f, size_t stride, float scale,
                            float *__restrict__ out, size_t n)
{
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x)
        out[q] = st::tof(f[q * stride]) * scale;
}
template <typename T>
__global__ void k_field_in(const float *__restrict__ in, size_t stride, float inv_scale,
                           T *__restrict__ f, size_t n)
{
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x)
        st::stv(f + q * stride, in[q] * inv_scale);
}
// out = in * scale, or out = scale where in is NULL (fill)
__global__ void k_scale_copy(const float *__restrict__ in, float scale, float *__restrict__ out,
                             size_t n)
{
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x)
        out[q] = in ? in[q] * scale : scale;
}

// p(t) = A cos(w t + phi): C = A N/2 cos phi, S = -A N/2 sin phi
__global__ void k_amp_phase(const double *__restrict__ C, const double *__restrict__ S, size_t n,
                            double inv_half_n, double scale, double *amp, double *ph)
{
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x) {
        const double c = C[q], s = S[q];
        if (amp) amp[q] = sqrt(c * c + s * s) * inv_half_n * scale;
        if (ph) ph[q] = atan2(-s, c);
    }
}

// One thread per plane point, elements staged through shared memory.
// p = pref * sum_e dA_e (sin(k r) + i cos(k r)) / r   with pref = k p0 / (2 pi):
// the i k p0 / (2 pi) prefactor times exp(-i k r) = cos kr - i sin kr.
// Elements with complex weights w_e (phased arrays): the element's term is
// multiplied by w_e = wr + i wi.
__global__ void __launch_bounds__(kThreads) k_rs_weighted(const float4 *__restrict__ el,
                                                          const float2 *__restrict__ wt, int ne,
                                                          int nx, int ny, float dx, float zp,
                                                          float k_over_pi, double pref,
                                                          float2 *__restrict__ out)
{
    __shared__ float4 s_el[kThreads];
    __shared__ float2 s_w[kThreads];
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = q < nx * ny;
    const float x = live ? (q % nx) * dx : 0.0f;
    const float y = live ? (q / nx) * dx : 0.0f;
    double re = 0.0, im = 0.0;
    for (int base = 0; base < ne; base += kThreads) {
        if (base + threadIdx.x < ne) {
            s_el[threadIdx.x] = el[base + threadIdx.x];
            s_w[threadIdx.x] = wt[base + threadIdx.x];
        }
        __syncthreads();
        const int cnt = min(kThreads, ne - base);
        float pre = 0.0f, pim = 0.0f;
        for (int e = 0; e < cnt; ++e) {
            const float4 E = s_el[e];
            const float2 W = s_w[e];
            const float ddx = x - E.x, ddy = y - E.y, ddz = zp - E.z;
            const float r = sqrtf(fmaf(ddx, ddx, fmaf(ddy, ddy, ddz * ddz)));
            float sn, cs;
            sincospif(k_over_pi * r, &sn, &cs);
            const float w = E.w / r;
            // (wr + i wi)(sin kr + i cos kr)
            pre = fmaf(w, fmaf(W.x, sn, -W.y * cs), pre);
            pim = fmaf(w, fmaf(W.x, cs, W.y * sn), pim);
        }
        re += pre;
        im += pim;
        __syncthreads();
    }
    if (live) out[q] = make_float2((float)(pref * re), (float)(pref * im));
}

__global__ void __launch_bounds__(kThreads) k_rs(const float4 *__restrict__ el, int ne, int nx,
                                                 int ny, float dx, float zp, float k_over_pi,
                                                 double pref, float2 *__restrict__ out)
{
    __shared__ float4 s_el[kThreads];
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = q < nx * ny;
    const float x = live ? (q % nx) * dx : 0.0f;
    const float y = live ? (q / nx) * dx : 0.0f;
    double re = 0.0, im = 0.0;
    for (int base = 0; base < ne; base += kThreads) {
        if (base + threadIdx.x < ne) s_el[threadIdx.x] = el[base + threadIdx.x];
        __syncthreads();
        const int cnt = min(kThreads, ne - base);
        float pre = 0.0f, pim = 0.0f;   // partial sums of one tile in FP32
        for (int e = 0; e < cnt; ++e) {
            const float4 E = s_el[e];
            const float ddx = x - E.x, ddy = y - E.y, ddz = zp - E.z;
            const float r = sqrtf(fmaf(ddx, ddx, fmaf(ddy, ddy, ddz * ddz)));
            float sn, cs;
            sincospif(k_over_pi * r, &sn, &cs);
            const float w = E.w / r;
            pre = fmaf(w, sn, pre);
            pim = fmaf(w, cs, pim);
        }
        re += pre;
        im += pim;
        __syncthreads();
    }
    if (live) out[q] = make_float2((float)(pref * re), (float)(pref * im));
}

__global__ void k_heat_source(const uint8_t *__restrict__ idx, const ThermCoef *__restrict__ lut,
                              const double *__restrict__ amp, double p_scale,
                              float *__restrict__ Q, size_t n)
{
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x) {
        const float A = amp ? (float)(p_scale * amp[q]) : 0.0f;
        Q[q] = lut[idx[q]].qfac * A * A;
    }
}

// Pennes forward-Euler step on the rise; border voxels held at T_a (rise 0);
// T_max and CEM43 fused.
// A 32 x 8 block walks a chunk of z.  Every value plane k needs (T and the
// material of the voxel and its four in-plane neighbours, Q, T_max, the dose
// partial) is loaded one plane ahead, so those loads are in flight while the
// previous plane is computed; the z-neighbours come from the planes already
// held.  Face conductivity: harmonic mean 2 k_c k_n / (k_c + k_n).  The
// chunk length p.kz comes from thermal_kchunk.

// One interior voxel's forward-Euler step on the rise theta = T - T_a:
// theta + dt (div(k grad theta) - w_b c_b theta + DC Q) / (rho c) (T_a is
// constant, so the diffusion of theta is that of T), the six face terms
// summed in the order
// x-, x+, y-, y+, z-, z+ (k_f from the pair table of the centre material c;
// where all six neighbours share c's material, its diagonal entry, held in
// c.k, serves every face without a table read).  Explicit round-to-nearest
// operations, so the direct and TMA kernels agree bit for bit.
__device__ __forceinline__ float thermal_update(const ThParams &p, const ThermCoef &c, int mc,
                                                const float *kf, float Tc, float Tw, int mw,
                                                float Te, int me, float Ts, int ms, float Tq,
                                                int mq, float Tm, int mm, float Tp, int mp, float Q)
{
    float kw, ke, ks, kq, km, kp;
    if (mw == mc && me == mc && ms == mc && mq == mc && mm == mc && mp == mc) {
        kw = ke = ks = kq = km = kp = c.k;
    } else {
        kw = __ldg(kf + mw);
        ke = __ldg(kf + me);
        ks = __ldg(kf + ms);
        kq = __ldg(kf + mq);
        km = __ldg(kf + mm);
        kp = __ldg(kf + mp);
    }
    float lap = __fmul_rn(kw, __fsub_rn(Tw, Tc));
    lap = __fmaf_rn(ke, __fsub_rn(Te, Tc), lap);
    lap = __fmaf_rn(ks, __fsub_rn(Ts, Tc), lap);
    lap = __fmaf_rn(kq, __fsub_rn(Tq, Tc), lap);
    lap = __fmaf_rn(km, __fsub_rn(Tm, Tc), lap);
    lap = __fmaf_rn(kp, __fsub_rn(Tp, Tc), lap);
    const float perf = __fmul_rn(c.perfw, Tc);
    const float rhs = __fmaf_rn(p.dc, Q, __fmaf_rn(lap, p.inv_dx2, -perf));
    return __fmaf_rn(__fmul_rn(p.dt, rhs), c.inv_rhoc, Tc);
}

// The maximum rise and the CEM43 partial of a voxel after its step (dose
// rate R^(43-T) per minute, R = 1/2 at T >= 43 C, 1/4 below: exp2(l2r
// (rise43 - theta)) with l2r = -1 or -2); every 32nd step the FP32 partial
// goes into the FP64 sum.
__device__ __forceinline__ void thermal_outputs(const ThParams &p, size_t q, float Tn, float Tmax,
                                                float cemf)
{
    p.Tmax[q] = fmaxf(Tmax, Tn);
    const float l2r = (Tn >= p.rise43) ? -1.0f : -2.0f;
    const float part = __fmaf_rn(p.dt60, exp2f(__fmul_rn(l2r, __fsub_rn(p.rise43, Tn))), cemf);
    if (p.flush) {
        p.cem[q] += (double)part;
        p.cemf[q] = 0.0f;
    } else {
        p.cemf[q] = part;
    }
}

__global__ void __launch_bounds__(256) k_thermal(ThParams p)
{
    extern __shared__ ThermCoef s_th[];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int m = tid; m < p.n_mat; m += blockDim.x * blockDim.y) s_th[m] = p.lut[m];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    if (i >= nx || j >= ny) return;
    const int k0 = blockIdx.z * p.kz, k1 = min(nz, k0 + p.kz);
    const int SZ = nx * ny, col = j * nx + i;
    const bool xy_border = i == 0 || j == 0 || i == nx - 1 || j == ny - 1;
    const float *__restrict__ T = p.T;
    const uint8_t *__restrict__ idx = p.idx;
    // everything plane k needs, loaded one plane ahead
    struct Plane {
        float Tc, Tw, Te, Ts, Tq, Q, Tmax, cemf;
        int mc, mw, me, ms, mq;
    };
    auto load = [&](int k, Plane &P) {
        const int q = k * SZ + col;
        P.Tc = __ldg(T + q);
        P.mc = __ldg(idx + q);
        P.Q = p.Q[q];
        P.Tmax = p.Tmax[q];
        P.cemf = p.cemf[q];
        if (!xy_border) {
            P.Tw = __ldg(T + q - 1); P.Te = __ldg(T + q + 1);
            P.Ts = __ldg(T + q - nx); P.Tq = __ldg(T + q + nx);
            P.mw = __ldg(idx + q - 1); P.me = __ldg(idx + q + 1);
            P.ms = __ldg(idx + q - nx); P.mq = __ldg(idx + q + nx);
        }
    };
    float Tm = k0 > 0 ? __ldg(T + (k0 - 1) * SZ + col) : 0.0f;
    int mm = k0 > 0 ? __ldg(idx + (k0 - 1) * SZ + col) : 0;
    Plane cur, nxt;
    load(k0, cur);
    for (int k = k0; k < k1; ++k) {
        const int q = k * SZ + col;
        if (k + 1 < nz) load(k + 1, nxt);
        else { nxt.Tc = 0.0f; nxt.mc = 0; }
        float Tn;
        if (xy_border || k == 0 || k == nz - 1) {
            Tn = 0.0f;
        } else {
            // face conductivities 2 k_a k_b / (k_a + k_b) from the pair table
            Tn = thermal_update(p, s_th[cur.mc], cur.mc, p.kface + cur.mc * p.n_mat, cur.Tc, cur.Tw,
                                cur.mw, cur.Te, cur.me, cur.Ts, cur.ms, cur.Tq, cur.mq, Tm, mm,
                                nxt.Tc, nxt.mc, cur.Q);
        }
        p.Tn[q] = Tn;
        thermal_outputs(p, q, Tn, cur.Tmax, cur.cemf);
        Tm = cur.Tc;
        mm = cur.mc;
        cur = nxt;
    }
}

// TMA-fed step (grids with nx % 8 == 0).  A block of 32 x 8 threads owns a
// 32 x 16 x-y tile (thread (tx, ty) the voxels of rows ty and ty + 8) and
// walks a z-chunk.  Every input of a plane arrives through the tensor-memory
// accelerator in a four-plane shared-memory ring: T and the material index
// as halo'd boxes (T: x0-4 .. x0+35, index: x0-16 .. x0+47, both
// y0-1 .. y0+16; a TMA box starts on a 16-byte boundary, out-of-range
// elements read as zero and only feed border voxels, which are held at T_a),
// Q, T_max and the dose partial as 32 x 16 boxes.  Plane k reads planes k-1,
// k, k+1 of the ring while plane k+2 is in flight, so the kernel's loads run
// two planes ahead of its arithmetic; results are stored directly.  One
// thread issues the copies; waits are bounded as in the acoustic kernels (a
// time-out sets bit 2 of the flag after the block's armed copies have
// landed).
constexpr int kThRing = 4;                                             // planes k-1 .. k+2
constexpr int kThTileY = 16;
constexpr int kThTW = 40, kThTH = kThTileY + 2, kThTBytes = kThTW * kThTH * 4;   // 2880 B
constexpr int kThTSlot = 2944;                                         // 23 x 128 B
constexpr int kThIW = 64, kThIBytes = kThIW * kThTH;                   // 1152 B
constexpr int kThVBytes = 32 * kThTileY * 4;                           // Q, T_max, partial: 2048 B
constexpr int kThSlot = kThTSlot + kThIBytes + 3 * kThVBytes;          // one plane: 10240 B
constexpr int kThOffBar = kThRing * kThSlot;
constexpr int kThOffAbort = kThOffBar + 8 * kThRing;
constexpr int kThOffLut = (kThOffAbort + (int)sizeof(int) + 15) / 16 * 16;
constexpr unsigned kThPlaneBytes = kThTBytes + kThIBytes + 3 * kThVBytes;
static_assert(kThTSlot % 128 == 0 && kThTSlot >= kThTBytes && kThIBytes % 128 == 0 &&
                  kThVBytes % 128 == 0 && kThSlot % 128 == 0 && kThOffLut % 16 == 0,
              "ring slots 128-byte aligned, coefficients 16");

__global__ void __launch_bounds__(256, 5)
    k_thermal_tma(ThParams p, const __grid_constant__ ThermTmaMaps tm, int *flag)
{
    extern __shared__ __align__(128) unsigned char smb[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smb + kThOffBar);
    volatile int *s_abort = reinterpret_cast<volatile int *>(smb + kThOffAbort);
    ThermCoef *s_th = reinterpret_cast<ThermCoef *>(smb + kThOffLut);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    for (int m = tid; m < p.n_mat; m += 256) s_th[m] = p.lut[m];
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * kThTileY, i = x0 + tx;
    const int k0 = blockIdx.z * p.kz, k1 = min(nz, k0 + p.kz);
    if (tid == 0) {
        for (int b = 0; b < kThRing; ++b) tma::mbar_init(&bars[b], 1);
        tma::mbar_init_fence();
        *s_abort = -1;
    }
    __syncthreads();
    // plane pl of the chunk's window k0-1 .. k1 sits in slot (pl - k0 + 1) % 4,
    // the (pl - k0 + 1) / 4-th phase of that slot's barrier; a slot holds T,
    // the index, Q, T_max and the partial of its plane, in that order
    auto slot = [&](int pl) { return (pl - k0 + 1) & (kThRing - 1); };
    auto parity = [&](int pl) { return (unsigned)((pl - k0 + 1) >> 2) & 1u; };
    auto issue = [&](int pl) {
        uint64_t *bar = &bars[slot(pl)];
        unsigned char *d = smb + slot(pl) * kThSlot;
        // the per-voxel streams only for the chunk's own planes; its two
        // neighbour planes supply T and the index
        const bool own = pl >= k0 && pl < k1;
        tma::mbar_expect_tx(bar, own ? kThPlaneBytes : (unsigned)(kThTBytes + kThIBytes));
        if (p.hold_plane >= 0 && pl == p.hold_plane) return;   // test hook: armed, none issued
        tma::load3d(d, &tm.T, x0 - 4, y0 - 1, pl, bar);
        tma::load3d(d + kThTSlot, &tm.idx, x0 - 16, y0 - 1, pl, bar);
        if (own) {
            tma::load3d(d + kThTSlot + kThIBytes, &tm.Q, x0, y0, pl, bar);
            tma::load3d(d + kThTSlot + kThIBytes + kThVBytes, &tm.Tmax, x0, y0, pl, bar);
            tma::load3d(d + kThTSlot + kThIBytes + 2 * kThVBytes, &tm.cemf, x0, y0, pl, bar);
        }
    };
    auto wait = [&](int pl) { return tma::mbar_wait(&bars[slot(pl)], parity(pl), p.wait_limit); };
    const int first_last = min(k1, k0 + 2);
    if (tid == 0)
        for (int pl = k0 - 1; pl <= first_last; ++pl) issue(pl);
    int issued = first_last;

    // the thread's two voxels: rows j = y0 + ty + 8 h, h = 0, 1
    bool live[2], border[2];
    int ct[2], ci[2], cv[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int j = y0 + ty + 8 * h;
        live[h] = i < nx && j < ny;
        border[h] = i == 0 || j == 0 || i == nx - 1 || j == ny - 1;
        ct[h] = (ty + 8 * h + 1) * kThTW + tx + 4;
        ci[h] = (ty + 8 * h + 1) * kThIW + tx + 16;
        cv[h] = (ty + 8 * h) * 32 + tx;
    }
    const size_t SZ = (size_t)nx * ny;
    size_t q0 = (size_t)k0 * SZ + (size_t)(y0 + ty) * nx + i;     // row ty of plane k
    const size_t q8 = (size_t)8 * nx;                                // row ty + 8
    for (int k = k0; k < k1; ++k, q0 += SZ) {
        __syncthreads();
        if (*s_abort >= 0) break;                 // a wait of the previous plane ran out
        if (k + 2 <= k1 && k + 2 > issued) {      // into the slot plane k-2 has freed
            if (tid == 0) {
                tma::fence_async_smem();
                issue(k + 2);
            }
            issued = k + 2;
        }
        bool ready = true;
        if (k == k0) ready = wait(k0 - 1) && wait(k0);
        ready = ready && wait(k + 1);
        if (!ready) *s_abort = k;
        if (!ready) continue;                     // leaves at the next barrier
        const unsigned char *S0 = smb + slot(k) * kThSlot;
        const unsigned char *Sz0 = smb + slot(k - 1) * kThSlot;
        const unsigned char *Sz1 = smb + slot(k + 1) * kThSlot;
        const float *T0 = reinterpret_cast<const float *>(S0);
        const float *Tz0 = reinterpret_cast<const float *>(Sz0);
        const float *Tz1 = reinterpret_cast<const float *>(Sz1);
        const unsigned char *I0 = S0 + kThTSlot, *Iz0 = Sz0 + kThTSlot, *Iz1 = Sz1 + kThTSlot;
        const float *V0 = reinterpret_cast<const float *>(S0 + kThTSlot + kThIBytes);
        const bool zb = k == 0 || k == nz - 1;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (!live[h]) continue;
            const float Q = V0[cv[h]], Tmax = V0[cv[h] + kThVBytes / 4],
                        cemf = V0[cv[h] + kThVBytes / 2];
            float Tn;
            if (border[h] || zb) {
                Tn = 0.0f;
            } else {
                const int c = ct[h], d = ci[h];
                const int mc = I0[d];
                Tn = thermal_update(p, s_th[mc], mc, p.kface + mc * p.n_mat, T0[c], T0[c - 1],
                                    I0[d - 1], T0[c + 1], I0[d + 1], T0[c - kThTW], I0[d - kThIW],
                                    T0[c + kThTW], I0[d + kThIW], Tz0[c], Iz0[d], Tz1[c], Iz1[d],
                                    Q);
            }
            const size_t q = q0 + h * q8;
            p.Tn[q] = Tn;
            thermal_outputs(p, q, Tn, Tmax, cemf);
        }
    }
    __syncthreads();
    const int ab = *s_abort;
    if (ab >= 0 && tid == 0) {
        // every armed phase from the one that ran out on has landed before
        // the block's shared memory is released
        for (int pl = max(k0 - 1, ab - 1); pl <= issued; ++pl) wait(pl);
        atomicOr(flag, 2);
    }
}

// Intensity I = A^2 / (2 rho c) = A^2 * zw[m] with zw[m] = 1 / (2 rho c).
// Positive doubles order like their bit patterns, so atomicMax on the bits
// finds the maximum.
__global__ void k_int_max(const uint8_t *__restrict__ idx, const double *__restrict__ zw,
                          const double *__restrict__ amp, size_t n, unsigned long long *best)
{
    unsigned long long m = 0;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x) {
        const double I = amp[q] * amp[q] * zw[idx[q]];
        m = max(m, (unsigned long long)__double_as_longlong(I));
    }
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(best, m);
}

__global__ void k_int_argmin(const uint8_t *__restrict__ idx, const double *__restrict__ zw,
                             const double *__restrict__ amp, size_t n,
                             const unsigned long long *best, unsigned long long *out)
{
    const unsigned long long b = *best;
    unsigned long long m = ~0ull;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x) {
        const double I = amp[q] * amp[q] * zw[idx[q]];
        if ((unsigned long long)__double_as_longlong(I) == b) m = min(m, (unsigned long long)q);
    }
    for (int o = 16; o; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMin(out, m);
}

// Plane sums of both intensity maps at z_m, one block, fixed order.
__global__ void __launch_bounds__(1024) k_plane_sums(
    const uint8_t *__restrict__ ia, const double *__restrict__ za, const double *__restrict__ aa,
    const uint8_t *__restrict__ iw, const double *__restrict__ zw, const double *__restrict__ aw,
    int nx, int ny, int nz, const unsigned long long *qbest, double *sums)
{
    __shared__ double s_a[1024], s_w[1024];
    const long long plane = (long long)nx * ny;
    if (*qbest >= (unsigned long long)(plane * nz)) {   // no maximum found
        if (threadIdx.x == 0) sums[0] = sums[1] = sums[2] = 0.0;
        return;
    }
    const long long z = (long long)(*qbest / (unsigned long long)plane);
    const long long base = z * plane;
    double sa = 0.0, sw = 0.0;
    for (long long t = threadIdx.x; t < plane; t += blockDim.x) {
        const long long q = base + t;
        sa += aa[q] * aa[q] * za[ia[q]];
        sw += aw[q] * aw[q] * zw[iw[q]];
    }
    s_a[threadIdx.x] = sa;
    s_w[threadIdx.x] = sw;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if ((int)threadIdx.x < o) {
            s_a[threadIdx.x] += s_a[threadIdx.x + o];
            s_w[threadIdx.x] += s_w[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sums[0] = s_a[0];
        sums[1] = s_w[0];
        sums[2] = (double)z;
    }
}

// Time-reversal (phase-conjugation) plane from the FP64 DFT sums of one
// z-plane: with amplitude 2 |C - iS| / N and phase atan2(-S, C) the captured
// complex amplitude is P = (2/N)(C - iS), so conj(P) / max|P| over the plane is
// (C + iS) / max |C + iS|.  First pass: the largest |C + iS|^2 of the plane
// (non-negative doubles order like their bit patterns, so one 64-bit
// atomicMax keeps it); second pass: the normalised conjugate.
__global__ void k_plane_absmax(const double *__restrict__ C, const double *__restrict__ S,
                               size_t n, unsigned long long *out)
{
    double m = 0.0;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x)
        m = fmax(m, C[q] * C[q] + S[q] * S[q]);
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

__global__ void k_conj_normalise(const double *__restrict__ C, const double *__restrict__ S,
                                 size_t n, const unsigned long long *mx, float2 *__restrict__ out)
{
    const double m2 = __longlong_as_double((long long)*mx);
    const double inv = m2 > 0.0 ? 1.0 / sqrt(m2) : 0.0;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x)
        out[q] = make_float2((float)(C[q] * inv), (float)(S[q] * inv));
}

}  // namespace

cudaError_t launch_conj_plane(const double *C, const double *S, size_t n,
                              unsigned long long *d_max, float2 *out, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(d_max, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_plane_absmax<<<blocks_for(n), kThreads, 0, s>>>(C, S, n, d_max);
    k_conj_normalise<<<blocks_for(n), kThreads, 0, s>>>(C, S, n, d_max, out);
    return cudaGetLastError();
}

cudaError_t launch_index_max(const uint8_t *idx, size_t n, unsigned *d_out, cudaStream_t s)
{
    k_index_max<<<blocks_for(n), kThreads, 0, s>>>(idx, n, d_out);
    return cudaGetLastError();
}

cudaError_t launch_pressure(const void *sxx, const void *syy, const void *szz, int h16,
                            float scale, float *out, size_t n, cudaStream_t s)
{
    if (h16)
        k_pressure<__half><<<blocks_for(n), kThreads, 0, s>>>(
            static_cast<const __half *>(sxx), static_cast<const __half *>(syy),
            static_cast<const __half *>(szz), scale, out, n);
    else
        k_pressure<float><<<blocks_for(n), kThreads, 0, s>>>(
            static_cast<const float *>(sxx), static_cast<const float *>(syy),
            static_cast<const float *>(szz), scale, out, n);
    return cudaGetLastError();
}

cudaError_t launch_field_out(const void *f, int h16, size_t stride, float scale, float *out,
                             size_t n, cudaStream_t s)
{
    if (h16)
        k_field_out<__half><<<blocks_for(n), kThreads, 0, s>>>(static_cast<const __half *>(f),
                                                              stride, scale, out, n);
    else
        k_field_out<float><<<blocks_for(n), kThreads, 0, s>>>(static_cast<const float *>(f),
                                                             stride, scale, out, n);
    return cudaGetLastError();
}

cudaError_t launch_field_in(const float *in, int h16, size_t stride, float inv_scale, void *f,
                            size_t n, cudaStream_t s)
{
    if (h16)
        k_field_in<__half><<<blocks_for(n), kThreads, 0, s>>>(in, stride, inv_scale,
                                                             static_cast<__half *>(f), n);
    else
        k_field_in<float><<<blocks_for(n), kThreads, 0, s>>>(in, stride, inv_scale,
                                                            static_cast<float *>(f), n);
    return cudaGetLastError();
}

__global__ void k_add_const(float *__restrict__ x, float c, size_t n)
{
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x)
        x[q] = __fadd_rn(x[q], c);
}

cudaError_t launch_add_const(float *x, float c, size_t n, cudaStream_t s)
{
    k_add_const<<<blocks_for(n), kThreads, 0, s>>>(x, c, n);
    return cudaGetLastError();
}

cudaError_t launch_fill(float *out, float value, size_t n, cudaStream_t s)
{
    k_scale_copy<<<blocks_for(n), kThreads, 0, s>>>(nullptr, value, out, n);
    return cudaGetLastError();
}

cudaError_t launch_scale_copy(const float *in, float scale, float *out, size_t n, cudaStream_t s)
{
    k_scale_copy<<<blocks_for(n), kThreads, 0, s>>>(in, scale, out, n);
    return cudaGetLastError();
}

cudaError_t launch_amp_phase(const double *C, const double *S, size_t n, int count, double scale,
                             double *amp, double *ph, cudaStream_t s)
{
    k_amp_phase<<<blocks_for(n), kThreads, 0, s>>>(C, S, n, 2.0 / count, scale, amp, ph);
    return cudaGetLastError();
}

cudaError_t launch_rs(const float4 *el, int ne, int nx, int ny, float dx, float zp, float k_over_pi,
                      double pref, float2 *out, cudaStream_t s)
{
    const int n = nx * ny;
    k_rs<<<(n + kThreads - 1) / kThreads, kThreads, 0, s>>>(el, ne, nx, ny, dx, zp, k_over_pi,
                                                           pref, out);
    return cudaGetLastError();
}

cudaError_t launch_rs_weighted(const float4 *el, const float2 *wt, int ne, int nx, int ny,
                               float dx, float zp, float k_over_pi, double pref, float2 *out,
                               cudaStream_t s)
{
    const int n = nx * ny;
    k_rs_weighted<<<(n + kThreads - 1) / kThreads, kThreads, 0, s>>>(el, wt, ne, nx, ny, dx, zp,
                                                                    k_over_pi, pref, out);
    return cudaGetLastError();
}

cudaError_t launch_heat_source(const uint8_t *idx, const ThermCoef *lut, int n_mat,
                               const double *amp, double p_scale, float *Q, size_t n,
                               cudaStream_t s)
{
    (void)n_mat;
    k_heat_source<<<blocks_for(n), kThreads, 0, s>>>(idx, lut, amp, p_scale, Q, n);
    return cudaGetLastError();
}

// The z-chunk of a BHTE launch: blocks of a chunk run in waves of
// (resident blocks per SM) x (SMs); a block's time is about its planes plus
// two (the z-neighbour planes and the pipeline fill), so the chunk length kz
// in 4 .. 32 that minimises waves(kz) x (kz + 2) is taken.
int thermal_kchunk(int nx, int ny, int nz, bool tma, int n_mat)
{
    int dev = 0, n_sm = 152, per_sm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = tma ? kThOffLut + n_mat * sizeof(ThermCoef) : n_mat * sizeof(ThermCoef);
    const cudaError_t e =
        tma ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_thermal_tma, 256, smem)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_thermal, 256, smem);
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    const long long tiles = (long long)((nx + 31) / 32) * ((ny + (tma ? kThTileY : 8) - 1) /
                                                           (tma ? kThTileY : 8));
    const long long slots = (long long)per_sm * n_sm;
    int best = 16;
    long long best_cost = -1;
    for (int kz = 4; kz <= 32; ++kz) {
        const long long blocks = tiles * ((nz + kz - 1) / kz);
        const long long cost = ((blocks + slots - 1) / slots) * (kz + 2);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = kz;
        }
    }
    return best < nz ? best : (nz > 0 ? nz : 1);
}

cudaError_t launch_thermal_step(const ThParams &p, const ThermTmaMaps *tm, int *flag,
                               cudaStream_t s)
{
    dim3 blk(32, 8, 1);
    dim3 grd((p.nx + 31) / 32, (p.ny + 7) / 8, (p.nz + p.kz - 1) / p.kz);
    if (tm) {
        grd.y = (p.ny + kThTileY - 1) / kThTileY;
        k_thermal_tma<<<grd, blk, kThOffLut + p.n_mat * sizeof(ThermCoef), s>>>(p, *tm, flag);
    } else {
        k_thermal<<<grd, blk, p.n_mat * sizeof(ThermCoef), s>>>(p);
    }
    return cudaGetLastError();
}

cudaError_t launch_intensity_argmax(const uint8_t *idx, const double *zw, const double *amp,
                                    size_t n, unsigned long long *d_best, cudaStream_t s)
{
    k_int_max<<<blocks_for(n), kThreads, 0, s>>>(idx, zw, amp, n, d_best);
    return cudaGetLastError();
}

cudaError_t launch_intensity_argmin_index(const uint8_t *idx, const double *zw,
                                          const double *amp, size_t n,
                                          const unsigned long long *d_best,
                                          unsigned long long *d_idx, cudaStream_t s)
{
    k_int_argmin<<<blocks_for(n), kThreads, 0, s>>>(idx, zw, amp, n, d_best, d_idx);
    return cudaGetLastError();
}

cudaError_t launch_plane_sums(const uint8_t *idx_a, const double *za, const double *amp_a,
                              const uint8_t *idx_w, const double *zw, const double *amp_w,
                              int nx, int ny, int nz, const unsigned long long *d_idx,
                              double *d_sums, cudaStream_t s)
{
    k_plane_sums<<<1, 1024, 0, s>>>(idx_a, za, amp_a, idx_w, zw, amp_w, nx, ny, nz, d_idx, d_sums);
    return cudaGetLastError();
}

}  // namespace bvf
