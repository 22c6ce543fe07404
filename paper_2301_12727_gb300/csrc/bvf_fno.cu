// Fourier-neural-operator surrogate: inference kernels and the C ABI of
// bvf_fno.h.  The network is the Fourier neural operator of Li et al. (ICLR
// 2021, Sec. 4); the paper's Discussion names learned models as the route to
// interactive planning, with the FDTD as the reference they are judged by.
//
// The truncated FFT of a Fourier layer is done as direct DFT sums over the
// kept modes, one axis at a time, because only m of the n frequencies of
// each axis survive.  Twiddles come from per-grid tables e^{2 pi i f j / n}
// computed in FP64 on the host.  Per layer:
//   - the y and z transforms, the mode mix and their inverses run on the
//     truncated spectra (a few MB, L2-resident);
//   - the layer output (inverse x transform, W v + b and GELU) is one
//     tensor-core product per 128-point tile of a (z, y) row (k_row_tc), and
//     the next layer's forward x transform is one tall product over all rows
//     of the new v (k_dftx_tc);
//   - the lift is the layer output without the spectral term.
// The projection is a tensor-core product with GELU in its epilogue
// (k_project_tc).  All three run on the fifth-generation tensor cores
// (tcgen05.mma into TMEM, tcgen05.ld epilogues), and every product uses the
// three-term TF32 split, which keeps FP32 accuracy.  Rows too long for
// shared memory take unfused SIMT kernels (k_lift, k_dftx, k_layer_out).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/bvf_fno.h"
#include "bvf_internal.cuh"
#include "bvf_tc.cuh"
#include "bvf_tma.cuh"

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

int fno_fail(int code, const std::string &msg)
{
    bvf::set_context_free_error(msg.c_str());
    return code;
}

int fno_cuda(cudaError_t e, const char *where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fno_fail(e == cudaErrorMemoryAllocation ? BVF_E_NOMEM : BVF_E_CUDA, m);
}

#define FCK(call, where)                                \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return fno_cuda(e_, where); \
    } while (0)

bool dims_valid(const bvf_fno_dims *d)
{
    return d && d->c_in >= 1 && d->c_in <= BVF_FNO_MAX_CIN && d->width >= 16 &&
           d->width <= BVF_FNO_MAX_WIDTH && d->width % 16 == 0 && d->modes >= 1 &&
           d->modes <= BVF_FNO_MAX_MODES && d->n_layers >= 1 &&
           d->n_layers <= BVF_FNO_MAX_LAYERS && d->hidden >= 1 &&
           d->hidden <= BVF_FNO_MAX_HIDDEN && d->c_out >= 1 && d->c_out <= BVF_FNO_MAX_COUT;
}

size_t layer_floats(const bvf_fno_dims &d)
{
    const size_t m3 = (size_t)(2 * d.modes) * (2 * d.modes) * d.modes;
    return m3 * d.width * d.width * 2 + (size_t)d.width * d.width + d.width;
}

// signed frequency of mode slot j in [0, 2m) of a y or z axis
__host__ __device__ __forceinline__ int slot_freq(int j, int m) { return j < m ? j : j - 2 * m; }

// GELU(s) = s Phi(s) = (s/2)(1 + erf(s/sqrt 2)).  erf is Hastings' rational
// approximation as printed in Abramowitz & Stegun, Handbook of Mathematical
// Functions, 7.1.26: for x >= 0, erf(x) = 1 - t(a1 + t(a2 + t(a3 + t(a4 + t a5))))
// e^{-x^2} with t = 1/(1 + p x), |error| <= 1.5e-7; odd symmetry for x < 0.
__device__ __forceinline__ float gelu(float s)
{
    const float x = fabsf(s) * 0.70710678118654752f;
    const float t = __fdividef(1.0f, fmaf(0.3275911f, x, 1.0f));
    float q = fmaf(1.061405429f, t, -1.453152027f);
    q = fmaf(q, t, 1.421413741f);
    q = fmaf(q, t, -0.284496736f);
    q = fmaf(q, t, 0.254829592f);
    const float erfc_x = q * t * __expf(-x * x);
    // s Phi(s): Phi(|s|) = 1 - erfc/2 for s >= 0, Phi(-|s|) = erfc/2
    const float phi = s >= 0.0f ? 1.0f - 0.5f * erfc_x : 0.5f * erfc_x;
    return s * phi;
}

// The same GELU on two values at once: the polynomial, the products and the
// final scaling on the packed FP32x2 multiply / fused multiply-add of sm_100
// and later (half the instructions); the reciprocal and the exponential stay
// per value.
__device__ __forceinline__ float2 gelu2(float2 s)
{
    const float2 k = make_float2(0.70710678118654752f, 0.70710678118654752f);
    const float2 x = __fmul2_rn(make_float2(fabsf(s.x), fabsf(s.y)), k);
    const float2 den = __ffma2_rn(make_float2(0.3275911f, 0.3275911f), x, make_float2(1.0f, 1.0f));
    const float2 t = make_float2(__fdividef(1.0f, den.x), __fdividef(1.0f, den.y));
    float2 q = __ffma2_rn(make_float2(1.061405429f, 1.061405429f), t,
                          make_float2(-1.453152027f, -1.453152027f));
    q = __ffma2_rn(q, t, make_float2(1.421413741f, 1.421413741f));
    q = __ffma2_rn(q, t, make_float2(-0.284496736f, -0.284496736f));
    q = __ffma2_rn(q, t, make_float2(0.254829592f, 0.254829592f));
    const float2 e = make_float2(__expf(-x.x * x.x), __expf(-x.y * x.y));
    const float2 h = __fmul2_rn(__fmul2_rn(__fmul2_rn(q, t), e), make_float2(0.5f, 0.5f));
    const float2 phi =
        make_float2(s.x >= 0.0f ? 1.0f - h.x : h.x, s.y >= 0.0f ? 1.0f - h.y : h.y);
    return __fmul2_rn(s, phi);
}

// ------------------------------------------------------------------ lift
__global__ void k_lift(const float *__restrict__ a, int c_in, int width,
                       const float *__restrict__ Wp, const float *__restrict__ bp,
                       float *__restrict__ v, int N)
{
    extern __shared__ float s_w[];
    const int nw = width * c_in;
    for (int t = threadIdx.x; t < nw + width; t += blockDim.x)
        s_w[t] = t < nw ? Wp[t] : bp[t - nw];
    __syncthreads();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    float x[BVF_FNO_MAX_CIN];
#pragma unroll
    for (int i = 0; i < BVF_FNO_MAX_CIN; ++i) x[i] = i < c_in ? a[(size_t)i * N + p] : 0.0f;
    for (int o = 0; o < width; ++o) {
        float acc = s_w[nw + o];
#pragma unroll
        for (int i = 0; i < BVF_FNO_MAX_CIN; ++i)
            if (i < c_in) acc = fmaf(s_w[o * c_in + i], x[i], acc);
        v[(size_t)o * N + p] = acc;
    }
}

// ------------------------------------------------------ forward DFT along x
// A[r][kx] = sum_x v[r][x] e^{-2 pi i kx x / nx} for the rows r = (c, z, y):
// a [rows x nx] by [nx x m] complex product.  A block takes TR = 128 rows and
// walks x in chunks of 32: the chunk of its rows (coalesced, row pitch 34
// floats) and of the twiddle table go to shared memory, then each thread
// accumulates one frequency of 8 rows, two x at a time.
constexpr int kXR = 8;          // rows per thread
constexpr int kXT = 128;        // rows per block
constexpr int kXC = 32;         // x per chunk
constexpr int kXP = kXC + 2;    // row pitch in shared memory

__global__ void k_dftx(const float *__restrict__ v, int rows, int nx, int m,
                       const float2 *__restrict__ tx, float2 *__restrict__ A)
{
    __shared__ __align__(16) float s_u[kXT * kXP];
    __shared__ __align__(16) float2 s_t[BVF_FNO_MAX_MODES * kXC];
    const int tid = threadIdx.x, nth = blockDim.x;
    const long r0 = (long)blockIdx.x * kXT;
    const int kx = tid % m, g = tid / m;       // g < kXT / kXR
    float re[kXR], im[kXR];
#pragma unroll
    for (int q = 0; q < kXR; ++q) re[q] = im[q] = 0.0f;
    for (int x0 = 0; x0 < nx; x0 += kXC) {
        const int w = min(kXC, nx - x0);
        __syncthreads();
        for (int e = tid; e < kXT * kXC; e += nth) {
            const int r = e / kXC, x = e - r * kXC;
            const long rr = r0 + r;
            s_u[r * kXP + x] = (x < w && rr < rows) ? v[rr * nx + x0 + x] : 0.0f;
        }
        for (int e = tid; e < m * kXC; e += nth) {
            const int k = e / kXC, x = e - k * kXC;
            s_t[e] = x < w ? tx[(long)k * nx + x0 + x] : make_float2(0.0f, 0.0f);
        }
        __syncthreads();
        const float *u = s_u + g * kXR * kXP;
        const float2 *t = s_t + kx * kXC;
#pragma unroll 4
        for (int x = 0; x < kXC; x += 2) {
            const float2 t0 = t[x], t1 = t[x + 1];
#pragma unroll
            for (int q = 0; q < kXR; ++q) {
                const float2 uu = *reinterpret_cast<const float2 *>(u + q * kXP + x);
                re[q] = fmaf(uu.x, t0.x, fmaf(uu.y, t1.x, re[q]));
                im[q] = fmaf(-uu.x, t0.y, fmaf(-uu.y, t1.y, im[q]));
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kXR; ++q) {
        const long r = r0 + g * kXR + q;
        if (r < rows) A[r * m + kx] = make_float2(re[q], im[q]);
    }
}

// complex a * e^{s i theta} with the table entry t = (cos, sin) and s = +-1
__device__ __forceinline__ float2 cmul_tw(float2 a, float2 t, float s)
{
    return make_float2(a.x * t.x - s * a.y * t.y, a.y * t.x + s * a.x * t.y);
}

// ------------------------------------------------------ forward DFT along y
// B[c][z][jy][kx] = sum_y A[c][z][y][kx] e^{-2 pi i f(jy) y / ny}; one block
// per (c, z) slab; each thread takes the mode slots jy and jy + m of one kx
// (the same A column against two twiddle rows).
__global__ void k_dfty(const float2 *__restrict__ A, int ny, int m,
                       const float2 *__restrict__ ty, float2 *__restrict__ B)
{
    extern __shared__ float2 s_y[];
    float2 *s_a = s_y;                  // [ny][m]
    const long slab = blockIdx.x;
    const float2 *a = A + slab * ny * m;
    for (int e = threadIdx.x; e < ny * m; e += blockDim.x) s_a[e] = a[e];
    __syncthreads();
    const int t = threadIdx.x;
    if (t >= m * m) return;
    const int jy = t / m, kx = t - jy * m;           // jy in [0, m); the pair is jy + m
    const float2 *tw0 = ty + (long)jy * ny, *tw1 = ty + (long)(jy + m) * ny;
    float2 a0[2] = {{0.0f, 0.0f}, {0.0f, 0.0f}}, a1[2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
    int y = 0;
    for (; y + 2 <= ny; y += 2) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const float2 v = s_a[(y + q) * m + kx];
            const float2 p0 = cmul_tw(v, __ldg(tw0 + y + q), -1.0f);
            const float2 p1 = cmul_tw(v, __ldg(tw1 + y + q), -1.0f);
            a0[q].x += p0.x;
            a0[q].y += p0.y;
            a1[q].x += p1.x;
            a1[q].y += p1.y;
        }
    }
    for (; y < ny; ++y) {
        const float2 v = s_a[y * m + kx];
        const float2 p0 = cmul_tw(v, __ldg(tw0 + y), -1.0f);
        const float2 p1 = cmul_tw(v, __ldg(tw1 + y), -1.0f);
        a0[0].x += p0.x;
        a0[0].y += p0.y;
        a1[0].x += p1.x;
        a1[0].y += p1.y;
    }
    B[(slab * 2 * m + jy) * m + kx] = make_float2(a0[0].x + a0[1].x, a0[0].y + a0[1].y);
    B[(slab * 2 * m + jy + m) * m + kx] = make_float2(a1[0].x + a1[1].x, a1[0].y + a1[1].y);
}

// ------------------------------------------------------ forward DFT along z
// H[c][jz][q] = sum_z B[c][z][q] e^{-2 pi i f(jz) z / nz}, q = (jy, kx).
__global__ void k_dftz(const float2 *__restrict__ B, int nz, int m, int width,
                       const float2 *__restrict__ tz, float2 *__restrict__ H)
{
    const int M2 = 2 * m * m;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)width * 2 * m * M2) return;
    const int q = (int)(t % M2);
    const long rest = t / M2;
    const int jz = (int)(rest % (2 * m)), c = (int)(rest / (2 * m));
    const float2 *b = B + (long)c * nz * M2 + q;
    const float2 *tw = tz + (long)jz * nz;
    float2 acc = make_float2(0.0f, 0.0f);
    for (int z = 0; z < nz; ++z) {
        const float2 p = cmul_tw(b[(long)z * M2], __ldg(tw + z), -1.0f);
        acc.x += p.x;
        acc.y += p.y;
    }
    H[t] = acc;     // t = (c * 2m + jz) * M2 + q
}

// ------------------------------------------------------------ mode mixing
// G[o][mode] = sum_c R[mode][c][o] H[c][mode]; block (width, 256/width modes).
__global__ void k_mix(const float2 *__restrict__ H, const float2 *__restrict__ R, int width,
                      int n_modes, float2 *__restrict__ G)
{
    extern __shared__ float2 s_h[];              // [blockDim.y][width]
    const int o = threadIdx.x, ty = threadIdx.y;
    const int mode = blockIdx.x * blockDim.y + ty;
    for (int c = o; c < width; c += blockDim.x)
        s_h[ty * width + c] = mode < n_modes ? H[(long)c * n_modes + mode] : make_float2(0.f, 0.f);
    __syncthreads();
    if (mode >= n_modes) return;
    const float2 *r = R + (long)mode * width * width + o;
    float2 acc = make_float2(0.0f, 0.0f);
    for (int c = 0; c < width; ++c) {
        const float2 w = r[(long)c * width], h = s_h[ty * width + c];
        acc.x = fmaf(w.x, h.x, fmaf(-w.y, h.y, acc.x));
        acc.y = fmaf(w.x, h.y, fmaf(w.y, h.x, acc.y));
    }
    G[(long)o * n_modes + mode] = acc;
}

// ------------------------------------------------------ inverse along z
// B'[o][z][q] = sum_jz G[o][jz][q] e^{+2 pi i f(jz) z / nz}
__global__ void k_idftz(const float2 *__restrict__ G, int nz, int m, int width,
                        const float2 *__restrict__ tz, float2 *__restrict__ Bp)
{
    const int M2 = 2 * m * m;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)width * nz * M2) return;
    const int q = (int)(t % M2);
    const long rest = t / M2;
    const int z = (int)(rest % nz), o = (int)(rest / nz);
    const float2 *g = G + (long)o * 2 * m * M2 + q;
    float2 acc = make_float2(0.0f, 0.0f);
    for (int jz = 0; jz < 2 * m; ++jz) {
        const float2 p = cmul_tw(g[(long)jz * M2], __ldg(tz + (long)jz * nz + z), 1.0f);
        acc.x += p.x;
        acc.y += p.y;
    }
    Bp[t] = acc;    // t = (o * nz + z) * M2 + q
}

// ------------------------------------------------------ inverse along y
// A'[o][z][y][kx] = sum_jy B'[o][z][jy][kx] e^{+2 pi i f(jy) y / ny}; one block
// per (o, z) slab.
__global__ void k_idfty(const float2 *__restrict__ Bp, int ny, int m,
                        const float2 *__restrict__ ty, float2 *__restrict__ Ap)
{
    extern __shared__ float2 s_y[];
    const int M2 = 2 * m * m;
    float2 *s_b = s_y;               // [2m][m]
    const long slab = blockIdx.x;
    for (int e = threadIdx.x; e < M2; e += blockDim.x) s_b[e] = Bp[slab * M2 + e];
    __syncthreads();
    float2 *out = Ap + slab * ny * m;
    // two y per thread (y0, y0 + 1) share each spectral value
    const int npairs = (ny + 1) / 2;
    for (int e = threadIdx.x; e < npairs * m; e += blockDim.x) {
        const int yp = e / m, kx = e - yp * m;
        const int y0 = 2 * yp, y1 = y0 + 1 < ny ? y0 + 1 : y0;
        float2 acc0 = make_float2(0.0f, 0.0f), acc1 = make_float2(0.0f, 0.0f);
        for (int jy = 0; jy < 2 * m; ++jy) {
            const float2 b = s_b[jy * m + kx];
            const float2 *tw = ty + (long)jy * ny;
            const float2 p0 = cmul_tw(b, __ldg(tw + y0), 1.0f);
            const float2 p1 = cmul_tw(b, __ldg(tw + y1), 1.0f);
            acc0.x += p0.x;
            acc0.y += p0.y;
            acc1.x += p1.x;
            acc1.y += p1.y;
        }
        out[y0 * m + kx] = acc0;
        if (y0 + 1 < ny) out[(y0 + 1) * m + kx] = acc1;
    }
}

// ------------------------------- inverse along x + pointwise mix + GELU
// v'[o][p] = act( (1/N)[Re A'_0 + 2 sum_{kx>=1} Re(A'_kx e^{+2 pi i kx x/nx})]
//                 + sum_c W[o][c] v[c][p] + b[o] ); one block per (z, y) row.
template <int WMAX>
__global__ void k_layer_out(const float *__restrict__ v, const float2 *__restrict__ Ap,
                            const float *__restrict__ W, const float *__restrict__ b, int nx,
                            int rows, int m, int width, float invN, int act,
                            const float2 *__restrict__ tx, float *__restrict__ vout, int N)
{
    extern __shared__ float s_o[];
    float *s_w = s_o;                                   // [width][width]
    float *s_b = s_w + width * width;                   // [width]
    float2 *s_a = reinterpret_cast<float2 *>(s_b + width + (width & 1));   // [width][m]
    const int row = blockIdx.x;                         // z * ny + y
    for (int e = threadIdx.x; e < width * width; e += blockDim.x) s_w[e] = W[e];
    for (int e = threadIdx.x; e < width; e += blockDim.x) s_b[e] = b[e];
    for (int e = threadIdx.x; e < width * m; e += blockDim.x) {
        const int o = e / m, kx = e - o * m;
        const float2 a = Ap[((long)o * rows + row) * m + kx];
        const float s = (kx == 0 ? 1.0f : 2.0f) * invN;
        s_a[e] = make_float2(a.x * s, a.y * s);
    }
    __syncthreads();
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
        const long p = (long)row * nx + x;
        float u[WMAX];
#pragma unroll
        for (int c = 0; c < WMAX; ++c) u[c] = c < width ? v[(long)c * N + p] : 0.0f;
        float2 e[BVF_FNO_MAX_MODES];
#pragma unroll
        for (int k = 0; k < BVF_FNO_MAX_MODES; ++k)
            e[k] = k < m ? __ldg(tx + (long)k * nx + x) : make_float2(0.0f, 0.0f);
        for (int o = 0; o < width; ++o) {
            float acc = s_b[o];
            const float4 *w4 = reinterpret_cast<const float4 *>(s_w + o * width);
#pragma unroll
            for (int c = 0; c < WMAX; c += 4) {
                if (c < width) {
                    const float4 w = w4[c / 4];
                    acc = fmaf(w.x, u[c], acc);
                    acc = fmaf(w.y, u[c + 1], acc);
                    acc = fmaf(w.z, u[c + 2], acc);
                    acc = fmaf(w.w, u[c + 3], acc);
                }
            }
            const float2 *a = s_a + o * m;
#pragma unroll
            for (int k = 0; k < BVF_FNO_MAX_MODES; ++k) {
                if (k < m) {
                    const float2 ak = a[k];
                    acc = fmaf(ak.x, e[k].x, fmaf(-ak.y, e[k].y, acc));
                }
            }
            vout[(long)o * N + p] = act ? gelu(acc) : acc;
        }
    }
}

// ------------------------------------------- tensor-core tiles (TF32 x 3)
// Each FP32 operand of a tensor-core product is split into a TF32 head and a
// remainder, and a b is taken as a_lo b_hi + a_hi b_lo + a_hi b_hi (the
// three-product scheme of Ootomo and Yokota, 2022), which keeps FP32-level
// accuracy.  The head is x with its low 13 mantissa bits cleared (a TF32
// value exactly); the remainder x - head is exact in FP32, below 2^-10 |x|,
// and the tensor core reads it at TF32 precision (relative error 2^-10 at
// most), so each product is off by about 3 * 2^-20 of |a b|.
__device__ __forceinline__ void tf32_split(float x, uint32_t &hi, uint32_t &lo)
{
    hi = __float_as_uint(x) & 0xFFFFE000u;
    lo = __float_as_uint(x - __uint_as_float(hi));
}

// the three products of one K step: D (+)= A_lo B_hi + A_hi B_lo + A_hi B_hi
__device__ __forceinline__ void mma3_tc(uint32_t d, uint64_t ah, uint64_t al, uint64_t bh,
                                        uint64_t bl, uint32_t idesc, int acc)
{
    tc::mma(d, al, bh, idesc, acc);
    tc::mma(d, ah, bl, idesc, 1);
    tc::mma(d, ah, bh, idesc, 1);
}

// ------------------------------------------------ tcgen05 layer output
// The output of a Fourier layer (or of the lift) on 128-point tiles of one
// (z, y) row, points x = 128 t .. 128 t + 127:
//   D[x][o] = sum_c v[c][x] W[o][c] + sum_j T[j][x] S[j][o]     (TMEM)
//   vout[o][x] = act(D[x][o] + b[o])
// T[j][x] holds cos and sin of the kept kx at x (j = 2 kx, 2 kx + 1) and S
// the row's spectral pairs S[2 kx][o] = Re A'(o, kx) s_kx,
// S[2 kx + 1][o] = -Im A'(o, kx) s_kx with s_0 = 1/N and s_kx = 2/N: the
// real inverse DFT along x of the kept half spectrum.  The lift is the same
// product without the spectral term.
// Operands sit in shared memory in the canonical K-major layout: A = the
// tile's input channels (staged, split, each tile) and T (all x tiles of a
// row, staged once per block); B = W (once per block) and S (once per row).
// 256 threads: thread i stages point i mod 128 of its half of the channels
// and, in the epilogue, reads half of the output channels of that point.
struct RowTcLayout {
    int JP, nxt, sAh, sAl, sTh, sTl, sBh, sBl, sSh, sSl, sb, bar, tmem, bytes;
    __host__ __device__ RowTcLayout(int width, int kc, int m, int nx, bool spec)
    {
        JP = ((2 * m + 7) / 8) * 8;
        nxt = (nx + 127) / 128;
        const int a = 128 * kc * 4, t = spec ? nxt * 128 * JP * 4 : 0, bw = width * kc * 4,
                  s = spec ? width * JP * 4 : 0;
        sAh = 0;
        sAl = sAh + a;
        sTh = sAl + a;
        sTl = sTh + t;
        sBh = sTl + t;
        sBl = sBh + bw;
        sSh = sBl + bw;
        sSl = sSh + s;
        sb = sSl + s;
        bar = (sb + width * 4 + 15) & ~15;
        tmem = bar + 16;
        bytes = tmem + 16;
    }
};

template <int W, int KC>     // W output channels; input channels padded to KC (a multiple of 8)
__global__ void __launch_bounds__(256, 2)
k_row_tc(const float *__restrict__ vin, int cin, const float2 *__restrict__ Ap,
         const float *__restrict__ Wm, const float *__restrict__ b, int nx, int rows, int m,
         float invN, int act, const float2 *__restrict__ tx, float *__restrict__ vout, int N,
         int *flag)
{
    static_assert(W % 16 == 0 && W <= 64 && KC % 8 == 0, "tile shape");
    extern __shared__ __align__(128) unsigned char s_r[];
    const bool spec = Ap != nullptr;
    const RowTcLayout L(W, KC, m, nx, spec);
    const int JP = L.JP, nxt = L.nxt;
    unsigned char *sAh = s_r + L.sAh, *sAl = s_r + L.sAl, *sTh = s_r + L.sTh, *sTl = s_r + L.sTl,
                  *sBh = s_r + L.sBh, *sBl = s_r + L.sBl, *sSh = s_r + L.sSh, *sSl = s_r + L.sSl;
    float *sb = reinterpret_cast<float *>(s_r + L.sb);
    uint64_t *bar = reinterpret_cast<uint64_t *>(s_r + L.bar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(s_r + L.tmem);
    const int tid = threadIdx.x, warp = tid >> 5, pt = tid & 127, half = tid >> 7;
    constexpr int NCOLS = W <= 32 ? 32 : 64;
    // block-constant operands: W (zero beyond cin), T (zero beyond 2m and nx),
    // the zero rows j >= 2m of S, b
    for (int e = tid; e < W * KC; e += 256) {
        const int o = e / KC, c = e - o * KC;
        uint32_t h, l;
        tf32_split(c < cin ? Wm[(long)o * cin + c] : 0.0f, h, l);
        const uint32_t off = tc::kmaj_off(o, c, KC);
        *reinterpret_cast<uint32_t *>(sBh + off) = h;
        *reinterpret_cast<uint32_t *>(sBl + off) = l;
    }
    if (spec) {
        for (int e = tid; e < nxt * 128 * JP; e += 256) {
            const int t = e / (128 * JP), r = e - t * 128 * JP, xl = r / JP, j = r - xl * JP;
            const int x = 128 * t + xl;
            float val = 0.0f;
            if (j < 2 * m && x < nx) {
                const float2 c = tx[(long)(j >> 1) * nx + x];
                val = (j & 1) ? c.y : c.x;
            }
            uint32_t h, l;
            tf32_split(val, h, l);
            const uint32_t off = (uint32_t)(t * 128 * JP * 4) + tc::kmaj_off(xl, j, JP);
            *reinterpret_cast<uint32_t *>(sTh + off) = h;
            *reinterpret_cast<uint32_t *>(sTl + off) = l;
        }
        for (int e = tid; e < W * JP; e += 256) {
            const int o = e / JP, j = e - o * JP;
            if (j >= 2 * m) {
                const uint32_t off = tc::kmaj_off(o, j, JP);
                *reinterpret_cast<uint32_t *>(sSh + off) = 0u;
                *reinterpret_cast<uint32_t *>(sSl + off) = 0u;
            }
        }
    }
    for (int o = tid; o < W; o += 256) sb[o] = b[o];
    if (tid == 0) {
        bvf::tma::mbar_init(bar, 1);
        bvf::tma::mbar_init_fence();
    }
    if (warp == 0) {
        tc::alloc(tslot, NCOLS);
        tc::relinquish();
    }
    bvf::tma::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = *tslot;
    const uint32_t idesc = tc::idesc_tf32(128, W);
    constexpr int CH = KC / 2;                  // channels a thread stages
    constexpr uint32_t SBO_A = (KC / 4) * 128;
    const uint32_t sbo_t = (uint32_t)(JP / 4) * 128;
    // this thread's channels of its point of a tile, loaded one tile ahead
    float xr[CH];
    auto load_v = [&](int row, int t) {
        const int x = 128 * t + pt;
        const bool ok = x < nx;
        const long p = (long)row * nx + x;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int ch = half * CH + c;
            xr[c] = (ok && ch < cin) ? vin[(long)ch * N + p] : 0.0f;
        }
    };
    // the (o, kx) pairs of A' this thread converts, loaded one row ahead
    constexpr int PRE = (W * BVF_FNO_MAX_MODES + 255) / 256;
    float2 pre[PRE];
    auto load_pairs = [&](int row) {
#pragma unroll
        for (int i = 0; i < PRE; ++i) {
            const int e = tid + i * 256;
            if (e < W * m) {
                const int o = e / m, kx = e - o * m;
                pre[i] = Ap[((long)o * rows + row) * m + kx];
            }
        }
    };
    int row = blockIdx.x, t = 0, it = 0;
    if (row < rows) {
        load_v(row, 0);
        if (spec) load_pairs(row);
    }
    bool gave_up = false;
    while (row < rows) {
        // stage the tile's channels (and, for a new row, its spectral pairs)
#pragma unroll
        for (int c4 = 0; c4 < CH / 4; ++c4) {
            uint32_t h[4], l[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) tf32_split(xr[4 * c4 + q], h[q], l[q]);
            const uint32_t off = tc::kmaj_off(pt, half * CH + 4 * c4, KC);
            *reinterpret_cast<uint4 *>(sAh + off) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4 *>(sAl + off) = make_uint4(l[0], l[1], l[2], l[3]);
        }
        if (spec && t == 0) {
#pragma unroll
            for (int i = 0; i < PRE; ++i) {
                const int e = tid + i * 256;
                if (e < W * m) {
                    const int o = e / m, kx = e - o * m;
                    const float sc = (kx == 0 ? 1.0f : 2.0f) * invN;
                    uint32_t h0, l0, h1, l1;
                    tf32_split(pre[i].x * sc, h0, l0);
                    tf32_split(-pre[i].y * sc, h1, l1);
                    const uint32_t off = tc::kmaj_off(o, 2 * kx, JP);
                    *reinterpret_cast<uint2 *>(sSh + off) = make_uint2(h0, h1);
                    *reinterpret_cast<uint2 *>(sSl + off) = make_uint2(l0, l1);
                }
            }
        }
        bvf::tma::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after();
#pragma unroll
            for (int ks = 0; ks < KC / 8; ++ks) {
                const uint32_t ko = ks * 2 * 128;      // two core matrices per K step of 8
                mma3_tc(tbase, tc::smem_desc(sAh + ko, 128, SBO_A),
                        tc::smem_desc(sAl + ko, 128, SBO_A), tc::smem_desc(sBh + ko, 128, SBO_A),
                        tc::smem_desc(sBl + ko, 128, SBO_A), idesc, ks > 0);
            }
            if (spec) {
                const uint32_t to = (uint32_t)(t * 128 * JP * 4);
                for (int ks = 0; ks < JP / 8; ++ks) {
                    const uint32_t ko = ks * 2 * 128;
                    mma3_tc(tbase, tc::smem_desc(sTh + to + ko, 128, sbo_t),
                            tc::smem_desc(sTl + to + ko, 128, sbo_t),
                            tc::smem_desc(sSh + ko, 128, sbo_t), tc::smem_desc(sSl + ko, 128, sbo_t),
                            idesc, 1);
                }
            }
            tc::commit(bar);
        }
        // the next tile's loads overlap the products and this tile's epilogue
        int nrow = row, nt = t + 1;
        if (nt == nxt) {
            nt = 0;
            nrow = row + gridDim.x;
        }
        if (nrow < rows) {
            load_v(nrow, nt);
            if (spec && nt == 0) load_pairs(nrow);
        }
        const bool ready =
            __all_sync(0xffffffffu, bvf::tma::mbar_wait(bar, it & 1, bvf::tma::kWaitLimit));
        tc::fence_after();
        if (ready) {
            const int x = 128 * t + pt;
            const long p = (long)row * nx + x;
#pragma unroll
            for (int c0 = 0; c0 < W / 2; c0 += 8) {
                float r[8];
                tc::ld8(tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(half * (W / 2) + c0),
                        r);
                tc::wait_ld();
                if (x < nx) {
#pragma unroll
                    for (int i = 0; i < 8; i += 2) {
                        const int o = half * (W / 2) + c0 + i;
                        float2 val = make_float2(r[i] + sb[o], r[i + 1] + sb[o + 1]);
                        if (act) val = gelu2(val);
                        vout[(long)o * N + p] = val.x;
                        vout[(long)(o + 1) * N + p] = val.y;
                    }
                }
            }
        }
        tc::fence_before();
        // tensor memory and the staged operands are free again; every thread
        // learns whether some warp's wait for the products ran out
        gave_up = __syncthreads_or(!ready) != 0;
        // after a time-out no further product is issued: the block waits,
        // bounded, for the products in flight, frees its tensor memory and
        // ends (the flag makes bvf_fno_synchronize report it)
        if (gave_up) break;
        row = nrow;
        t = nt;
        ++it;
    }
    if (gave_up && tid == 0) {
        bvf::tma::mbar_wait(bar, it & 1, bvf::tma::kWaitLimit);
        atomicOr(flag, 2);
    }
    tc::fence_after();
    __syncthreads();
    if (warp == 0) tc::dealloc(tbase, NCOLS);
}

// ------------------------------------------------ tcgen05 forward x transform
// A[i][kx] = sum_x v[i][x] e^{-2 pi i kx x / nx} for every row i = (c, z, y)
// of v (row-major, nx per row) as one tall product on 128-row tiles:
//   D[i][j] = sum_x v[i][x] T[j][x],  A[i][kx] = (D[i][2 kx], -D[i][2 kx + 1])
// with T[j][x] = cos, sin (2 pi kx x / nx) for j = 2 kx, 2 kx + 1 (zero rows
// up to NB, a multiple of 16).  x runs in chunks of 16 through two staged
// buffers (A, split, K-major); T is resident, split, for the whole row.  The
// next chunk's loads are issued before the current chunk is staged.
constexpr int kDxC = 16;     // x per chunk

struct DftxTcLayout {
    int nxp, sA, sB, bar, tmem, bytes;
    __host__ __device__ DftxTcLayout(int nb, int nx)
    {
        nxp = ((nx + kDxC - 1) / kDxC) * kDxC;
        const int a = 128 * kDxC * 4;                // one split half of one stage
        sA = 0;                                      // [stage][hi, lo]
        sB = sA + 4 * a;                             // [hi, lo] of NB x nxp
        bar = sB + 2 * nb * nxp * 4;
        tmem = bar + 16;
        bytes = tmem + 16;
    }
};

template <int NB, bool VEC>     // NB: T rows (16 or 32); VEC: rows start on 16 bytes (nx % 4 == 0)
__global__ void __launch_bounds__(256, 2)
k_dftx_tc(const float *__restrict__ v, long R, int nx, int m, const float2 *__restrict__ tx,
          float2 *__restrict__ A, int *flag)
{
    extern __shared__ __align__(128) unsigned char s_d[];
    const DftxTcLayout L(NB, nx);
    const int nxp = L.nxp, nch = nxp / kDxC;
    unsigned char *sA = s_d + L.sA, *sBh = s_d + L.sB, *sBl = sBh + NB * nxp * 4;
    uint64_t *bar = reinterpret_cast<uint64_t *>(s_d + L.bar);     // one per stage
    uint32_t *tslot = reinterpret_cast<uint32_t *>(s_d + L.tmem);
    constexpr int SA = 128 * kDxC * 4;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int e = tid; e < NB * nxp; e += 256) {
        const int j = e / nxp, x = e - j * nxp;
        float val = 0.0f;
        if (j < 2 * m && x < nx) {
            const float2 c = tx[(long)(j >> 1) * nx + x];
            val = (j & 1) ? c.y : c.x;
        }
        uint32_t h, l;
        tf32_split(val, h, l);
        const uint32_t off = tc::kmaj_off(j, x, nxp);
        *reinterpret_cast<uint32_t *>(sBh + off) = h;
        *reinterpret_cast<uint32_t *>(sBl + off) = l;
    }
    if (tid == 0) {
        bvf::tma::mbar_init(&bar[0], 1);
        bvf::tma::mbar_init(&bar[1], 1);
        bvf::tma::mbar_init_fence();
    }
    if (warp == 0) {
        tc::alloc(tslot, 32);
        tc::relinquish();
    }
    bvf::tma::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = *tslot;
    const uint32_t idesc = tc::idesc_tf32(128, NB);
    constexpr uint32_t SBO_A = (kDxC / 4) * 128;
    const uint32_t sbo_b = (uint32_t)(nxp / 4) * 128;
    // warp w stages rows 16 w .. 16 w + 15 of a chunk: 8 rows by 4 groups of
    // 4 x per access (512 contiguous bytes in shared memory)
    const int r_lo = 16 * warp + (lane & 7), kg = lane >> 3;
    const long tiles = (R + 127) / 128;
    auto load = [&](long tile, int ch, float4 (&dst)[2]) {
        const int x = ch * kDxC + 4 * kg;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const long i = tile * 128 + r_lo + 8 * q;
            const float *src = v + i * nx + x;
            if (VEC) {
                dst[q] = (i < R && x < nx) ? *reinterpret_cast<const float4 *>(src)
                                           : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            } else {
                const bool ok = i < R;
                dst[q] = make_float4(ok && x < nx ? src[0] : 0.0f, ok && x + 1 < nx ? src[1] : 0.0f,
                                     ok && x + 2 < nx ? src[2] : 0.0f,
                                     ok && x + 3 < nx ? src[3] : 0.0f);
            }
        }
    };
    float4 cur[2], nxt[2];
    long tile = blockIdx.x;
    if (tile < tiles) load(tile, 0, cur);
    int gc = 0;                 // chunks issued by this block
    bool gave_up = false;
    for (; tile < tiles && !gave_up; tile += gridDim.x) {
        for (int ch = 0; ch < nch; ++ch, ++gc) {
            long ntile = tile;
            int nc = ch + 1;
            if (nc == nch) {
                nc = 0;
                ntile = tile + gridDim.x;
            }
            if (ntile < tiles) load(ntile, nc, nxt);
            const int st = gc & 1;
            // the products that read this stage two chunks ago are done
            bool ok = true;
            if (gc >= 2)
                ok = __all_sync(0xffffffffu, bvf::tma::mbar_wait(&bar[st], ((gc - 2) >> 1) & 1,
                                                                 bvf::tma::kWaitLimit));
            tc::fence_after();
            unsigned char *ah = sA + st * 2 * SA, *al = ah + SA;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                uint32_t h[4], l[4];
                tf32_split(cur[q].x, h[0], l[0]);
                tf32_split(cur[q].y, h[1], l[1]);
                tf32_split(cur[q].z, h[2], l[2]);
                tf32_split(cur[q].w, h[3], l[3]);
                const uint32_t off = tc::kmaj_off(r_lo + 8 * q, 4 * kg, kDxC);
                *reinterpret_cast<uint4 *>(ah + off) = make_uint4(h[0], h[1], h[2], h[3]);
                *reinterpret_cast<uint4 *>(al + off) = make_uint4(l[0], l[1], l[2], l[3]);
            }
            bvf::tma::fence_async_smem();
            tc::fence_before();
            if (__syncthreads_or(!ok)) {
                gave_up = true;
                break;
            }
            if (tid == 0) {
                tc::fence_after();
#pragma unroll
                for (int ks = 0; ks < kDxC / 8; ++ks) {
                    const uint32_t ko = ks * 2 * 128, kb = (ch * (kDxC / 8) + ks) * 2 * 128;
                    mma3_tc(tbase, tc::smem_desc(ah + ko, 128, SBO_A),
                            tc::smem_desc(al + ko, 128, SBO_A), tc::smem_desc(sBh + kb, 128, sbo_b),
                            tc::smem_desc(sBl + kb, 128, sbo_b), idesc, ch > 0 || ks > 0);
                }
                tc::commit(&bar[st]);
            }
            cur[0] = nxt[0];
            cur[1] = nxt[1];
        }
        if (gave_up) break;
        // epilogue: the tile's last chunk is done, so is every product of it
        const int lst = (gc - 1) & 1;
        const bool ready = __all_sync(
            0xffffffffu, bvf::tma::mbar_wait(&bar[lst], ((gc - 1) >> 1) & 1, bvf::tma::kWaitLimit));
        tc::fence_after();
        if (ready) {
            const int half = tid >> 7;
            const long i = tile * 128 + (tid & 127);
#pragma unroll
            for (int c0 = 0; c0 < NB / 2; c0 += 8) {
                float r[8];
                tc::ld8(tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(half * (NB / 2) + c0),
                        r);
                tc::wait_ld();
                if (i < R) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int kx = (half * (NB / 2) + c0) / 2 + q;
                        if (kx < m) A[i * m + kx] = make_float2(r[2 * q], -r[2 * q + 1]);
                    }
                }
            }
        }
        tc::fence_before();
        gave_up = __syncthreads_or(!ready) != 0;
    }
    // after a time-out no further product is issued: wait, bounded, for the
    // last one issued, free tensor memory, flag it
    if (gave_up && tid == 0) {
        if (gc > 0)
            bvf::tma::mbar_wait(&bar[(gc - 1) & 1], ((gc - 1) >> 1) & 1, bvf::tma::kWaitLimit);
        atomicOr(flag, 2);
    }
    tc::fence_after();
    __syncthreads();
    if (warp == 0) tc::dealloc(tbase, 32);
}

// tcgen05 helpers (descriptors, TMEM, products): bvf_tc.cuh

// ------------------------------------------------ tcgen05 projection
// out[k][p] = q2[k] + sum_j Q2[k][j] GELU(q1[j] + sum_c Q1[j][c] v[c][p]) on
// 128-point tiles: D[128 points][HP hidden] = A[128][W] B[W][HP] in TMEM, as
// three TF32 products (A_lo B_hi + A_hi B_lo + A_hi B_hi) per K step of 8.
// 128 threads: thread i owns point i of the tile (A staging and epilogue).
struct ProjTcLayout {
    int HP, ncols, sAh, sAl, sBh, sBl, sq1, sq2, sred, bar, tmem, bytes;
    __host__ __device__ ProjTcLayout(int width, int hidden, int c_out)
    {
        HP = (hidden + 15) & ~15;
        ncols = 32;
        while (ncols < HP) ncols *= 2;
        const int a = 128 * width * 4, b = HP * width * 4;
        sAh = 0;
        sAl = sAh + a;
        sBh = sAl + a;
        sBl = sBh + b;
        sq1 = sBl + b;
        sq2 = sq1 + HP * 4;
        sred = sq2 + c_out * HP * 4;
        bar = (sred + c_out * 128 * 4 + 15) & ~15;
        tmem = bar + 16;
        bytes = tmem + 16;
    }
};

template <int W, int COUT>     // COUT: output count rounded up to 1 or 8
__global__ void __launch_bounds__(256, 2)
k_project_tc(const float *__restrict__ v, const float *__restrict__ Q1, const float *__restrict__ q1,
             const float *__restrict__ Q2, const float *__restrict__ q2, int hidden, int c_out,
             float *__restrict__ out, int N, int *flag)
{
    extern __shared__ __align__(128) unsigned char s_t[];
    const ProjTcLayout L(W, hidden, COUT);
    const int HP = L.HP;
    unsigned char *sAh = s_t + L.sAh, *sAl = s_t + L.sAl, *sBh = s_t + L.sBh, *sBl = s_t + L.sBl;
    float *sq1 = reinterpret_cast<float *>(s_t + L.sq1), *sq2 = reinterpret_cast<float *>(s_t + L.sq2);
    float *sred = reinterpret_cast<float *>(s_t + L.sred);     // [COUT][128] second-half sums
    uint64_t *bar = reinterpret_cast<uint64_t *>(s_t + L.bar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(s_t + L.tmem);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int pt = tid & 127, half = tid >> 7;   // point of the tile; channel / column half
    // B = Q1 as [HP rows][W] K-major, split; q1, Q2 (zero beyond hidden)
    for (int e = tid; e < HP * W; e += 256) {
        const int j = e / W, c = e - j * W;
        const float w = j < hidden ? Q1[(long)j * W + c] : 0.0f;
        uint32_t h, l;
        tf32_split(w, h, l);
        const uint32_t off = tc::kmaj_off(j, c, W);
        *reinterpret_cast<uint32_t *>(sBh + off) = h;
        *reinterpret_cast<uint32_t *>(sBl + off) = l;
    }
    for (int j = tid; j < HP; j += 256) sq1[j] = j < hidden ? q1[j] : 0.0f;
    for (int e = tid; e < COUT * HP; e += 256) {
        const int k = e / HP, j = e - k * HP;
        sq2[e] = (k < c_out && j < hidden) ? Q2[(long)k * hidden + j] : 0.0f;
    }
    if (tid == 0) {
        bvf::tma::mbar_init(bar, 1);
        bvf::tma::mbar_init_fence();
    }
    if (warp == 0) {
        tc::alloc(tslot, L.ncols);
        tc::relinquish();
    }
    bvf::tma::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = *tslot;
    constexpr int KS = W / 8, CH = W / 2;      // K steps; channels staged per thread
    const uint32_t idesc = tc::idesc_tf32(128, HP);
    const uint32_t sbo = (W / 4) * 128;
    const long tiles = ((long)N + 127) / 128;
    // this thread's channels of its point, loaded one tile ahead
    float xr[CH];
    auto load = [&](long tile) {
        const long p = tile * 128 + pt;
        const bool ok = p < N;
#pragma unroll
        for (int c = 0; c < CH; ++c) xr[c] = ok ? v[(long)(half * CH + c) * N + p] : 0.0f;
    };
    if ((long)blockIdx.x < tiles) load(blockIdx.x);
    int it = 0;
    bool gave_up = false;
    for (long tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++it) {
        const long p = tile * 128 + pt;
#pragma unroll
        for (int c4 = 0; c4 < CH / 4; ++c4) {
            uint32_t h[4], l[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) tf32_split(xr[4 * c4 + q], h[q], l[q]);
            const uint32_t off = tc::kmaj_off(pt, half * CH + 4 * c4, W);
            *reinterpret_cast<uint4 *>(sAh + off) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4 *>(sAl + off) = make_uint4(l[0], l[1], l[2], l[3]);
        }
        bvf::tma::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after();
#pragma unroll
            for (int ks = 0; ks < KS; ++ks) {
                const uint32_t ko = ks * 2 * 128;      // two core matrices per K step of 8
                const uint64_t ah = tc::smem_desc(sAh + ko, 128, sbo);
                const uint64_t al = tc::smem_desc(sAl + ko, 128, sbo);
                const uint64_t bh = tc::smem_desc(sBh + ko, 128, sbo);
                const uint64_t bl = tc::smem_desc(sBl + ko, 128, sbo);
                tc::mma(tbase, al, bh, idesc, ks > 0);
                tc::mma(tbase, ah, bl, idesc, 1);
                tc::mma(tbase, ah, bh, idesc, 1);
            }
            tc::commit(bar);
        }
        // the next tile's loads overlap the products and this tile's epilogue
        if (tile + gridDim.x < tiles) load(tile + gridDim.x);
        // a warp reads tensor memory only when all its lanes saw the commit
        const bool ready =
            __all_sync(0xffffffffu, bvf::tma::mbar_wait(bar, it & 1, bvf::tma::kWaitLimit));
        tc::fence_after();
        float o[COUT];
#pragma unroll
        for (int k = 0; k < COUT; ++k) o[k] = 0.0f;
        if (ready) {
            // 32-column chunks alternate between the two warp halves
            for (int c0 = 32 * half; c0 < HP; c0 += 64) {
                float r[32];
                tc::ld32(tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c0, r);
                tc::wait_ld();
                const int nv = min(32, HP - c0);
#pragma unroll
                for (int i = 0; i < 32; i += 2) {      // nv is a multiple of 16
                    if (i < nv) {
                        const float2 h =
                            gelu2(make_float2(r[i] + sq1[c0 + i], r[i + 1] + sq1[c0 + i + 1]));
#pragma unroll
                        for (int k = 0; k < COUT; ++k) {
                            o[k] = fmaf(sq2[k * HP + c0 + i], h.x, o[k]);
                            o[k] = fmaf(sq2[k * HP + c0 + i + 1], h.y, o[k]);
                        }
                    }
                }
            }
        }
        if (half) {
#pragma unroll
            for (int k = 0; k < COUT; ++k) sred[k * 128 + pt] = o[k];
        }
        tc::fence_before();
        // TMEM, the A buffers and sred are settled; every thread learns
        // whether some warp's wait for the products ran out
        gave_up = __syncthreads_or(!ready) != 0;
        if (!half && p < N) {
#pragma unroll
            for (int k = 0; k < COUT; ++k)
                if (k < c_out) out[(long)k * N + p] = q2[k] + o[k] + sred[k * 128 + pt];
        }
        // after a time-out no further product is issued: the block waits,
        // bounded, for the products in flight, frees its tensor memory and
        // ends (the flag makes bvf_fno_synchronize report it)
        if (gave_up) break;
    }
    if (gave_up && tid == 0) {
        bvf::tma::mbar_wait(bar, it & 1, bvf::tma::kWaitLimit);
        atomicOr(flag, 2);
    }
    tc::fence_after();
    __syncthreads();
    if (warp == 0) tc::dealloc(tbase, L.ncols);
}

// --------------------------------------------------------------- features
struct FeatTable {
    float f[BVF_MAX_MATERIALS][3];     // cL/cL_w - 1, rho/rho_w - 1, alphaL cL_w / f0
};

__global__ void k_features(const uint8_t *__restrict__ idx, const __grid_constant__ FeatTable tab,
                           int nx, int ny, int nz, int k_src, const float2 *__restrict__ src,
                           float inv_p, float *__restrict__ out)
{
    const long N = (long)nx * ny * nz;
    const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    const int i = (int)(p % nx);
    const long r = p / nx;
    const int j = (int)(r % ny), k = (int)(r / ny);
    const int mat = idx[p];
    out[p] = tab.f[mat][0];
    out[N + p] = tab.f[mat][1];
    out[2 * N + p] = tab.f[mat][2];
    float sr = 0.0f, si = 0.0f;
    if (k == k_src) {
        const float2 s = src[(long)j * nx + i];
        sr = s.x * inv_p;
        si = s.y * inv_p;
    }
    out[3 * N + p] = sr;
    out[4 * N + p] = si;
    out[5 * N + p] = ((float)i + 0.5f) / (float)nx;
    out[6 * N + p] = ((float)j + 0.5f) / (float)ny;
    out[7 * N + p] = ((float)k + 0.5f) / (float)nz;
}

}  // namespace

// ================================================================== context
struct bvf_fno {
    bvf_fno_dims d{};
    float *w = nullptr;                      // device copy of the blob
    size_t n_w = 0;
    int *flag = nullptr;                     // device: bit 1 = a bounded wait ran out
    // grid-dependent state
    int nx = 0, ny = 0, nz = 0;
    float2 *tw = nullptr;                    // twiddle tables [m][nx], [2m][ny], [2m][nz]
    size_t tw_cap = 0;
    float *v0 = nullptr, *v1 = nullptr;
    size_t v_cap = 0;
    float2 *A = nullptr, *B = nullptr, *H = nullptr, *G = nullptr;
    size_t a_cap = 0, b_cap = 0, h_cap = 0;
    // stage timing
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_stage;
    int n_ev = 0;
    cudaStream_t last_stream = nullptr;
};

namespace {

void free_ws(bvf_fno *f)
{
    cudaFree(f->tw);
    cudaFree(f->v0);
    cudaFree(f->v1);
    cudaFree(f->A);
    cudaFree(f->B);
    cudaFree(f->H);
    cudaFree(f->G);
    f->tw = nullptr;
    f->v0 = f->v1 = nullptr;
    f->A = f->B = f->H = f->G = nullptr;
    f->tw_cap = f->v_cap = f->a_cap = f->b_cap = f->h_cap = 0;
    f->nx = f->ny = f->nz = 0;
}

template <typename T>
int grow(T **p, size_t *cap, size_t n, const char *what)
{
    if (n <= *cap) return BVF_OK;
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    FCK(cudaMalloc(p, n * sizeof(T)), what);
    *cap = n;
    return BVF_OK;
}

// e^{+2 pi i f j / n} for j < n and each signed frequency f of `freqs`
// (FP64 angle, reduced exactly as (f j mod n) / n before the multiplication)
void mode_table(std::vector<float2> &t, const std::vector<int> &freqs, int n)
{
    for (int f : freqs)
        for (int j = 0; j < n; ++j) {
            const long r = (((long)f * j) % n + n) % n;
            const double a = kTwoPi * (double)r / (double)n;
            t.push_back(make_float2((float)std::cos(a), (float)std::sin(a)));
        }
}

int prepare_grid(bvf_fno *f, int nx, int ny, int nz)
{
    if (f->nx == nx && f->ny == ny && f->nz == nz) return BVF_OK;
    const int m = f->d.modes, W = f->d.width;
    const size_t N = (size_t)nx * ny * nz;
    const size_t M2 = (size_t)2 * m * m;
    int rc;
    // buffers of an earlier grid may still be in use on some stream
    FCK(cudaDeviceSynchronize(), "bvf_fno_forward: sync before a grid change");
    if ((size_t)W * N > f->v_cap) {
        cudaFree(f->v0);
        cudaFree(f->v1);
        f->v0 = f->v1 = nullptr;
        f->v_cap = 0;
        FCK(cudaMalloc(&f->v0, (size_t)W * N * sizeof(float)), "workspace v0");
        FCK(cudaMalloc(&f->v1, (size_t)W * N * sizeof(float)), "workspace v1");
        f->v_cap = (size_t)W * N;
    }
    if ((rc = grow(&f->A, &f->a_cap, (size_t)W * nz * ny * m, "workspace A")) != BVF_OK) return rc;
    if ((rc = grow(&f->B, &f->b_cap, (size_t)W * nz * M2, "workspace B")) != BVF_OK) return rc;
    const size_t hn = (size_t)W * 2 * m * M2;      // H and G: the kept spectrum
    if (hn > f->h_cap) {
        cudaFree(f->H);
        cudaFree(f->G);
        f->H = f->G = nullptr;
        f->h_cap = 0;
        FCK(cudaMalloc(&f->H, hn * sizeof(float2)), "workspace H");
        FCK(cudaMalloc(&f->G, hn * sizeof(float2)), "workspace G");
        f->h_cap = hn;
    }
    // twiddle tables: [m][nx] for kx = 0 .. m-1, [2m][ny] and [2m][nz] for the
    // signed slots of y and z
    std::vector<int> fx(m), fs(2 * m);
    for (int k = 0; k < m; ++k) fx[k] = k;
    for (int j = 0; j < 2 * m; ++j) fs[j] = slot_freq(j, m);
    std::vector<float2> t;
    t.reserve((size_t)m * nx + (size_t)2 * m * (ny + nz));
    mode_table(t, fx, nx);
    mode_table(t, fs, ny);
    mode_table(t, fs, nz);
    if ((rc = grow(&f->tw, &f->tw_cap, t.size(), "twiddle table")) != BVF_OK) return rc;
    FCK(cudaMemcpy(f->tw, t.data(), t.size() * sizeof(float2), cudaMemcpyHostToDevice),
        "twiddle upload");
    f->nx = nx;
    f->ny = ny;
    f->nz = nz;
    return BVF_OK;
}

}  // namespace

namespace {
// A kernel's dynamic shared-memory limit, raised only when a launch needs more
// than any earlier one (per process), so that repeated inferences on a grid
// make no runtime call besides their launches and can be recorded in a graph.
// The record is keyed by the kernel itself (a template argument), not by its
// type: instantiations of one kernel template share a signature but each has
// its own limit.
template <auto Kernel>
cudaError_t smem_at_least(size_t bytes)
{
    static std::atomic<size_t> cur{0};
    size_t have = cur.load(std::memory_order_acquire);
    if (bytes <= have) return cudaSuccess;
    const cudaError_t e =
        cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
        while (have < bytes && !cur.compare_exchange_weak(have, bytes)) {
        }
    return e;
}

template <int W, int KC>
cudaError_t launch_row_tc_k(int grid, int bytes, cudaStream_t s, const float *vin, int cin,
                            const float2 *Ap, const float *Wm, const float *bm, int nx, int rows,
                            int m, float invN, int act, const float2 *tx, float *vout, int N,
                            int *flag)
{
    cudaError_t e = smem_at_least<k_row_tc<W, KC>>((size_t)bytes);
    if (e != cudaSuccess) return e;
    k_row_tc<W, KC><<<grid, 256, bytes, s>>>(vin, cin, Ap, Wm, bm, nx, rows, m, invN, act, tx,
                                             vout, N, flag);
    return cudaGetLastError();
}

// input channels padded to 8 or 16 (the lift) or to W (a Fourier layer)
template <int W>
cudaError_t launch_row_tc(int kc, int grid, int bytes, cudaStream_t s, const float *vin, int cin,
                          const float2 *Ap, const float *Wm, const float *bm, int nx, int rows,
                          int m, float invN, int act, const float2 *tx, float *vout, int N,
                          int *flag)
{
    if (kc == 8)
        return launch_row_tc_k<W, 8>(grid, bytes, s, vin, cin, Ap, Wm, bm, nx, rows, m, invN, act,
                                     tx, vout, N, flag);
    if (kc == 16 || W == 16)
        return launch_row_tc_k<W, 16>(grid, bytes, s, vin, cin, Ap, Wm, bm, nx, rows, m, invN,
                                      act, tx, vout, N, flag);
    return launch_row_tc_k<W, W>(grid, bytes, s, vin, cin, Ap, Wm, bm, nx, rows, m, invN, act,
                                 tx, vout, N, flag);
}

template <int NB, bool VEC>
cudaError_t launch_dftx_tc(int grid, int bytes, cudaStream_t s, const float *v, long R, int nx,
                           int m, const float2 *tx, float2 *A, int *flag)
{
    cudaError_t e = smem_at_least<k_dftx_tc<NB, VEC>>((size_t)bytes);
    if (e != cudaSuccess) return e;
    k_dftx_tc<NB, VEC><<<grid, 256, bytes, s>>>(v, R, nx, m, tx, A, flag);
    return cudaGetLastError();
}
}  // namespace

extern "C" {

size_t bvf_fno_weight_count(const bvf_fno_dims *d)
{
    if (!dims_valid(d)) return 0;
    return (size_t)d->width * d->c_in + d->width + (size_t)d->n_layers * layer_floats(*d) +
           (size_t)d->hidden * d->width + d->hidden + (size_t)d->c_out * d->hidden + d->c_out;
}

int bvf_fno_create(bvf_fno **out, const bvf_fno_dims *d, const float *h_weights, size_t n)
{
    if (!out) return fno_fail(BVF_E_ARG, "bvf_fno_create: out is NULL");
    *out = nullptr;
    if (!dims_valid(d)) return fno_fail(BVF_E_ARG, "bvf_fno_create: dimensions out of range");
    if (!h_weights) return fno_fail(BVF_E_ARG, "bvf_fno_create: weights are NULL");
    if (n != bvf_fno_weight_count(d))
        return fno_fail(BVF_E_ARG, "bvf_fno_create: weight count does not match the layout");
    bvf_fno *f = new bvf_fno;
    f->d = *d;
    f->n_w = n;
    cudaError_t e = cudaMalloc(&f->w, n * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(f->w, h_weights, n * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&f->flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(f->flag, 0, sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(f->w);
        cudaFree(f->flag);
        delete f;
        return fno_cuda(e, "bvf_fno_create: weights");
    }
    *out = f;
    return BVF_OK;
}

int bvf_fno_destroy(bvf_fno *f)
{
    if (!f) return BVF_OK;
    cudaDeviceSynchronize();
    for (cudaEvent_t e : f->ev) cudaEventDestroy(e);
    free_ws(f);
    cudaFree(f->w);
    cudaFree(f->flag);
    delete f;
    return BVF_OK;
}

int bvf_fno_synchronize(bvf_fno *f, void *stream)
{
    if (!f) return fno_fail(BVF_E_ARG, "bvf_fno_synchronize: NULL surrogate");
    FCK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)), "bvf_fno_synchronize");
    int h = 0;
    FCK(cudaMemcpy(&h, f->flag, sizeof(int), cudaMemcpyDeviceToHost), "bvf_fno_synchronize");
    if (h) {
        FCK(cudaMemset(f->flag, 0, sizeof(int)), "bvf_fno_synchronize");
        return fno_fail(BVF_E_CUDA, "bvf_fno_synchronize: a tensor-core completion wait ran out");
    }
    return BVF_OK;
}

int bvf_fno_timing(bvf_fno *f, int enable)
{
    if (!f) return fno_fail(BVF_E_ARG, "bvf_fno_timing: NULL surrogate");
    f->timing = enable != 0;
    f->n_ev = 0;
    return BVF_OK;
}

int bvf_fno_stage_times(bvf_fno *f, double *ms_out)
{
    if (!f || !ms_out) return fno_fail(BVF_E_ARG, "bvf_fno_stage_times: NULL argument");
    for (int s = 0; s < BVF_FNO_STAGES; ++s) ms_out[s] = 0.0;
    if (!f->timing || f->n_ev < 2) return BVF_OK;
    FCK(cudaEventSynchronize(f->ev[f->n_ev - 1]), "bvf_fno_stage_times");
    for (int i = 1; i < f->n_ev; ++i) {
        float ms = 0.0f;
        FCK(cudaEventElapsedTime(&ms, f->ev[i - 1], f->ev[i]), "bvf_fno_stage_times");
        ms_out[f->ev_stage[i]] += ms;
    }
    return BVF_OK;
}


int bvf_fno_forward(bvf_fno *f, int nx, int ny, int nz, const float *d_in, float *d_out,
                    void *stream)
{
    if (!f || !d_in || !d_out) return fno_fail(BVF_E_ARG, "bvf_fno_forward: NULL argument");
    const bvf_fno_dims &d = f->d;
    const int m = d.modes, W = d.width;
    if (nx < 1 || ny < 1 || nz < 1 || nx > 1024 || ny > 1024 || nz > 4096)
        return fno_fail(BVF_E_ARG, "bvf_fno_forward: grid sizes out of range");
    if (m > nx / 2 || 2 * m > ny || 2 * m > nz)
        return fno_fail(BVF_E_ARG, "bvf_fno_forward: grid too small for the kept modes");
    const long long N64 = (long long)nx * ny * nz;
    if (N64 >= (1LL << 31)) return fno_fail(BVF_E_ARG, "bvf_fno_forward: nx*ny*nz >= 2^31");
    const size_t in_bytes = (size_t)d.c_in * N64 * sizeof(float);
    const size_t out_bytes = (size_t)d.c_out * N64 * sizeof(float);
    const char *ib = reinterpret_cast<const char *>(d_in), *ob = reinterpret_cast<const char *>(d_out);
    if (ib < ob + out_bytes && ob < ib + in_bytes)
        return fno_fail(BVF_E_ARG, "bvf_fno_forward: input and output overlap");
    int rc = prepare_grid(f, nx, ny, nz);
    if (rc != BVF_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    f->last_stream = s;
    const int N = (int)N64;
    const int M2 = 2 * m * m, n_modes = 2 * m * M2;
    const float2 *tx = f->tw, *ty = tx + (size_t)m * nx, *tz = ty + (size_t)2 * m * ny;

    // stage events
    const int n_ev_need = 2 + 7 * d.n_layers + 1;
    if (f->timing) {
        while ((int)f->ev.size() < n_ev_need) {
            cudaEvent_t e;
            FCK(cudaEventCreate(&e), "bvf_fno_forward: event");
            f->ev.push_back(e);
        }
        f->ev_stage.assign(n_ev_need, 0);
        f->n_ev = 0;
        FCK(cudaEventRecord(f->ev[f->n_ev++], s), "bvf_fno_forward: event");
    }
    auto mark = [&](int stage) -> cudaError_t {
        if (!f->timing) return cudaSuccess;
        f->ev_stage[f->n_ev] = stage;
        return cudaEventRecord(f->ev[f->n_ev++], s);
    };

    // weight offsets
    const float *Wp = f->w, *bp = Wp + (size_t)W * d.c_in;
    const float *lay0 = bp + W;
    const size_t lf = layer_floats(d);
    const float *proj = lay0 + d.n_layers * lf;
    const float *Q1 = proj, *q1 = Q1 + (size_t)d.hidden * W, *Q2 = q1 + d.hidden,
                *q2 = Q2 + (size_t)d.c_out * d.hidden;

    const int TB = 256;
    const int pblocks = (N + TB - 1) / TB;
    const int rows_p = nz * ny;
    const float invN = (float)(1.0 / (double)N64);
    // the row pass: k_row_tc (layer output: inverse x transform, W v + b,
    // GELU) and, when a further layer follows, k_dftx_tc (its forward x
    // transform); grids whose rows do not fit shared memory take the unfused
    // kernels
    const int kc_lift = ((d.c_in + 7) / 8) * 8;
    const int nb = 2 * m <= 16 ? 16 : 32;
    const DftxTcLayout dl(nb, nx);
    constexpr int kSmemCap = 200 * 1024;
    const bool fused = RowTcLayout(W, W, m, nx, true).bytes <= kSmemCap &&
                       RowTcLayout(W, kc_lift, m, nx, false).bytes <= kSmemCap &&
                       dl.bytes <= kSmemCap;
    int dev = 0, n_sm = 0;
    FCK(cudaGetDevice(&dev), "bvf_fno_forward: device");
    FCK(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev), "sm count");
    // resident blocks per SM: two where shared memory allows (launch bounds)
    auto blocks_per_sm = [](int bytes) {
        return std::max(1, std::min(2, (227 * 1024) / (bytes + 1024)));
    };
    auto row_pass = [&](const float *vin, int cin, const float2 *Ap, const float *Wm,
                        const float *bm, int act, float *vout, float2 *An) -> cudaError_t {
        const int kc = Ap ? W : kc_lift;
        const RowTcLayout rl(W, kc, m, nx, Ap != nullptr);
        const int grid = std::min(rows_p, n_sm * blocks_per_sm(rl.bytes));
        cudaError_t e;
#define BVF_ROW(WW)                                                                            \
    e = launch_row_tc<WW>(kc, grid, rl.bytes, s, vin, cin, Ap, Wm, bm, nx, rows_p, m, invN, act, \
                          tx, vout, N, f->flag)
        switch (W) {
        case 16: BVF_ROW(16); break;
        case 32: BVF_ROW(32); break;
        case 48: BVF_ROW(48); break;
        default: BVF_ROW(64); break;
        }
#undef BVF_ROW
        if (e != cudaSuccess || !An) return e;
        const long R = (long)W * rows_p, tiles = (R + 127) / 128;
        const int g2 = (int)std::min<long>(tiles, (long)n_sm * blocks_per_sm(dl.bytes));
        const bool vec = nx % 4 == 0;
        if (nb == 16)
            return vec ? launch_dftx_tc<16, true>(g2, dl.bytes, s, vout, R, nx, m, tx, An, f->flag)
                       : launch_dftx_tc<16, false>(g2, dl.bytes, s, vout, R, nx, m, tx, An, f->flag);
        return vec ? launch_dftx_tc<32, true>(g2, dl.bytes, s, vout, R, nx, m, tx, An, f->flag)
                   : launch_dftx_tc<32, false>(g2, dl.bytes, s, vout, R, nx, m, tx, An, f->flag);
    };

    if (fused) {
        FCK(row_pass(d_in, d.c_in, nullptr, Wp, bp, 0, f->v0, f->A), "bvf_fno_forward: lift");
    } else {
        k_lift<<<pblocks, TB, (W * d.c_in + W) * sizeof(float), s>>>(d_in, d.c_in, W, Wp, bp,
                                                                      f->v0, N);
        FCK(cudaGetLastError(), "bvf_fno_forward: lift");
    }
    FCK(mark(0), "event");

    const size_t sy = (size_t)ny * m * sizeof(float2);
    FCK(smem_at_least<k_dfty>(sy),
        "bvf_fno_forward: dfty smem");
    const size_t s_out = ((size_t)W * W + W + 1) * sizeof(float) + (size_t)W * m * sizeof(float2);
    const int rows_x = W * nz * ny;
    const int bo = std::min(256, ((nx + 31) / 32) * 32);

    float *vc = f->v0, *vn = f->v1;
    for (int l = 0; l < d.n_layers; ++l) {
        const float *lw = lay0 + l * lf;
        const float2 *R = reinterpret_cast<const float2 *>(lw);
        const float *Wl = lw + (size_t)n_modes * W * W * 2, *bl = Wl + (size_t)W * W;
        if (!fused) {
            k_dftx<<<(rows_x + kXT - 1) / kXT, m * (kXT / kXR), 0, s>>>(vc, rows_x, nx, m, tx,
                                                                       f->A);
            FCK(cudaGetLastError(), "bvf_fno_forward: dftx");
        }
        FCK(mark(1), "event");
        k_dfty<<<W * nz, std::max(32, ((m * m + 31) / 32) * 32), sy, s>>>(f->A, ny, m, ty, f->B);
        FCK(cudaGetLastError(), "bvf_fno_forward: dfty");
        FCK(mark(2), "event");
        const long nh = (long)W * 2 * m * M2;
        k_dftz<<<(unsigned)((nh + TB - 1) / TB), TB, 0, s>>>(f->B, nz, m, W, tz, f->H);
        FCK(cudaGetLastError(), "bvf_fno_forward: dftz");
        FCK(mark(3), "event");
        const dim3 mb(W, 256 / W);
        k_mix<<<(n_modes + mb.y - 1) / mb.y, mb, mb.y * W * sizeof(float2), s>>>(f->H, R, W,
                                                                                 n_modes, f->G);
        FCK(cudaGetLastError(), "bvf_fno_forward: mix");
        FCK(mark(4), "event");
        const long nb = (long)W * nz * M2;
        k_idftz<<<(unsigned)((nb + TB - 1) / TB), TB, 0, s>>>(f->G, nz, m, W, tz, f->B);
        FCK(cudaGetLastError(), "bvf_fno_forward: idftz");
        FCK(mark(5), "event");
        k_idfty<<<W * nz, TB, (size_t)M2 * sizeof(float2), s>>>(f->B, ny, m, ty, f->A);
        FCK(cudaGetLastError(), "bvf_fno_forward: idfty");
        FCK(mark(6), "event");
        const int act = l < d.n_layers - 1;
        if (fused) {
            FCK(row_pass(vc, W, f->A, Wl, bl, act, vn, act ? f->A : nullptr),
                "bvf_fno_forward: row pass");
        } else {
            if (W <= 16)
                k_layer_out<16><<<rows_p, bo, s_out, s>>>(vc, f->A, Wl, bl, nx, rows_p, m, W, invN,
                                                         act, tx, vn, N);
            else if (W <= 32)
                k_layer_out<32><<<rows_p, bo, s_out, s>>>(vc, f->A, Wl, bl, nx, rows_p, m, W, invN,
                                                         act, tx, vn, N);
            else
                k_layer_out<64><<<rows_p, bo, s_out, s>>>(vc, f->A, Wl, bl, nx, rows_p, m, W, invN,
                                                         act, tx, vn, N);
            FCK(cudaGetLastError(), "bvf_fno_forward: layer_out");
        }
        FCK(mark(7), "event");
        std::swap(vc, vn);
    }
    {
        const int cp = d.c_out == 1 ? 1 : 8;
        const ProjTcLayout pl(W, d.hidden, cp);
        const long tiles = (N64 + 127) / 128;
        const int per_sm = std::max(1, std::min(2, 512 / pl.ncols));
        const int grid = (int)std::min<long>(tiles, (long)n_sm * per_sm);
        cudaError_t e = cudaSuccess;
#define BVF_PRJ(WW, CP)                                                                      \
    e = smem_at_least<k_project_tc<WW, CP>>((size_t)pl.bytes);                                 \
    if (e == cudaSuccess)                                                                      \
        k_project_tc<WW, CP><<<grid, 256, pl.bytes, s>>>(vc, Q1, q1, Q2, q2, d.hidden, d.c_out, \
                                                        d_out, N, f->flag);
        if (cp == 1) {
            switch (W) {
            case 16: BVF_PRJ(16, 1) break;
            case 32: BVF_PRJ(32, 1) break;
            case 48: BVF_PRJ(48, 1) break;
            default: BVF_PRJ(64, 1) break;
            }
        } else {
            switch (W) {
            case 16: BVF_PRJ(16, 8) break;
            case 32: BVF_PRJ(32, 8) break;
            case 48: BVF_PRJ(48, 8) break;
            default: BVF_PRJ(64, 8) break;
            }
        }
#undef BVF_PRJ
        FCK(e, "bvf_fno_forward: project smem");
    }
    FCK(cudaGetLastError(), "bvf_fno_forward: project");
    FCK(mark(8), "event");
    return BVF_OK;
}

int bvf_fno_features(const uint8_t *d_index, const bvf_material *h_table, int n_mat,
                     const bvf_material *h_water, int nx, int ny, int nz, double f0, int k_src,
                     const float *d_src, double p_norm, float *d_out, void *stream)
{
    if (!d_index || !h_table || !h_water || !d_src || !d_out)
        return fno_fail(BVF_E_ARG, "bvf_fno_features: NULL argument");
    if (nx < 1 || ny < 1 || nz < 1 || (long long)nx * ny * nz >= (1LL << 31))
        return fno_fail(BVF_E_ARG, "bvf_fno_features: bad grid");
    if (n_mat < 1 || n_mat > BVF_MAX_MATERIALS)
        return fno_fail(BVF_E_ARG, "bvf_fno_features: n_mat out of range");
    if (k_src < 0 || k_src >= nz) return fno_fail(BVF_E_ARG, "bvf_fno_features: k_src outside the grid");
    if (!(p_norm > 0.0) || !(f0 > 0.0))
        return fno_fail(BVF_E_ARG, "bvf_fno_features: p_norm and f0 must be positive");
    if (!(h_water->rho > 0.0) || !(h_water->cL > 0.0))
        return fno_fail(BVF_E_MATERIAL, "bvf_fno_features: water row needs rho, cL > 0");
    FeatTable tab;
    std::memset(&tab, 0, sizeof(tab));
    for (int i = 0; i < n_mat; ++i) {
        tab.f[i][0] = (float)(h_table[i].cL / h_water->cL - 1.0);
        tab.f[i][1] = (float)(h_table[i].rho / h_water->rho - 1.0);
        tab.f[i][2] = (float)(h_table[i].alphaL * h_water->cL / f0);
    }
    const long N = (long)nx * ny * nz;
    k_features<<<(unsigned)((N + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        d_index, tab, nx, ny, nz, k_src, reinterpret_cast<const float2 *>(d_src),
        (float)(1.0 / p_norm), d_out);
    FCK(cudaGetLastError(), "bvf_fno_features");
    return BVF_OK;
}

}  // extern "C"
