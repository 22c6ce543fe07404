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
//   - one row pass per (z, y) row does the inverse x transform, W v + b and
//     GELU as one tensor-core product, keeps the new row in shared memory
//     and takes the next layer's forward x transform from it, so v is read
//     and written once per layer (k_row_mma, mma.sync TF32);
//   - the lift is the same row pass without the spectral term.
// The projection runs on the fifth-generation tensor cores (k_project_tc:
// tcgen05.mma into TMEM, tcgen05.ld epilogue with GELU).  Every product uses
// the three-term TF32 split, which keeps FP32 accuracy.  Rows too long for
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
// mma.sync m16n8k8 with TF32 operands and FP32 accumulation.  Each FP32
// operand is split into a TF32 head and the TF32 rounding of its remainder,
// and a b is taken as a_lo b_hi + a_hi b_lo + a_hi b_hi (the three-product
// scheme of Ootomo and Yokota, 2022), which keeps FP32-level accuracy.
// Fragment layout (lane = 4 g + t): A rows g, g+8 and columns t, t+4;
// B rows t, t+4 and column g; C/D rows g, g+8 and columns 2t, 2t+1.
__device__ __forceinline__ uint32_t tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void tf32_split(float x, uint32_t &hi, uint32_t &lo)
{
    hi = tf32_rna(x);
    lo = tf32_rna(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// d += a b in three products (small terms first)
__device__ __forceinline__ void mma3(float (&d)[4], const uint32_t (&ah)[4],
                                     const uint32_t (&al)[4], uint32_t bh0, uint32_t bh1,
                                     uint32_t bl0, uint32_t bl1)
{
    mma_tf32(d, al, bh0, bh1);
    mma_tf32(d, ah, bl0, bl1);
    mma_tf32(d, ah, bh0, bh1);
}

// ------------------------------------------------ tensor-core row pass
// The row pass above as two tensor-core products per (z, y) row:
//   phase 2: D[x][o] = sum_k X[x][k] Y[k][o], X = [v[c][x] | cos, sin of the
//            kept kx at x], Y = [W^T ; (Re A', -Im A') s_kx], s_0 = 1/N,
//            s_kx = 2/N, plus b, then GELU;
//   phase 3: Anext[o][kx] = sum_x v'[o][x] (cos - i sin)(kx x 2 pi / nx),
//            a product over x of the new row (shared memory) and the table.
// Persistent blocks keep the split twiddle table T[j][x] (j = 2 kx for cos,
// 2 kx + 1 for sin, zero rows up to a multiple of 8) and the split W; each
// row brings its own spectral rows of Y.  Pitches: P = 8 mod 32 for [.][x]
// arrays and PW = 8 mod 32 for [k][o] arrays.
struct RowMmaLayout {
    int P, PW, JP, sTh, sTl, sWh, sWl, sSh, sSl, sV, sb, words;
    __host__ __device__ RowMmaLayout(int ksw, int cout, int m, int nx)
    {
        const int nx16 = (nx + 15) & ~15;
        P = nx16 + ((8 - nx16 % 32) + 32) % 32;
        PW = cout + ((8 - cout % 32) + 32) % 32;
        JP = ((2 * m + 7) / 8) * 8;
        sTh = 0;
        sTl = sTh + JP * P;
        sWh = sTl + JP * P;
        sWl = sWh + 8 * ksw * PW;
        sSh = sWl + 8 * ksw * PW;
        sSl = sSh + JP * PW;
        sV = sSl + JP * PW;
        sb = sV + cout * P;
        words = sb + cout;
    }
};

template <int NT, int KSW>     // cout = 8 NT output channels; input channels padded to 8 KSW
__global__ void __launch_bounds__(256, 2)
k_row_mma(const float *__restrict__ vin, int cin, const float2 *Ap, const float *__restrict__ W,
          const float *__restrict__ b, int nx, int rows, int m, float invN, int act,
          const float2 *__restrict__ tx, float *__restrict__ vout, float2 *Anext, int N)
{
    constexpr int cout = 8 * NT;
    extern __shared__ __align__(16) uint32_t s_m[];
    const RowMmaLayout L(KSW, cout, m, nx);
    const int P = L.P, PW = L.PW, JP = L.JP, KSS = JP / 8;
    const int nx16 = (nx + 15) & ~15;
    uint32_t *sTh = s_m + L.sTh, *sTl = s_m + L.sTl, *sWh = s_m + L.sWh, *sWl = s_m + L.sWl,
             *sSh = s_m + L.sSh, *sSl = s_m + L.sSl;
    float *sV = reinterpret_cast<float *>(s_m + L.sV), *sb = reinterpret_cast<float *>(s_m + L.sb);
    const int tid = threadIdx.x, nth = blockDim.x;
    const bool spec = Ap != nullptr, fwd = Anext != nullptr;
    // block-constant operands
    if (spec || fwd) {
        for (int j = 0; j < JP; ++j)
            for (int x = tid; x < P; x += nth) {
                float val = 0.0f;
                if (j < 2 * m && x < nx) {
                    const float2 e = tx[(long)(j >> 1) * nx + x];
                    val = (j & 1) ? e.y : e.x;
                }
                tf32_split(val, sTh[j * P + x], sTl[j * P + x]);
            }
    }
    for (int k = 0; k < 8 * KSW; ++k)
        for (int o = tid; o < PW; o += nth) {
            const float w = (k < cin && o < cout) ? W[(long)o * cin + k] : 0.0f;
            tf32_split(w, sWh[k * PW + o], sWl[k * PW + o]);
        }
    for (int o = tid; o < cout; o += nth) sb[o] = b[o];

    const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    // rows j >= 2m and columns o >= cout of the spectral part of Y stay zero
    if (spec) {
        for (int e = tid; e < JP * PW; e += nth) {
            const int j = e / PW, o = e - j * PW;
            if (j >= 2 * m || o >= cout) tf32_split(0.0f, sSh[e], sSl[e]);
        }
    }
    // the (o, kx) pairs of A' a thread converts, loaded one row ahead
    constexpr int PRE = (8 * NT * BVF_FNO_MAX_MODES + 255) / 256;
    float2 pre[PRE];
    auto load_pairs = [&](int r) {
#pragma unroll
        for (int i = 0; i < PRE; ++i) {
            const int e = tid + i * nth;
            if (e < cout * m) {
                const int o = e / m, kx = e - o * m;
                pre[i] = Ap[((long)o * rows + r) * m + kx];
            }
        }
    };
    if (spec && (int)blockIdx.x < rows) load_pairs(blockIdx.x);
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const long base = (long)row * nx;
        __syncthreads();          // the previous row is done with sS and sV
        if (spec) {
            // this row's spectral rows of Y from the pairs loaded one row ahead
#pragma unroll
            for (int i = 0; i < PRE; ++i) {
                const int e = tid + i * nth;
                if (e < cout * m) {
                    const int o = e / m, kx = e - o * m;
                    const float sc = (kx == 0 ? 1.0f : 2.0f) * invN;
                    tf32_split(pre[i].x * sc, sSh[(2 * kx) * PW + o], sSl[(2 * kx) * PW + o]);
                    tf32_split(-pre[i].y * sc, sSh[(2 * kx + 1) * PW + o],
                               sSl[(2 * kx + 1) * PW + o]);
                }
            }
            if (row + (int)gridDim.x < rows) load_pairs(row + gridDim.x);
        }
        __syncthreads();
        // phase 2: 16-point tiles of the row
        for (int mt = warp; mt < nx16 / 16; mt += nth / 32) {
            const int xa = 16 * mt + g, xb = xa + 8;
            float d[NT][4];
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const float b0 = sb[8 * nt + 2 * t], b1 = sb[8 * nt + 2 * t + 1];
                d[nt][0] = b0;
                d[nt][1] = b1;
                d[nt][2] = b0;
                d[nt][3] = b1;
            }
#pragma unroll
            for (int ks = 0; ks < KSW; ++ks) {
                const int c0 = 8 * ks + t, c1 = c0 + 4;
                uint32_t ah[4], al[4];
                const bool c0ok = c0 < cin, c1ok = c1 < cin;
                tf32_split(c0ok && xa < nx ? vin[(long)c0 * N + base + xa] : 0.0f, ah[0], al[0]);
                tf32_split(c0ok && xb < nx ? vin[(long)c0 * N + base + xb] : 0.0f, ah[1], al[1]);
                tf32_split(c1ok && xa < nx ? vin[(long)c1 * N + base + xa] : 0.0f, ah[2], al[2]);
                tf32_split(c1ok && xb < nx ? vin[(long)c1 * N + base + xb] : 0.0f, ah[3], al[3]);
                const uint32_t *wh = sWh + c0 * PW + g, *wl = sWl + c0 * PW + g;
#pragma unroll
                for (int nt = 0; nt < NT; ++nt)
                    mma3(d[nt], ah, al, wh[8 * nt], wh[4 * PW + 8 * nt], wl[8 * nt],
                         wl[4 * PW + 8 * nt]);
            }
            if (spec) {
                for (int ks = 0; ks < KSS; ++ks) {
                    const int j0 = 8 * ks + t;
                    const uint32_t ah[4] = {sTh[j0 * P + xa], sTh[j0 * P + xb],
                                            sTh[(j0 + 4) * P + xa], sTh[(j0 + 4) * P + xb]};
                    const uint32_t al[4] = {sTl[j0 * P + xa], sTl[j0 * P + xb],
                                            sTl[(j0 + 4) * P + xa], sTl[(j0 + 4) * P + xb]};
                    const uint32_t *yh = sSh + j0 * PW + g, *yl = sSl + j0 * PW + g;
#pragma unroll
                    for (int nt = 0; nt < NT; ++nt)
                        mma3(d[nt], ah, al, yh[8 * nt], yh[4 * PW + 8 * nt], yl[8 * nt],
                             yl[4 * PW + 8 * nt]);
                }
            }
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int o = 8 * nt + 2 * t + (i & 1), x = i < 2 ? xa : xb;
                    const float val = act ? gelu(d[nt][i]) : d[nt][i];
                    if (x < nx) vout[(long)o * N + base + x] = val;
                    if (fwd) sV[o * P + x] = x < nx ? val : 0.0f;
                }
            }
        }
        if (!fwd) continue;
        __syncthreads();
        // phase 3: forward x transform of the new row
        const int units = (cout / 16) * KSS;
        for (int u = warp; u < units; u += nth / 32) {
            const int o0 = 16 * (u / KSS), n0 = 8 * (u % KSS);
            float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            const float *va = sV + (o0 + g) * P + t, *vb = sV + (o0 + g + 8) * P + t;
            const uint32_t *th = sTh + (n0 + g) * P + t, *tl = sTl + (n0 + g) * P + t;
            for (int x0 = 0; x0 < nx16; x0 += 8) {
                uint32_t ah[4], al[4];
                tf32_split(va[x0], ah[0], al[0]);
                tf32_split(vb[x0], ah[1], al[1]);
                tf32_split(va[x0 + 4], ah[2], al[2]);
                tf32_split(vb[x0 + 4], ah[3], al[3]);
                mma3(d, ah, al, th[x0], th[x0 + 4], tl[x0], tl[x0 + 4]);
            }
            const int kx = n0 / 2 + t;
            if (kx < m) {
                Anext[((long)(o0 + g) * rows + row) * m + kx] = make_float2(d[0], -d[1]);
                Anext[((long)(o0 + g + 8) * rows + row) * m + kx] = make_float2(d[2], -d[3]);
            }
        }
    }
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
                for (int i = 0; i < 32; ++i) {
                    if (i < nv) {
                        const float h = gelu(r[i] + sq1[c0 + i]);
#pragma unroll
                        for (int k = 0; k < COUT; ++k) o[k] = fmaf(sq2[k * HP + c0 + i], h, o[k]);
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
    // the row pass keeps the twiddle table and one (z, y) row of every output
    // channel in shared memory; rows too long for that take the unfused kernels
    const int ksw_lift = (d.c_in + 7) / 8;
    const size_t row_bytes =
        (size_t)std::max(RowMmaLayout(W / 8, W, m, nx).words,
                         RowMmaLayout(ksw_lift, W, m, nx).words) * sizeof(uint32_t);
    const bool fused = row_bytes <= 110 * 1024;
    int dev = 0, n_sm = 0;
    FCK(cudaGetDevice(&dev), "bvf_fno_forward: device");
    FCK(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev), "sm count");
    const int row_grid = std::min(rows_p, 2 * n_sm);
    auto row_pass = [&](const float *vin, int cin, const float2 *Ap, const float *Wm,
                        const float *bm, int act, float *vout, float2 *An) -> cudaError_t {
        const int ksw = (cin + 7) / 8;
        const size_t bytes = (size_t)RowMmaLayout(ksw, W, m, nx).words * sizeof(uint32_t);
        cudaError_t e = cudaSuccess;
#define BVF_ROW(NT, KSW)                                                                     \
    e = smem_at_least<k_row_mma<NT, KSW>>(bytes);                                              \
    if (e == cudaSuccess)                                                                     \
        k_row_mma<NT, KSW><<<row_grid, 256, bytes, s>>>(vin, cin, Ap, Wm, bm, nx, rows_p, m,   \
                                                        invN, act, tx, vout, An, N);
        if (ksw == W / 8) {
            switch (W / 8) {
            case 2: BVF_ROW(2, 2) break;
            case 4: BVF_ROW(4, 4) break;
            case 6: BVF_ROW(6, 6) break;
            default: BVF_ROW(8, 8) break;
            }
        } else if (ksw == 1) {
            switch (W / 8) {
            case 2: BVF_ROW(2, 1) break;
            case 4: BVF_ROW(4, 1) break;
            case 6: BVF_ROW(6, 1) break;
            default: BVF_ROW(8, 1) break;
            }
        } else {
            switch (W / 8) {
            case 2: BVF_ROW(2, 2) break;
            case 4: BVF_ROW(4, 2) break;
            case 6: BVF_ROW(6, 2) break;
            default: BVF_ROW(8, 2) break;
            }
        }
#undef BVF_ROW
        return e != cudaSuccess ? e : cudaGetLastError();
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
