// BF16 path of the surrogate: inference and training of the Fourier neural
// operator (Li et al., ICLR 2021, Sec. 4; the network of include/bvf_fno.h)
// with every contraction on the tcgen05 BF16 product of bvf_gemm_bf16.cu
// (BF16 operands, FP32 accumulation) and FP32 master weights.
//
// Layouts (per sample b, channel c, voxel p = (z ny + y) nx + x):
//   volumes  [b][c][p];
//   spectra  [b][c][ky][kx][part][kz] with ky, kz the 2m signed slots, kx in
//            0 .. m-1, part 0 = real, 1 = imaginary (8 m^3 floats per channel).
// Forward transform of a layer (the kept modes of rfftn), three products:
//   x: rows (b, c, z, y) x nx  ->  [part][kx]      (cos, -sin)
//   y: rows (b, c, z, kx) x [part][y]  ->  [part][ky]   (e^{-i theta} as a
//      real 2 x 2 block)
//   z: rows (b, c, ky, kx) x [part][z]  ->  [part][kz]
// with axis permutes in between; the inverse (irfftn of the kept half
// spectrum) is the same chain backwards with e^{+i theta} and, on x, the
// weights c(kx)/N (c = 1 for kx = 0, 2 otherwise).  The mode mix (per mode a
// W x W complex matrix) is a small SIMT kernel.
//
// Backward (gradients of the loss below): the adjoint of the inverse is the
// forward transform with the weights c(kx)/N, the adjoint of the forward
// transform is the inverse without them, the mix's adjoints take conj(R);
// weight gradients are products summed over the batch and the voxels (split
// K, added atomically), bias gradients channel sums.  GELU's derivative is
// applied in the product epilogue from the stored pre-activation.
//
// Loss of a batch: the mean over samples of the relative L2 error
// ||out_0 - target|| / ||target|| of output channel 0, plus, when the net has
// a second output channel, el_weight times the mean squared error of that
// channel's spatial mean against the sample's transmission target.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/bvf_fno.h"
#include "bvf_internal.cuh"

namespace bvf {
cudaError_t launch_gemm_bf16(const bvf_gemm &g, int *flag, cudaStream_t s);
}

using bvf::launch_gemm_bf16;

namespace {

constexpr double kPi = 3.14159265358979323846;

int b16_fail(int code, const std::string &msg)
{
    bvf::set_context_free_error(msg.c_str());
    return code;
}

#define BCK(call, where)                                                           \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess)                                                     \
            return b16_fail(e_ == cudaErrorMemoryAllocation ? BVF_E_NOMEM : BVF_E_CUDA, \
                            std::string(where) + ": " + cudaGetErrorString(e_));   \
    } while (0)

__host__ __device__ __forceinline__ int slot_freq(int j, int m) { return j < m ? j : j - 2 * m; }

// out[p][c][q][a] = in[p][a][q][c]
__global__ void k_permute(const float *__restrict__ in, float *__restrict__ out, long long P, int A,
                          int Q, int C)
{
    const long long n = P * A * Q * C;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        // t indexes the output [p][c][q][a]
        const int a = (int)(t % A);
        long long r = t / A;
        const int q = (int)(r % Q);
        r /= Q;
        const int c = (int)(r % C);
        const long long p = r / C;
        out[t] = in[((p * A + a) * Q + q) * C + c];
    }
}

// spectrum position of mode (kz, ky, kx), part, in a channel's 8 m^3 floats
__device__ __forceinline__ int spec_pos(int kz, int ky, int kx, int part, int m)
{
    return ((ky * m + kx) * 2 + part) * (2 * m) + kz;
}

// Y[b][o][mode] = sum_c R[mode][c][o] X[b][c][mode]  (R: [kz][ky][kx][c][o][2])
__global__ void k_mix_fwd(const float *__restrict__ X, const float *__restrict__ R, int B, int W,
                          int m, float *__restrict__ Y)
{
    const int modes = 4 * m * m * m, S = 8 * m * m * m;
    const long long n = (long long)B * modes * W;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int o = (int)(t % W);
        const int mode = (int)((t / W) % modes);
        const int b = (int)(t / ((long long)W * modes));
        const int kx = mode % m, ky = (mode / m) % (2 * m), kz = mode / (2 * m * m);
        const int pr = spec_pos(kz, ky, kx, 0, m), pi = spec_pos(kz, ky, kx, 1, m);
        const float *Rm = R + (size_t)mode * W * W * 2;
        float yr = 0.0f, yi = 0.0f;
        for (int c = 0; c < W; ++c) {
            const float *xc = X + ((size_t)b * W + c) * S;
            const float xr = xc[pr], xi = xc[pi];
            const float rr = Rm[((size_t)c * W + o) * 2], ri = Rm[((size_t)c * W + o) * 2 + 1];
            yr = fmaf(rr, xr, fmaf(-ri, xi, yr));
            yi = fmaf(rr, xi, fmaf(ri, xr, yi));
        }
        float *yo = Y + ((size_t)b * W + o) * S;
        yo[pr] = yr;
        yo[pi] = yi;
    }
}

// dX[b][c][mode] = sum_o conj(R[mode][c][o]) dY[b][o][mode]
__global__ void k_mix_adj(const float *__restrict__ dY, const float *__restrict__ R, int B, int W,
                          int m, float *__restrict__ dX)
{
    const int modes = 4 * m * m * m, S = 8 * m * m * m;
    const long long n = (long long)B * modes * W;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t % W);
        const int mode = (int)((t / W) % modes);
        const int b = (int)(t / ((long long)W * modes));
        const int kx = mode % m, ky = (mode / m) % (2 * m), kz = mode / (2 * m * m);
        const int pr = spec_pos(kz, ky, kx, 0, m), pi = spec_pos(kz, ky, kx, 1, m);
        const float *Rc = R + ((size_t)mode * W + c) * W * 2;
        float xr = 0.0f, xi = 0.0f;
        for (int o = 0; o < W; ++o) {
            const float *yo = dY + ((size_t)b * W + o) * S;
            const float yr = yo[pr], yi = yo[pi];
            const float rr = Rc[2 * o], ri = Rc[2 * o + 1];
            xr = fmaf(rr, yr, fmaf(ri, yi, xr));
            xi = fmaf(rr, yi, fmaf(-ri, yr, xi));
        }
        float *xc = dX + ((size_t)b * W + c) * S;
        xc[pr] = xr;
        xc[pi] = xi;
    }
}

// dR[mode][c][o] += sum_b dY[b][o][mode] conj(X[b][c][mode])
__global__ void k_mix_dR(const float *__restrict__ dY, const float *__restrict__ X, int B, int W,
                         int m, float *__restrict__ dR)
{
    const int modes = 4 * m * m * m, S = 8 * m * m * m;
    const long long n = (long long)modes * W * W;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int o = (int)(t % W);
        const int c = (int)((t / W) % W);
        const int mode = (int)(t / ((long long)W * W));
        const int kx = mode % m, ky = (mode / m) % (2 * m), kz = mode / (2 * m * m);
        const int pr = spec_pos(kz, ky, kx, 0, m), pi = spec_pos(kz, ky, kx, 1, m);
        float gr = 0.0f, gi = 0.0f;
        for (int b = 0; b < B; ++b) {
            const float *yo = dY + ((size_t)b * W + o) * S;
            const float *xc = X + ((size_t)b * W + c) * S;
            const float yr = yo[pr], yi = yo[pi], xr = xc[pr], xi = xc[pi];
            gr = fmaf(yr, xr, fmaf(yi, xi, gr));
            gi = fmaf(yi, xr, fmaf(-yr, xi, gi));
        }
        dR[t * 2] += gr;
        dR[t * 2 + 1] += gi;
    }
}

// out[c] += sum over samples and voxels of x[b][c][p]
__global__ void k_chan_sum(const float *__restrict__ x, int B, int C, int N, float *__restrict__ out)
{
    const int c = blockIdx.y;
    float acc = 0.0f;
    for (int b = 0; b < B; ++b) {
        const float *xc = x + ((size_t)b * C + c) * N;
        for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x)
            acc += xc[p];
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ float sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0f;
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) atomicAdd(out + c, v);
    }
}

// per sample: [0] sum (out0 - y)^2, [1] sum y^2, [2] sum out1 (FP64)
__global__ void k_loss_sums(const float *__restrict__ out, const float *__restrict__ y, int c_out,
                            int N, double *__restrict__ sums)
{
    const int b = blockIdx.y;
    const float *o0 = out + (size_t)b * c_out * N, *yb = y + (size_t)b * N;
    double e = 0.0, t = 0.0, s1 = 0.0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
        const double d = (double)o0[p] - yb[p];
        e += d * d;
        t += (double)yb[p] * yb[p];
        if (c_out > 1) s1 += o0[N + p];
    }
    for (int o = 16; o; o >>= 1) {
        e += __shfl_xor_sync(0xffffffffu, e, o);
        t += __shfl_xor_sync(0xffffffffu, t, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(sums + 3 * b, e);
        atomicAdd(sums + 3 * b + 1, t);
        atomicAdd(sums + 3 * b + 2, s1);
    }
}

// d loss / d out for the loss of the file header (scale = 1 / batch)
__global__ void k_loss_grad(const float *__restrict__ out, const float *__restrict__ y,
                            const float *__restrict__ el, const double *__restrict__ sums, int B,
                            int c_out, int N, float el_weight, float *__restrict__ dout)
{
    const long long n = (long long)B * c_out * N;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(t % N);
        const int k = (int)((t / N) % c_out);
        const int b = (int)(t / ((long long)c_out * N));
        const double *s = sums + 3 * b;
        float g = 0.0f;
        if (k == 0) {
            const double rel = sqrt(s[0] / s[1]);
            g = rel > 0.0 ? (float)(((double)out[t] - y[(size_t)b * N + p]) / (rel * s[1] * B))
                          : 0.0f;
        } else if (k == 1 && el) {
            const double mean = s[2] / N;
            g = (float)(2.0 * el_weight * (mean - el[b]) / ((double)N * B));
        }
        dout[t] = g;
    }
}

// sum of n floats into *out (FP64)
__global__ void k_sum(const float *__restrict__ x, size_t n, double *__restrict__ out)
{
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        acc += x[i];
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m1,
                       float *__restrict__ m2, size_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float a = b1 * m1[i] + (1.0f - b1) * gi;
        const float v = b2 * m2[i] + (1.0f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = v;
        w[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
    }
}

inline unsigned grid_for(long long n)
{
    long long b = (n + 255) / 256;
    return (unsigned)std::max(1LL, std::min(b, 152LL * 32));
}

}  // namespace

struct bvf_fno_bf16 {
    bvf_fno_dims d{};
    int nx = 0, ny = 0, nz = 0, N = 0, Bmax = 0;
    size_t n_w = 0;
    float *w = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;
    long long adam_t = 0;
    // stage matrices: forward x (plain, weighted c/N), y, z; inverse z, y, x (weighted, plain)
    float *Fx = nullptr, *Fxw = nullptr, *Fy = nullptr, *Fz = nullptr;
    float *Gz = nullptr, *Gy = nullptr, *Gxw = nullptr, *Gx = nullptr;
    std::vector<float *> v, s, X;       // L+1 volumes, L-1 pre-activations, L spectra
    float *pre1 = nullptr, *h = nullptr, *out = nullptr;
    float *w1 = nullptr, *w2 = nullptr, *S1 = nullptr, *S2 = nullptr;
    float *dv = nullptr, *dv2 = nullptr, *dh = nullptr, *dout = nullptr;
    double *sums = nullptr;
    int *flag = nullptr;
    std::vector<void *> all;
    int ksplit = 1;                     // K split of the voxel-sum products
};

namespace {

size_t layer_floats(const bvf_fno_dims &d)
{
    const size_t m = d.modes, W = d.width;
    return (2 * m) * (2 * m) * m * W * W * 2 + W * W + W;      // R, W, b
}

struct Off {
    size_t Wp, bp, lay0, lf, Q1, q1, Q2, q2;
};
Off offsets(const bvf_fno_dims &d)
{
    Off o{};
    o.Wp = 0;
    o.bp = (size_t)d.width * d.c_in;
    o.lay0 = o.bp + d.width;
    o.lf = layer_floats(d);
    o.Q1 = o.lay0 + (size_t)d.n_layers * o.lf;
    o.q1 = o.Q1 + (size_t)d.hidden * d.width;
    o.Q2 = o.q1 + d.hidden;
    o.q2 = o.Q2 + (size_t)d.c_out * d.hidden;
    return o;
}

template <typename P>
int dalloc(bvf_fno_bf16 *t, P **p, size_t n, const char *what)
{
    cudaError_t e = cudaMalloc((void **)p, n * sizeof(P));
    if (e != cudaSuccess) return b16_fail(BVF_E_NOMEM, std::string("bvf_fno_bf16_create: ") + what);
    t->all.push_back(*p);
    return BVF_OK;
}

// stage matrices in FP64, rounded once to FP32
void build_matrices(int nx, int ny, int nz, int m, std::vector<std::vector<float>> &out)
{
    const double N = (double)nx * ny * nz;
    auto wk = [&](int kx) { return (kx == 0 ? 1.0 : 2.0) / N; };
    std::vector<float> Fx((size_t)nx * 2 * m), Fxw(Fx.size()), Gx((size_t)2 * m * nx), Gxw(Gx.size());
    for (int x = 0; x < nx; ++x)
        for (int kx = 0; kx < m; ++kx) {
            const double ph = 2.0 * kPi * kx * x / nx, c = std::cos(ph), s = std::sin(ph);
            Fx[(size_t)x * 2 * m + kx] = (float)c;
            Fx[(size_t)x * 2 * m + m + kx] = (float)(-s);
            Fxw[(size_t)x * 2 * m + kx] = (float)(wk(kx) * c);
            Fxw[(size_t)x * 2 * m + m + kx] = (float)(-wk(kx) * s);
            Gx[(size_t)kx * nx + x] = (float)c;
            Gx[(size_t)(m + kx) * nx + x] = (float)(-s);
            Gxw[(size_t)kx * nx + x] = (float)(wk(kx) * c);
            Gxw[(size_t)(m + kx) * nx + x] = (float)(-wk(kx) * s);
        }
    // complex stage along an axis of length n over the 2m slots, forward
    // (e^{-i theta}, K = [part][n] -> N = [part][slot]) and inverse
    // (e^{+i theta}, K = [part][slot] -> N = [part][n])
    auto axis = [&](int n, std::vector<float> &F, std::vector<float> &G) {
        const int S = 2 * m;
        F.assign((size_t)2 * n * 2 * S, 0.0f);
        G.assign((size_t)2 * S * 2 * n, 0.0f);
        for (int q = 0; q < n; ++q)
            for (int j = 0; j < S; ++j) {
                const double th = 2.0 * kPi * slot_freq(j, m) * q / n, c = std::cos(th), s = std::sin(th);
                // forward: re' = a cos + b sin, im' = b cos - a sin
                F[(size_t)q * 2 * S + j] = (float)c;
                F[(size_t)q * 2 * S + S + j] = (float)(-s);
                F[(size_t)(n + q) * 2 * S + j] = (float)s;
                F[(size_t)(n + q) * 2 * S + S + j] = (float)c;
                // inverse: re' = a cos - b sin, im' = b cos + a sin
                G[(size_t)j * 2 * n + q] = (float)c;
                G[(size_t)j * 2 * n + n + q] = (float)s;
                G[(size_t)(S + j) * 2 * n + q] = (float)(-s);
                G[(size_t)(S + j) * 2 * n + n + q] = (float)c;
            }
    };
    std::vector<float> Fy, Gy, Fz, Gz;
    axis(ny, Fy, Gy);
    axis(nz, Fz, Gz);
    out = {Fx, Fxw, Fy, Fz, Gz, Gy, Gxw, Gx};
}

// C[rows][N] = A[rows][K] B[K][N] (all row-major, B shared)
bvf_gemm rowmajor(const float *A, const float *B, float *C, long long rows, int K, int N)
{
    bvf_gemm g{};
    g.A = A;
    g.sam = K;
    g.sak = 1;
    g.B = B;
    g.sbk = N;
    g.sbn = 1;
    g.C = C;
    g.scm = N;
    g.scn = 1;
    g.M = (int)rows;
    g.N = N;
    g.K = K;
    g.batch = 1;
    g.ksplit = 1;
    g.alpha = 1.0f;
    return g;
}

int gemm(bvf_fno_bf16 *t, const bvf_gemm &g, cudaStream_t s, const char *what)
{
    BCK(launch_gemm_bf16(g, t->flag, s), what);
    return BVF_OK;
}

int permute(const float *in, float *out, long long P, int A, int Q, int C, cudaStream_t s)
{
    k_permute<<<grid_for(P * A * Q * C), 256, 0, s>>>(in, out, P, A, Q, C);
    BCK(cudaGetLastError(), "permute");
    return BVF_OK;
}

// forward transform of BC real volumes -> BC spectra (weighted: the x stage
// carries c(kx)/N, the adjoint of the inverse)
int spec_fwd(bvf_fno_bf16 *t, const float *in, long long BC, bool weighted, float *S, cudaStream_t s)
{
    const int nx = t->nx, ny = t->ny, nz = t->nz, m = t->d.modes;
    int rc;
    if ((rc = gemm(t, rowmajor(in, weighted ? t->Fxw : t->Fx, t->w1, BC * nz * ny, nx, 2 * m), s,
                   "spectral x")) != BVF_OK)
        return rc;
    if ((rc = permute(t->w1, t->w2, BC * nz, ny, 2, m, s)) != BVF_OK) return rc;
    if ((rc = gemm(t, rowmajor(t->w2, t->Fy, t->w1, BC * nz * m, 2 * ny, 4 * m), s, "spectral y")) !=
        BVF_OK)
        return rc;
    if ((rc = permute(t->w1, t->w2, BC, nz, 2 * m, 2 * m, s)) != BVF_OK) return rc;
    return gemm(t, rowmajor(t->w2, t->Fz, S, BC * 2 * m * m, 2 * nz, 4 * m), s, "spectral z");
}

// inverse transform of BC spectra into BC real volumes: out = beta out +
// Inv(S) (weighted: c(kx)/N, the real inverse of the kept half spectrum;
// plain: the adjoint of the forward transform), then act (2: times GELU'(pre))
int spec_inv(bvf_fno_bf16 *t, const float *S, long long BC, bool weighted, float *out, float beta,
             int act, const float *pre, cudaStream_t s)
{
    const int nx = t->nx, ny = t->ny, nz = t->nz, m = t->d.modes;
    int rc;
    if ((rc = gemm(t, rowmajor(S, t->Gz, t->w1, BC * 2 * m * m, 4 * m, 2 * nz), s, "inverse z")) !=
        BVF_OK)
        return rc;
    if ((rc = permute(t->w1, t->w2, BC, 2 * m, 2 * m, nz, s)) != BVF_OK) return rc;
    if ((rc = gemm(t, rowmajor(t->w2, t->Gy, t->w1, BC * nz * m, 4 * m, 2 * ny), s, "inverse y")) !=
        BVF_OK)
        return rc;
    if ((rc = permute(t->w1, t->w2, BC * nz, m, 2, ny, s)) != BVF_OK) return rc;
    bvf_gemm g = rowmajor(t->w2, weighted ? t->Gxw : t->Gx, out, BC * nz * ny, 2 * m, nx);
    g.beta = beta;
    g.act = act;
    g.C_pre = const_cast<float *>(pre);
    return gemm(t, g, s, "inverse x");
}

// channel mix out[b][o][p] (+)= sum_c Wt[o][c] in[b][c][p] (Wt row-major [O][C])
bvf_gemm chan(const float *in, int C, const float *Wt, float *out, int O, int N, int B)
{
    bvf_gemm g{};
    g.A = in;
    g.sam = 1;
    g.sak = N;
    g.sab = (long long)C * N;
    g.B = Wt;
    g.sbk = 1;
    g.sbn = C;
    g.sbb = 0;
    g.C = out;
    g.scm = 1;
    g.scn = N;
    g.scb = (long long)O * N;
    g.M = N;
    g.N = O;
    g.K = C;
    g.batch = B;
    g.ksplit = 1;
    g.alpha = 1.0f;
    return g;
}

// transposed channel mix out[b][c][p] = sum_o Wt[o][c] din[b][o][p]
bvf_gemm chanT(const float *din, int O, const float *Wt, float *out, int C, int N, int B)
{
    bvf_gemm g = chan(din, O, Wt, out, C, N, B);
    g.sbk = C;          // B(k = o, n = c) = Wt[o][c]
    g.sbn = 1;
    return g;
}

// weight gradient G[o][c] += sum_{b,p} d[b][o][p] x[b][c][p]
bvf_gemm wgrad(const float *d, int O, const float *x, int C, float *G, int N, int B, int ksplit)
{
    bvf_gemm g{};
    g.A = d;
    g.sam = N;
    g.sak = 1;
    g.sab = (long long)O * N;
    g.B = x;
    g.sbk = 1;
    g.sbn = N;
    g.sbb = (long long)C * N;
    g.C = G;
    g.scm = C;
    g.scn = 1;
    g.scb = 0;
    g.M = O;
    g.N = C;
    g.K = N;
    g.batch = B;
    g.ksplit = std::max(2, ksplit);   // the batch shares G: always the atomic path
    g.alpha = 1.0f;
    g.beta = 1.0f;
    return g;
}

int chan_sum(const float *x, int B, int C, int N, float *out, cudaStream_t s)
{
    k_chan_sum<<<dim3(std::min(64, (N + 255) / 256), C), 256, 0, s>>>(x, B, C, N, out);
    BCK(cudaGetLastError(), "channel sum");
    return BVF_OK;
}

// forward pass of `batch` samples into `out` ([batch][c_out][N]); with `keep`
// every activation the backward pass needs is kept, without it (inference)
// the pre-activations are not written
int forward(bvf_fno_bf16 *t, int batch, const float *in, float *out, bool keep, cudaStream_t s)
{
    const bvf_fno_dims &d = t->d;
    const int W = d.width, N = t->N, L = d.n_layers, m = d.modes;
    const Off o = offsets(d);
    const float *w = t->w;
    int rc;
    bvf_gemm g = chan(in, d.c_in, w + o.Wp, t->v[0], W, N, batch);
    g.bias = w + o.bp;
    g.bias_mode = 1;
    if ((rc = gemm(t, g, s, "lift")) != BVF_OK) return rc;
    for (int l = 0; l < L; ++l) {
        const float *lw = w + o.lay0 + l * o.lf;
        const float *R = lw, *Wl = lw + (size_t)4 * m * m * m * W * W * 2, *bl = Wl + (size_t)W * W;
        if ((rc = spec_fwd(t, t->v[l], (long long)batch * W, false, t->X[l], s)) != BVF_OK) return rc;
        k_mix_fwd<<<grid_for((long long)batch * 4 * m * m * m * W), 256, 0, s>>>(t->X[l], R, batch, W,
                                                                                   m, t->S1);
        BCK(cudaGetLastError(), "mix");
        if ((rc = spec_inv(t, t->S1, (long long)batch * W, true, t->v[l + 1], 0.0f, 0, nullptr, s)) !=
            BVF_OK)
            return rc;
        bvf_gemm p = chan(t->v[l], W, Wl, t->v[l + 1], W, N, batch);
        p.beta = 1.0f;
        p.bias = bl;
        p.bias_mode = 1;
        if (l < L - 1) {
            p.act = 1;
            p.C_pre = keep ? t->s[l] : nullptr;
        }
        if ((rc = gemm(t, p, s, "pointwise")) != BVF_OK) return rc;
    }
    g = chan(t->v[L], W, w + o.Q1, t->h, d.hidden, N, batch);
    g.bias = w + o.q1;
    g.bias_mode = 1;
    g.act = 1;
    g.C_pre = keep ? t->pre1 : nullptr;
    if ((rc = gemm(t, g, s, "projection 1")) != BVF_OK) return rc;
    g = chan(t->h, d.hidden, w + o.Q2, out, d.c_out, N, batch);
    g.bias = w + o.q2;
    g.bias_mode = 1;
    return gemm(t, g, s, "projection 2");
}

// loss and gradient into t->g (zeroed first); h_loss on the host
int gradient(bvf_fno_bf16 *t, int batch, const float *in, const float *target, const float *el,
             double el_weight, double *h_loss, cudaStream_t s)
{
    const bvf_fno_dims &d = t->d;
    const int W = d.width, N = t->N, L = d.n_layers, m = d.modes, H = d.hidden;
    const Off o = offsets(d);
    int rc = forward(t, batch, in, t->out, true, s);
    if (rc != BVF_OK) return rc;
    BCK(cudaMemsetAsync(t->sums, 0, 3 * sizeof(double) * batch, s), "loss");
    k_loss_sums<<<dim3(std::min(64, (N + 255) / 256), batch), 256, 0, s>>>(t->out, target, d.c_out,
                                                                          N, t->sums);
    k_loss_grad<<<grid_for((long long)batch * d.c_out * N), 256, 0, s>>>(
        t->out, target, d.c_out > 1 ? el : nullptr, t->sums, batch, d.c_out, N, (float)el_weight,
        t->dout);
    BCK(cudaGetLastError(), "loss");
    BCK(cudaMemsetAsync(t->g, 0, t->n_w * sizeof(float), s), "gradient");
    float *G = t->g;
    const float *w = t->w;
    const int ks = t->ksplit;
    // projection
    bvf_gemm g = chanT(t->dout, d.c_out, w + o.Q2, t->dh, H, N, batch);
    g.act = 2;
    g.C_pre = t->pre1;                                 // dh -> d pre1
    if ((rc = gemm(t, g, s, "d projection 2")) != BVF_OK) return rc;
    if ((rc = gemm(t, wgrad(t->dout, d.c_out, t->h, H, G + o.Q2, N, batch, ks), s, "dQ2")) != BVF_OK)
        return rc;
    if ((rc = chan_sum(t->dout, batch, d.c_out, N, G + o.q2, s)) != BVF_OK) return rc;
    if ((rc = gemm(t, wgrad(t->dh, H, t->v[L], W, G + o.Q1, N, batch, ks), s, "dQ1")) != BVF_OK)
        return rc;
    if ((rc = chan_sum(t->dh, batch, H, N, G + o.q1, s)) != BVF_OK) return rc;
    if ((rc = gemm(t, chanT(t->dh, H, w + o.Q1, t->dv, W, N, batch), s, "d projection 1")) != BVF_OK)
        return rc;
    // Fourier layers, top down; ds holds d(pre-activation) of layer l
    float *ds = t->dv, *dn = t->dv2;
    for (int l = L - 1; l >= 0; --l) {
        const float *lw = w + o.lay0 + l * o.lf;
        float *gl = G + o.lay0 + l * o.lf;
        const float *R = lw, *Wl = lw + (size_t)4 * m * m * m * W * W * 2;
        float *gR = gl, *gW = gl + (size_t)4 * m * m * m * W * W * 2, *gb = gW + (size_t)W * W;
        if ((rc = chan_sum(ds, batch, W, N, gb, s)) != BVF_OK) return rc;
        if ((rc = gemm(t, wgrad(ds, W, t->v[l], W, gW, N, batch, ks), s, "dW")) != BVF_OK) return rc;
        if ((rc = gemm(t, chanT(ds, W, Wl, dn, W, N, batch), s, "d pointwise")) != BVF_OK) return rc;
        if ((rc = spec_fwd(t, ds, (long long)batch * W, true, t->S1, s)) != BVF_OK) return rc;
        k_mix_dR<<<grid_for((long long)4 * m * m * m * W * W), 256, 0, s>>>(t->S1, t->X[l], batch, W,
                                                                            m, gR);
        k_mix_adj<<<grid_for((long long)batch * 4 * m * m * m * W), 256, 0, s>>>(t->S1, R, batch, W,
                                                                                 m, t->S2);
        BCK(cudaGetLastError(), "d mix");
        // dn = d v_l; for l > 0 it becomes d s_{l-1} = d v_l GELU'(s_{l-1})
        if ((rc = spec_inv(t, t->S2, (long long)batch * W, false, dn, 1.0f, l > 0 ? 2 : 0,
                           l > 0 ? t->s[l - 1] : nullptr, s)) != BVF_OK)
            return rc;
        std::swap(ds, dn);
    }
    // lift
    if ((rc = chan_sum(ds, batch, W, N, G + o.bp, s)) != BVF_OK) return rc;
    if ((rc = gemm(t, wgrad(ds, W, in, d.c_in, G + o.Wp, N, batch, ks), s, "dWp")) != BVF_OK)
        return rc;
    if (h_loss) {
        std::vector<double> h(3 * batch);
        BCK(cudaMemcpyAsync(h.data(), t->sums, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s),
            "loss");
        std::vector<float> e(batch);
        if (d.c_out > 1 && el)
            BCK(cudaMemcpyAsync(e.data(), el, batch * sizeof(float), cudaMemcpyDeviceToHost, s), "loss");
        BCK(cudaStreamSynchronize(s), "loss");
        double loss = 0.0;
        for (int b = 0; b < batch; ++b) {
            loss += std::sqrt(h[3 * b] / h[3 * b + 1]) / batch;
            if (d.c_out > 1 && el) {
                const double dm = h[3 * b + 2] / N - e[b];
                loss += el_weight * dm * dm / batch;
            }
        }
        *h_loss = loss;
    }
    return BVF_OK;
}

}  // namespace

extern "C" {

int bvf_fno_bf16_create(bvf_fno_bf16 **out, const bvf_fno_dims *d, const float *h_weights, size_t n,
                        int nx, int ny, int nz, int max_batch)
{
    if (!out) return b16_fail(BVF_E_ARG, "bvf_fno_bf16_create: out is NULL");
    *out = nullptr;
    if (!d || !h_weights || bvf_fno_weight_count(d) == 0 || n != bvf_fno_weight_count(d))
        return b16_fail(BVF_E_ARG, "bvf_fno_bf16_create: bad dims or weight count");
    const int m = d->modes;
    if (nx < 1 || ny < 1 || nz < 1 || m > nx / 2 || 2 * m > ny || 2 * m > nz || max_batch < 1 ||
        (long long)nx * ny * nz * max_batch * std::max(d->hidden, d->width) >= (1LL << 31))
        return b16_fail(BVF_E_ARG, "bvf_fno_bf16_create: grid too small for the modes, or too large");
    bvf_fno_bf16 *t = new (std::nothrow) bvf_fno_bf16;
    if (!t) return b16_fail(BVF_E_NOMEM, "bvf_fno_bf16_create: host allocation");
    t->d = *d;
    t->nx = nx;
    t->ny = ny;
    t->nz = nz;
    t->N = nx * ny * nz;
    t->Bmax = max_batch;
    t->n_w = n;
    auto fail = [&](int rc) {
        bvf_fno_bf16_destroy(t);
        return rc;
    };
    const size_t N = t->N, B = max_batch, W = d->width, H = d->hidden, S = 8 * (size_t)m * m * m;
    int rc = BVF_OK;
    for (float **p : {&t->w, &t->g, &t->m1, &t->m2})
        if ((rc = dalloc(t, p, n, "weights")) != BVF_OK) return fail(rc);
    std::vector<std::vector<float>> mats;
    build_matrices(nx, ny, nz, m, mats);
    float **mp[8] = {&t->Fx, &t->Fxw, &t->Fy, &t->Fz, &t->Gz, &t->Gy, &t->Gxw, &t->Gx};
    for (int i = 0; i < 8; ++i) {
        if ((rc = dalloc(t, mp[i], mats[i].size(), "stage matrices")) != BVF_OK) return fail(rc);
        if (cudaMemcpy(*mp[i], mats[i].data(), mats[i].size() * sizeof(float),
                       cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(b16_fail(BVF_E_CUDA, "bvf_fno_bf16_create: copy"));
    }
    t->v.resize(d->n_layers + 1);
    t->s.resize(std::max(0, d->n_layers - 1));
    t->X.resize(d->n_layers);
    for (auto &p : t->v)
        if ((rc = dalloc(t, &p, B * W * N, "activations")) != BVF_OK) return fail(rc);
    for (auto &p : t->s)
        if ((rc = dalloc(t, &p, B * W * N, "activations")) != BVF_OK) return fail(rc);
    for (auto &p : t->X)
        if ((rc = dalloc(t, &p, B * W * S, "spectra")) != BVF_OK) return fail(rc);
    const size_t ws = std::max({B * W * nz * ny * 2 * m, B * W * nz * m * 4 * m,
                                B * W * 2 * m * m * 4 * m, B * W * 2 * m * m * 2 * nz,
                                B * W * nz * m * 2 * ny});
    if ((rc = dalloc(t, &t->pre1, B * H * N, "projection")) != BVF_OK ||
        (rc = dalloc(t, &t->h, B * H * N, "projection")) != BVF_OK ||
        (rc = dalloc(t, &t->dh, B * H * N, "projection")) != BVF_OK ||
        (rc = dalloc(t, &t->out, B * d->c_out * N, "output")) != BVF_OK ||
        (rc = dalloc(t, &t->dout, B * d->c_out * N, "output")) != BVF_OK ||
        (rc = dalloc(t, &t->w1, ws, "work")) != BVF_OK ||
        (rc = dalloc(t, &t->w2, ws, "work")) != BVF_OK ||
        (rc = dalloc(t, &t->S1, B * W * S, "spectra")) != BVF_OK ||
        (rc = dalloc(t, &t->S2, B * W * S, "spectra")) != BVF_OK ||
        (rc = dalloc(t, &t->dv, B * W * N, "gradients")) != BVF_OK ||
        (rc = dalloc(t, &t->dv2, B * W * N, "gradients")) != BVF_OK ||
        (rc = dalloc(t, &t->sums, 3 * B, "loss")) != BVF_OK ||
        (rc = dalloc(t, &t->flag, 1, "flag")) != BVF_OK)
        return fail(rc);
    if (cudaMemcpy(t->w, h_weights, n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(t->m1, 0, n * sizeof(float)) != cudaSuccess ||
        cudaMemset(t->m2, 0, n * sizeof(float)) != cudaSuccess ||
        cudaMemset(t->flag, 0, sizeof(int)) != cudaSuccess)
        return fail(b16_fail(BVF_E_CUDA, "bvf_fno_bf16_create: initial copies"));
    // voxel sums of the weight gradients: enough K-split blocks to fill the GPU
    t->ksplit = (int)std::max<long long>(1, std::min<long long>(256, (long long)N / 4096));
    *out = t;
    return BVF_OK;
}

int bvf_fno_bf16_destroy(bvf_fno_bf16 *t)
{
    if (!t) return BVF_OK;
    cudaDeviceSynchronize();
    for (void *p : t->all) cudaFree(p);
    delete t;
    return BVF_OK;
}

int bvf_fno_bf16_forward(bvf_fno_bf16 *t, int batch, const float *d_in, float *d_out, void *stream)
{
    if (!t || !d_in || !d_out || batch < 1 || batch > t->Bmax)
        return b16_fail(BVF_E_ARG, "bvf_fno_bf16_forward: bad argument");
    return forward(t, batch, d_in, d_out, false, static_cast<cudaStream_t>(stream));
}

int bvf_fno_bf16_gradient(bvf_fno_bf16 *t, int batch, const float *d_in, const float *d_target,
                          const float *d_el, double el_weight, float *d_grad, double *h_loss,
                          void *stream)
{
    if (!t || !d_in || !d_target || batch < 1 || batch > t->Bmax || !(el_weight >= 0.0) ||
        (t->d.c_out > 1 && el_weight > 0.0 && !d_el))
        return b16_fail(BVF_E_ARG, "bvf_fno_bf16_gradient: bad argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int rc = gradient(t, batch, d_in, d_target, d_el, el_weight, h_loss, s);
    if (rc != BVF_OK) return rc;
    if (d_grad)
        BCK(cudaMemcpyAsync(d_grad, t->g, t->n_w * sizeof(float), cudaMemcpyDeviceToDevice, s),
            "bvf_fno_bf16_gradient: copy");
    return BVF_OK;
}

int bvf_fno_bf16_adam(bvf_fno_bf16 *t, int batch, const float *d_in, const float *d_target,
                      const float *d_el, double el_weight, double lr, double *h_loss, void *stream)
{
    if (!t || !(lr > 0.0)) return b16_fail(BVF_E_ARG, "bvf_fno_bf16_adam: bad argument");
    int rc = bvf_fno_bf16_gradient(t, batch, d_in, d_target, d_el, el_weight, nullptr, h_loss, stream);
    if (rc != BVF_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double b1 = 0.9, b2 = 0.999;
    ++t->adam_t;
    const float c1 = (float)(1.0 - std::pow(b1, (double)t->adam_t));
    const float c2 = (float)(1.0 - std::pow(b2, (double)t->adam_t));
    k_adam<<<grid_for((long long)t->n_w), 256, 0, s>>>(t->w, t->g, t->m1, t->m2, t->n_w, (float)lr,
                                                      (float)b1, (float)b2, 1e-8f, c1, c2);
    BCK(cudaGetLastError(), "bvf_fno_bf16_adam");
    return BVF_OK;
}

int bvf_fno_bf16_weights(bvf_fno_bf16 *t, float *h_weights)
{
    if (!t || !h_weights) return b16_fail(BVF_E_ARG, "bvf_fno_bf16_weights: bad argument");
    BCK(cudaDeviceSynchronize(), "bvf_fno_bf16_weights");
    BCK(cudaMemcpy(h_weights, t->w, t->n_w * sizeof(float), cudaMemcpyDeviceToHost),
        "bvf_fno_bf16_weights");
    return BVF_OK;
}

int bvf_fno_mean(const float *d_x, size_t n, double *h_mean, void *stream)
{
    if (!d_x || !h_mean || n == 0) return b16_fail(BVF_E_ARG, "bvf_fno_mean: bad argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *d = nullptr;
    BCK(cudaMallocAsync((void **)&d, sizeof(double), s), "bvf_fno_mean");
    double h = 0.0;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(double), s);
    if (e == cudaSuccess) {
        k_sum<<<grid_for((long long)n), 256, 0, s>>>(d_x, n, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(d, s);
    BCK(e, "bvf_fno_mean");
    *h_mean = h / (double)n;
    return BVF_OK;
}

int bvf_fno_bf16_synchronize(bvf_fno_bf16 *t, void *stream)
{
    if (!t) return b16_fail(BVF_E_ARG, "bvf_fno_bf16_synchronize: NULL");
    BCK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)), "bvf_fno_bf16_synchronize");
    int f = 0;
    BCK(cudaMemcpy(&f, t->flag, sizeof(int), cudaMemcpyDeviceToHost), "bvf_fno_bf16_synchronize");
    if (f) {
        cudaMemset(t->flag, 0, sizeof(int));
        return b16_fail(BVF_E_CUDA, "bvf_fno_bf16: a bounded wait for the tensor cores ran out");
    }
    return BVF_OK;
}

}  // extern "C"
