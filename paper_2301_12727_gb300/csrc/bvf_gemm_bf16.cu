// BF16 tensor-core product on the fifth-generation tensor cores (tcgen05):
// C = alpha A B + beta C (+ bias) (-> GELU), FP32 in and out, BF16 operands,
// FP32 accumulation in tensor memory.  Every contraction of the surrogate's
// BF16 path and of its training (channel mixes, the truncated DFT along each
// axis and their adjoints) is one call of this kernel on strided views.
//
// A block of 128 threads computes a 128 x BN tile of C:
//   * K runs in chunks of 64; the chunk's A (128 x 64) and B (BN x 64) tiles
//     are read from their strided FP32 arrays, rounded to BF16 and written to
//     shared memory in the canonical K-major layout (8 rows x 16 bytes per
//     core matrix), two stages deep, so the threads stage chunk c+1 while the
//     tensor cores multiply chunk c;
//   * thread 0 issues four tcgen05.mma.kind::f16 (K = 16 each) per chunk into
//     the TMEM accumulator and commits them to the stage's mbarrier;
//   * the epilogue reads the accumulator with tcgen05.ld (warp w holds rows
//     32 w .. 32 w + 31) and applies alpha, beta, the bias and GELU (keeping
//     the pre-activation when asked), or adds into C atomically when K is
//     split over several blocks.
// Waits are bounded: a block whose wait runs out stops issuing products,
// waits (bounded) for those in flight, frees its tensor memory, sets bit 2 of
// the flag and ends.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <atomic>

#include <algorithm>
#include <cmath>

#include "../../include/bvf_fno.h"
#include "bvf_internal.cuh"
#include "bvf_tc.cuh"
#include "bvf_tma.cuh"

namespace bvf {

namespace {

constexpr int GK = 64;                 // K chunk (BF16 elements): 128 bytes per row
constexpr int GSEG = GK / 8;           // 16-byte core-matrix rows per tile row and chunk

// NS shared-memory stages of GK-wide K chunks: two overlap the staging of a
// chunk with the products of the previous one; products of a single chunk
// (K <= GK) take one, so twice as many blocks fit per SM.
template <int BN, int NS>
struct GemmLayout {
    static constexpr int A_BYTES = 128 * GK * 2;
    static constexpr int B_BYTES = BN * GK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int off_bar = NS * STAGE;
    static constexpr int off_tmem = off_bar + 16;
    static constexpr int bytes = off_tmem + 16;
    static_assert(NS * STAGE >= 4 * 32 * 33 * 4, "the epilogue's transpose buffers fit the stages");
    static constexpr uint32_t SBO = GSEG * 128;      // byte step between 8-row groups
};

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// Rows [0, rows) x K-chunk [k0, k0 + GK) of a strided FP32 operand (element
// (r, k) at src[r * srow + k * sk]; zero for r >= valid or k >= K) written as
// BF16 in K-major core matrices.  With sk == 1 consecutive threads take
// consecutive 8-element pieces of one row, otherwise consecutive rows, so the
// global reads are coalesced in both layouts.
__device__ __forceinline__ void stage_tile(unsigned char *dst, const float *__restrict__ src,
                                           long long srow, long long sk, int rows, int valid,
                                           int k0, int K, int tid)
{
    const int segs = rows * GSEG;
    for (int s = tid; s < segs; s += 128) {
        int r, k8;
        if (sk == 1) {
            r = s / GSEG;
            k8 = (s % GSEG) * 8;
        } else {
            r = s % rows;
            k8 = (s / rows) * 8;
        }
        float v[8];
        const float *row = src + (long long)r * srow;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = k0 + k8 + j;
            v[j] = (r < valid && k < K) ? __ldg(row + (long long)k * sk) : 0.0f;
        }
        *reinterpret_cast<uint4 *>(dst + tc::kmaj_off16(r, k8, GK)) =
            make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                       pack_bf16(v[6], v[7]));
    }
}

__device__ __forceinline__ float gelu_exact(float s)
{
    return 0.5f * s * (1.0f + erff(s * 0.70710678118654752f));
}
// d GELU / ds = Phi(s) + s phi(s)
__device__ __forceinline__ float gelu_grad(float s)
{
    return 0.5f * (1.0f + erff(s * 0.70710678118654752f)) +
           s * 0.39894228040143268f * expf(-0.5f * s * s);
}

template <int BN, int NS>
__global__ void __launch_bounds__(128) k_gemm_bf16(const __grid_constant__ bvf_gemm g, int *flag)
{
    extern __shared__ __align__(128) unsigned char sm[];
    using Lay = GemmLayout<BN, NS>;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + Lay::off_bar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + Lay::off_tmem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * BN;
    const int b = blockIdx.z / g.ksplit, split = blockIdx.z % g.ksplit;
    const int n_chunks = (g.K + GK - 1) / GK;
    const int per = (n_chunks + g.ksplit - 1) / g.ksplit;
    const int c_begin = split * per, c_end = min(n_chunks, c_begin + per);
    const float *A = g.A + (long long)b * g.sab + (long long)m0 * g.sam;
    const float *B = g.B + (long long)b * g.sbb + (long long)n0 * g.sbn;
    const int va = min(128, g.M - m0), vb = min(BN, g.N - n0);
    if (tid == 0) {
        tma::mbar_init(&bar[0], 1);
        tma::mbar_init(&bar[1], 1);
        tma::mbar_init_fence();
    }
    if (warp == 0) {
        tc::alloc(tslot, BN);
        tc::relinquish();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = *tslot;
    const uint32_t idesc = tc::idesc_bf16(128, BN);

    bool bad = false;
    int nc = 0;                             // chunks whose products were issued
    for (int c = c_begin; c < c_end; ++c, ++nc) {
        const int st = nc % NS;
        unsigned char *sa = sm + st * Lay::STAGE, *sb = sa + Lay::A_BYTES;
        if (nc >= NS) {                     // the products of chunk nc - NS read this stage
            const bool ok = tma::mbar_wait(&bar[st], ((nc - NS) / NS) & 1, tma::kWaitLimit);
            if (__syncthreads_or(!ok)) {
                bad = true;
                break;
            }
        }
        stage_tile(sa, A, g.sam, g.sak, 128, va, c * GK, g.K, tid);
        stage_tile(sb, B, g.sbn, g.sbk, BN, vb, c * GK, g.K, tid);
        tma::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after();
#pragma unroll
            for (int ks = 0; ks < GK / 16; ++ks) {
                const uint32_t ko = ks * 2 * 128;        // two core matrices per K step of 16
                tc::mma_f16(tbase, tc::smem_desc(sa + ko, 128, Lay::SBO),
                            tc::smem_desc(sb + ko, 128, Lay::SBO), idesc, (nc > 0 || ks > 0) ? 1 : 0);
            }
            tc::commit(&bar[st]);
        }
    }
    if (!bad && nc > 0) {                   // the last commit covers every earlier product
        const int last = nc - 1;
        const bool ok = tma::mbar_wait(&bar[last % NS], (last / NS) & 1, tma::kWaitLimit);
        bad = __syncthreads_or(!ok) != 0;
    }
    if (bad) {
        if (tid == 0) {
            const int last = nc - 1;
            if (last >= 0) tma::mbar_wait(&bar[last % NS], (last / NS) & 1, tma::kWaitLimit);
            atomicOr(flag, 2);
        }
    } else {
        tc::fence_after();
        // element (mm, n) of the tile: alpha, beta C, bias, activation, store
        auto finish = [&](int mm, int n, float acc) {
            float *cp = g.C + (long long)b * g.scb + (long long)mm * g.scm + (long long)n * g.scn;
            float *pp = g.C_pre ? g.C_pre + (long long)b * g.scb + (long long)mm * g.scm +
                                      (long long)n * g.scn
                                : nullptr;
            float v = g.alpha * acc;
            if (g.ksplit > 1) {
                if (nc > 0) atomicAdd(cp, v);
                return;
            }
            if (g.beta != 0.0f) v = fmaf(g.beta, *cp, v);
            if (g.bias_mode == 1) v += __ldg(g.bias + n);
            else if (g.bias_mode == 2) v += __ldg(g.bias + mm);
            if (g.act == 1) {
                if (pp) *pp = v;
                v = gelu_exact(v);
            } else if (g.act == 2) {
                v *= gelu_grad(*pp);
            }
            *cp = v;
        };
        // Thread `lane` of a warp holds row warp * 32 + lane of the tile.  With
        // the columns of C contiguous (scn == 1) each warp transposes its
        // 32 x 32 block through shared memory (the stage buffers, free now
        // that every product has completed) so that a warp's stores cover 32
        // consecutive columns of one row; otherwise (rows contiguous) it
        // stores straight from the accumulator row.
        const bool by_rows = g.scn == 1 && g.ksplit == 1;
        float *wbuf = reinterpret_cast<float *>(sm) + warp * (32 * 33);
        const int m = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 32) {
            float r[32];
            if (nc > 0) {
                tc::ld32(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
                tc::wait_ld();
            } else {
#pragma unroll
                for (int i = 0; i < 32; ++i) r[i] = 0.0f;
            }
            if (by_rows) {
                __syncwarp();
#pragma unroll
                for (int i = 0; i < 32; ++i) wbuf[lane * 33 + i] = r[i];
                __syncwarp();
                const int n = n0 + c0 + lane;
#pragma unroll 4
                for (int i = 0; i < 32; ++i) {
                    const int mm = m0 + warp * 32 + i;
                    if (mm < g.M && n < g.N) finish(mm, n, wbuf[i * 33 + lane]);
                }
            } else {
                if (m >= g.M) continue;
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int n = n0 + c0 + i;
                    if (n < g.N) finish(m, n, r[i]);
                }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::dealloc(tbase, BN);
}

template <int BN, int NS>
cudaError_t launch_gemm_ns(const bvf_gemm &g, int *flag, cudaStream_t s)
{
    const dim3 grid((g.M + 127) / 128, (g.N + BN - 1) / BN, g.batch * g.ksplit);
    // the shared-memory limit is raised once per process, so that later
    // launches make no other runtime call (a forward can be recorded in a graph)
    static std::atomic<int> raised{0};
    if (!raised.load(std::memory_order_acquire)) {
        const cudaError_t e = cudaFuncSetAttribute(
            k_gemm_bf16<BN, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
            GemmLayout<BN, NS>::bytes);
        if (e != cudaSuccess) return e;
        raised.store(1, std::memory_order_release);
    }
    k_gemm_bf16<BN, NS><<<grid, 128, GemmLayout<BN, NS>::bytes, s>>>(g, flag);
    return cudaGetLastError();
}

// one stage when the product is a single K chunk
template <int BN>
cudaError_t launch_gemm_t(const bvf_gemm &g, int *flag, cudaStream_t s)
{
    const int per_split = ((g.K + GK - 1) / GK + g.ksplit - 1) / g.ksplit;
    return per_split <= 1 ? launch_gemm_ns<BN, 1>(g, flag, s) : launch_gemm_ns<BN, 2>(g, flag, s);
}

}  // namespace

// BN: the smallest tile width of 32, 64, 128, 256 that holds N (256 beyond),
// at most 64 for a single-chunk product
cudaError_t launch_gemm_bf16(const bvf_gemm &g, int *flag, cudaStream_t s)
{
    if (g.N <= 32) return launch_gemm_t<32>(g, flag, s);
    // a single-chunk product restages its small A tile per N tile but keeps
    // 64 TMEM columns per block, so up to 8 blocks share an SM's 512
    const int per_split = ((g.K + GK - 1) / GK + g.ksplit - 1) / g.ksplit;
    if (g.N <= 64 || per_split <= 1) return launch_gemm_t<64>(g, flag, s);
    if (g.N <= 128) return launch_gemm_t<128>(g, flag, s);
    return launch_gemm_t<256>(g, flag, s);
}

}  // namespace bvf

extern "C" int bvf_gemm_bf16(const bvf_gemm *g, int *d_flag, void *stream)
{
    if (!g || !g->A || !g->B || !g->C || !d_flag || g->M < 1 || g->N < 1 || g->K < 0 ||
        g->batch < 1 || g->ksplit < 1 || g->batch * g->ksplit > 65535 ||
        (g->bias_mode != 0 && !g->bias) || g->bias_mode < 0 || g->bias_mode > 2 || g->act < 0 ||
        g->act > 2 || (g->act == 2 && !g->C_pre) ||
        (g->ksplit > 1 && (g->bias_mode != 0 || g->act != 0 || g->beta != 1.0f))) {
        bvf::set_context_free_error("bvf_gemm_bf16: bad argument");
        return BVF_E_ARG;
    }
    const cudaError_t e = bvf::launch_gemm_bf16(*g, d_flag, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        bvf::set_context_free_error(cudaGetErrorString(e));
        return BVF_E_CUDA;
    }
    return BVF_OK;
}
