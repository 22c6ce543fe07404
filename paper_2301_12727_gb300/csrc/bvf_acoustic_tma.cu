// TMA-fed acoustic kernels (arXiv 2301.12727, Sec. 2.3, Eq. 1; Sec. 3.2, Eq. 3).
//
// Same arithmetic as the direct kernels in bvf_acoustic.cu, but every array
// moves between HBM and shared memory through the tensor-memory accelerator:
//   * a block owns one 32 x 8 x-y tile and walks a chunk of z; in the
//     velocity kernel (16 x 8 threads) thread (tx, ty) updates the voxel pair
//     (x0 + 2 tx, x0 + 2 tx + 1) of row y0 + ty, in the stress kernel (32 x 8
//     threads) one voxel each;
//   * stencil inputs arrive as halo'd boxes (the tile plus XO columns on each
//     side in x and 2 rows in y; out-of-range elements zero-filled by the TMA,
//     which gives the zero ghosts) held in per-array rings of z-planes that
//     serve the 4-point z-stencils as well;
//   * the 1-byte material index arrives as 48 x 9 boxes (planes k and k+1);
//   * velocity pairs: a y- or z-stencil is four paired shared-memory reads,
//     an x-stencil three (elements -2 .. +3 around the pair); the velocities
//     and the y- and z-slab CPML memories move as paired global accesses; the
//     FP32 arithmetic runs on the packed FP32x2 instructions (bit for bit two
//     single-voxel evaluations, see bvf_stencil.cuh); buoyancies and the
//     x-slab CPML stay per voxel.  This halves the velocity kernel's
//     instructions, which bound it.  The stress kernel is bound by the latency
//     of its per-voxel streams instead: it keeps one voxel per thread (64
//     registers, 32 resident warps per SM) and, with FP32 storage,
//     prefetches the next plane's streams into L2;
//   * velocity kernel: each stress array arrives in a box with exactly the
//     halo its stencil needs; the velocities go straight to registers and
//     back; copies for plane k+1 are issued while plane k is computed;
//   * stress kernel: the velocity and index rings run two planes ahead; the
//     per-voxel arrays go straight to registers with loads issued at the top
//     of each plane and back with coalesced stores;
//   * one thread issues every copy; one __syncthreads and one bounded mbarrier
//     wait per plane.
// The state is stored as T = float or __half (scaled FP16 storage; the
// arithmetic is FP32 either way).  A TMA box must start on a 16-byte boundary
// in x, so the x-halo is XO = 16 / sizeof(T) columns: 4 floats or 8 halves.
// Used when nx % 8 == 0 (state rows are whole multiples of 16 bytes in both
// storages, every pair lies inside the grid and every paired access is
// aligned; the index is mapped from a copy with rows padded to 16 bytes when
// nx % 16 != 0) and L <= 2.
#include <cuda_fp16.h>

#include <atomic>
#include <type_traits>

#include "bvf_stencil.cuh"
#include "bvf_tma.cuh"

namespace bvf {

namespace {

using st::dbw;
using st::dfw;
using st::pair;
using st::slab_pos;
using st::tof;
using st::splat;
using st::vadd;

// A tile is TX = 32 voxels wide and TH rows high, TH = 4, 8 or 16 (a template
// parameter of the single-domain kernels, chosen per context; the persistent
// batch kernels use TY).
constexpr int TX = 32, TY = 8;                      // width, default height
constexpr int PX = TX / 2;                          // threads per tile row (a pair each)
constexpr int NTH = PX * TY;                        // 128
constexpr int IW = 48;                              // index box: x0 .. x0+47
// Index box of a tile of height TH: rows y0 .. y0+TH, in a 128-byte ring slot.
template <int TH>
struct Idx {
    static constexpr int H = TH + 1, BYTES = IW * H, SLOT = (BYTES + 127) / 128 * 128;
};

// Box geometry of a storage type: x-halo XO columns each side, so halo'd
// boxes are BW = 32 + 2 XO wide (40 floats / 48 halves = 160 / 96 bytes).
template <typename T, int TH = TY>
struct Box {
    static constexpr int XO = 16 / (int)sizeof(T);
    static constexpr int BW = TX + 2 * XO;
    static constexpr int VH = TH + 4;                 // 2 rows each side
    static constexpr int VT = BW * VH;                // full-halo box (elements)
};

// the pair of elements (x, x+1) at an even offset of a shared-memory box
template <typename T>
__device__ __forceinline__ float2 lds2(const T *p)
{
    return st::ld2(p);
}

// x-stencils of a pair from three aligned pair reads a = (f[-2], f[-1]),
// b = (f[0], f[1]), c = (f[2], f[3]) around the pair's first voxel:
// D+ at x + 1/2 reads f[-1 .. 2] (first voxel) and f[0 .. 3] (second),
// D- at x reads f[-2 .. 1] and f[-1 .. 2].
__device__ __forceinline__ float2 dfw_x(float2 a, float2 b, float2 c, st::Dx d)
{
    return st::dfw<float2>(pair(a.y, b.x), b, pair(b.y, c.x), c, d);
}
__device__ __forceinline__ float2 dbw_x(float2 a, float2 b, float2 c, st::Dx d)
{
    return st::dbw<float2>(a, pair(a.y, b.x), b, pair(b.y, c.x), d);
}

// one lane of a pair
__device__ __forceinline__ float lane(float2 v, int l) { return l ? v.y : v.x; }
__device__ __forceinline__ void set_lane(float2 &v, int l, float x)
{
    if (l)
        v.y = x;
    else
        v.x = x;
}

// Time-out of a bounded ring wait.  The thread whose wait ran out records
// the plane in the block's abort word; every thread reads that word right
// after the next block barrier, so all of them leave the plane loop at the
// same point and no copy is issued after it.  Thread 0 then waits, again
// bounded, for the phases the block has armed (planes a .. a + ahead, at most
// one per barrier), sets bit 2 of the context flag and the tile ends.
// Barrier and parity of a plane t = pl - k0 of the chunk: velocity ring
// bar t % 2, phase t / 2; stress ring bar t % 3, phase t / 3.
template <int NBAR>
__device__ __forceinline__ void drain_after_timeout(uint64_t *bars, int a, int ahead, int k0,
                                                    int k1, unsigned limit, int *flag)
{
    for (int pl = a; pl <= a + ahead && pl < k1; ++pl) {
        const int t = pl - k0;
        tma::mbar_wait(&bars[t % NBAR], (unsigned)(t / NBAR) & 1u, limit);
    }
    atomicOr(flag, 2);
}

// ---------------------------------------------------------------- velocity
// Each stress array arrives in a box holding the halo its stencil reads:
// sxx BW x 8 (x-halo), syy 32 x 12 (y-halo), sxy BW x 12, sxz BW x 8,
// syz 32 x 12, szz 32 x 8 (z only).  The velocities go straight to registers
// and back.  Loads for plane k+1 are issued while plane k is computed.
//
// The plane loop is unrolled by the ring period R = 6 (every ring depth
// divides it), so each unrolled copy reads fixed ring slots: every shared
// memory access is one of five per-thread centres plus a constant.
template <typename T, int TH = TY>
struct VelLayout {
    using B = Box<T, TH>;
    static constexpr int R = 6;                               // ring period = unroll
    static constexpr int RA = 2, RB = 6, RC = 6, RI = 3;      // ring depths (divide R)
    static constexpr int XW = B::BW, XH = TH, YW = TX, YH = TH + 4;
    static constexpr int TXX = XW * XH, TYY = YW * YH, TXY = B::VT, TZZ = TX * TH;
    static constexpr int SA = TXX + TYY + TXY;                // elements per A slot (sxx, syy, sxy)
    static constexpr int SB = TXX + TYY;                      // B slot (sxz, syz)
    static constexpr int ES = (int)sizeof(T);
    static constexpr int off_a = 0;                           // bytes; plane k, k+1
    static constexpr int off_b = off_a + RA * SA * ES;        // k-2 .. k+2 (+1 spare)
    static constexpr int off_c = off_b + RB * SB * ES;        // szz: k-1 .. k+3 (+1 spare)
    static constexpr int off_i = off_c + RC * TZZ * ES;       // index: k .. k+2
    static constexpr int off_bar = off_i + RI * Idx<TH>::SLOT;
    static constexpr int off_abort = off_bar + 16;             // int: plane whose wait ran out
    static constexpr int off_end = off_abort + 16;
    static size_t bytes(int) { return off_end; }
    static_assert(R % RA == 0 && R % RB == 0 && R % RC == 0 && R % RI == 0,
                  "ring depths must divide the unroll period");
    static_assert(off_b % 128 == 0 && off_c % 128 == 0 && off_i % 128 == 0 &&
                      (SA * ES) % 128 == 0 && (SB * ES) % 128 == 0 && (TXX * ES) % 128 == 0 &&
                      (TYY * ES) % 128 == 0 && (TZZ * ES) % 128 == 0,
                  "TMA destinations must stay 128-byte aligned");
};

// One tile (bx, by) of the grid over z-chunk bz.  REUSE: the block runs
// further tiles afterwards (persistent batch kernel), so its mbarriers are
// invalidated at the end and the first copies are fenced against the
// previous tile's reads of the same shared memory.  Returns true (in every
// thread) when a ring wait ran out; the tile's results are then incomplete.
template <typename T, bool REUSE, int TH = TY>
__device__ __forceinline__ bool velocity_tile(const AcParams &p, const VelocityTmaMaps &tm,
                                              int kchunk, int bx, int by, int bz,
                                              unsigned char *smb)
{
    using Lay = VelLayout<T, TH>;
    using Bx = Box<T, TH>;
    constexpr int IT = Idx<TH>::BYTES, IT_SLOT = Idx<TH>::SLOT;
    constexpr int XW = Lay::XW, YW = Lay::YW, VW = Bx::BW;
    constexpr int TXX = Lay::TXX, TYY = Lay::TYY, TZZ = Lay::TZZ;
    const T *smt = reinterpret_cast<const T *>(smb);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smb + Lay::off_bar);
    volatile int *s_abort = reinterpret_cast<volatile int *>(smb + Lay::off_abort);

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * PX + tx;
    const int x0 = bx * TX, y0 = by * TH;
    const int i = x0 + 2 * tx, j = y0 + ty;         // the pair (i, i+1) of row j
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const bool live = i < nx && j < ny;              // nx is even: i + 1 < nx as well
    const int k0 = bz * kchunk, k1 = min(nz, k0 + kchunk);
    if (tid == 0) {
        tma::mbar_init(&bars[0], 1);
        tma::mbar_init(&bars[1], 1);
        tma::mbar_init_fence();
        *s_abort = -1;
    }
    __syncthreads();

    // ring slots: A holds plane pl in slot (pl-k0)%2, B in (pl-k0+2)%6,
    // C in (pl-k0+1)%6, the index in (pl-k0)%3
    constexpr unsigned A_BYTES = Lay::SA * Lay::ES, B_BYTES = Lay::SB * Lay::ES;
    constexpr unsigned C_BYTES = TZZ * Lay::ES;
    auto ldA = [&](int pl, int slot, uint64_t *bar) {
        unsigned char *d = smb + Lay::off_a + slot * A_BYTES;
        tma::load3d(d, &tm.sg[0], x0 - Bx::XO, y0, pl, bar);                            // sxx
        tma::load3d(d + TXX * Lay::ES, &tm.sg[1], x0, y0 - 2, pl, bar);                  // syy
        tma::load3d(d + (TXX + TYY) * Lay::ES, &tm.sg[3], x0 - Bx::XO, y0 - 2, pl, bar); // sxy
    };
    auto ldB = [&](int pl, int slot, uint64_t *bar) {
        unsigned char *d = smb + Lay::off_b + slot * B_BYTES;
        tma::load3d(d, &tm.sg[4], x0 - Bx::XO, y0, pl, bar);                            // sxz
        tma::load3d(d + TXX * Lay::ES, &tm.sg[5], x0, y0 - 2, pl, bar);                  // syz
    };
    auto ldC = [&](int pl, int slot, uint64_t *bar) {
        tma::load3d(smb + Lay::off_c + slot * C_BYTES, &tm.sg[2], x0, y0, pl, bar);
    };
    auto ldI = [&](int pl, int slot, uint64_t *bar) {
        tma::load3d(smb + Lay::off_i + slot * IT_SLOT, &tm.idx, x0, y0, pl, bar);
    };

    if (tid == 0) {
        if (REUSE) tma::fence_async_smem();
        tma::mbar_expect_tx(&bars[0], A_BYTES + 4 * B_BYTES + 4 * C_BYTES + 2 * IT);
        ldA(k0, 0, &bars[0]);
        for (int d = 0; d < 4; ++d) ldB(k0 - 2 + d, d, &bars[0]);
        for (int d = 0; d < 4; ++d) ldC(k0 - 1 + d, d, &bars[0]);
        ldI(k0, 0, &bars[0]);
        ldI(k0 + 1, 1, &bars[0]);
    }

    const st::Dx ix = st::make_dx(p.inv_dx);
    const float dt = p.dtv;
    // per-thread centres inside a slot (elements, all even): x-halo box,
    // y-halo box, full-halo box, plain box; index box (bytes)
    const int cx = ty * XW + 2 * tx + Bx::XO;
    const int cy = (ty + 2) * YW + 2 * tx;
    const int cxy = (ty + 2) * VW + 2 * tx + Bx::XO;
    const int cz = ty * TX + 2 * tx;
    const int cI = ty * IW + 2 * tx;
    const int xs[2] = {slab_pos(i, nx, p.P), slab_pos(i + 1, nx, p.P)};
    const int ys = slab_pos(j, ny, p.P);
    const int Sxs = nz * ny * p.W, Sys = nz * p.W * nx, Szs = p.W * ny * nx;
    const float2 *pmlx = p.pml, *pmly = p.pml + 2 * p.nmax, *pmlz = p.pml + 4 * p.nmax;
    T *__restrict__ vxg = static_cast<T *>(p.vx);
    T *__restrict__ vyg = static_cast<T *>(p.vy);
    T *__restrict__ vzg = static_cast<T *>(p.vz);
    // the pair's second voxel is not the last point in x (the first never is)
    const bool ix1 = i + 1 < nx - 1, jy1 = j < ny - 1;
    const int plane = nx * ny, col = j * nx + i;
    // velocities of the plane being computed, loaded one plane ahead
    float2 ux = pair(0.0f, 0.0f), uy = ux, uz = ux;
    if (live) {
        ux = st::ld2(vxg + k0 * plane + col);
        uy = st::ld2(vyg + k0 * plane + col);
        uz = st::ld2(vzg + k0 * plane + col);
    }
    int q = k0 * plane + col;                       // this pair in plane k
    int ox[2] = {(k0 * ny + j) * p.W + xs[0],       // in the x-slab (xs >= 0)
                 (k0 * ny + j) * p.W + xs[1]};
    int oy = (k0 * p.W + ys) * nx + i;              // in the y-slab (ys >= 0)
    const int dox = ny * p.W, doy = p.W * nx;

    unsigned mpar = 0;                              // parity of (k - k0) / R
    bool stop = false;
    for (int kb = k0; kb < k1 && !stop; kb += Lay::R, mpar ^= 1u) {
#pragma unroll
        for (int u = 0; u < Lay::R; ++u) {
            const int k = kb + u;
            if (k >= k1) break;
            __syncthreads();
            if (*s_abort >= 0) {      // a wait of the previous plane ran out
                stop = true;
                break;
            }
            if (tid == 0 && k + 1 < k1) {
                tma::fence_async_smem();
                uint64_t *bar = &bars[(u + 1) & 1];
                tma::mbar_expect_tx(bar, A_BYTES + B_BYTES + C_BYTES + IT);
                if (!(p.hold == 1 && k == p.hold_plane)) {
                    ldA(k + 1, (u + 1) % Lay::RA, bar);
                    ldB(k + 2, (u + 4) % Lay::RB, bar);
                    ldC(k + 3, (u + 4) % Lay::RC, bar);
                    ldI(k + 2, (u + 2) % Lay::RI, bar);
                }
            }
            float2 nux = pair(0.0f, 0.0f), nuy = nux, nuz = nux;
            if (live && k + 1 < k1) {
                nux = st::ld2(vxg + q + plane);
                nuy = st::ld2(vyg + q + plane);
                nuz = st::ld2(vzg + q + plane);
            }
            // CPML memories of this pair (components 0-2 of each slab it lies
            // in), all loads issued together before the ring wait; the x-slab
            // is per voxel, the y- and z-slabs per pair
            const int zs = slab_pos(k, nz, p.P);
            const int oz = zs * plane + col;
            float qx[2][3] = {{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};
            float2 qy[3] = {pair(0.0f, 0.0f), pair(0.0f, 0.0f), pair(0.0f, 0.0f)};
            float2 qz[3] = {qy[0], qy[0], qy[0]};
            if (live) {
#pragma unroll
                for (int l = 0; l < 2; ++l)
                    if (xs[l] >= 0) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) qx[l][c] = p.psx[c * Sxs + ox[l]];
                    }
                if (ys >= 0) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) qy[c] = st::ld2(p.psy + c * Sys + oy);
                }
                if (zs >= 0) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) qz[c] = st::ld2(p.psz + c * Szs + oz);
                }
            }
            const bool ready =
                tma::mbar_wait(&bars[u & 1], mpar ^ ((u >> 1) & 1u), p.wait_limit);
            if (!ready) *s_abort = k;
            if (ready && live) {
                // fixed slots of this unrolled copy
                const T *A = smt + (Lay::off_a / Lay::ES) + (u % Lay::RA) * Lay::SA;
                const T *XX = A + cx, *YY = A + TXX + cy, *XY = A + TXX + TYY + cxy;
                const T *Bm2 = smt + Lay::off_b / Lay::ES + ((u + 0) % Lay::RB) * Lay::SB;
                const T *Bm1 = smt + Lay::off_b / Lay::ES + ((u + 1) % Lay::RB) * Lay::SB;
                const T *B0 = smt + Lay::off_b / Lay::ES + ((u + 2) % Lay::RB) * Lay::SB;
                const T *Bp1 = smt + Lay::off_b / Lay::ES + ((u + 3) % Lay::RB) * Lay::SB;
                const T *Cm1 = smt + Lay::off_c / Lay::ES + ((u + 0) % Lay::RC) * TZZ + cz;
                const T *C0 = smt + Lay::off_c / Lay::ES + ((u + 1) % Lay::RC) * TZZ + cz;
                const T *Cp1 = smt + Lay::off_c / Lay::ES + ((u + 2) % Lay::RC) * TZZ + cz;
                const T *Cp2 = smt + Lay::off_c / Lay::ES + ((u + 3) % Lay::RC) * TZZ + cz;
                const unsigned char *I0 = smb + Lay::off_i + (u % Lay::RI) * IT_SLOT + cI;
                const unsigned char *I1 = smb + Lay::off_i + ((u + 1) % Lay::RI) * IT_SLOT + cI;
                const T *XZ = B0 + cx, *YZ = B0 + TXX + cy;
                const bool kz1 = k < nz - 1;

                // all three components are computed; ghost points (the last
                // half point of each axis) are simply not stored
                float2 ax1 = dfw_x(lds2(XX - 2), lds2(XX), lds2(XX + 2), ix);
                float2 ax2 = st::dbw<float2>(lds2(XY - 2 * VW), lds2(XY - VW), lds2(XY),
                                             lds2(XY + VW), ix);
                float2 ax3 = st::dbw<float2>(lds2(Bm2 + cx), lds2(Bm1 + cx), lds2(XZ),
                                             lds2(Bp1 + cx), ix);
                float2 ay1 = dbw_x(lds2(XY - 2), lds2(XY), lds2(XY + 2), ix);
                float2 ay2 = st::dfw<float2>(lds2(YY - YW), lds2(YY), lds2(YY + YW),
                                             lds2(YY + 2 * YW), ix);
                float2 ay3 = st::dbw<float2>(lds2(Bm2 + TXX + cy), lds2(Bm1 + TXX + cy), lds2(YZ),
                                             lds2(Bp1 + TXX + cy), ix);
                float2 az1 = dbw_x(lds2(XZ - 2), lds2(XZ), lds2(XZ + 2), ix);
                float2 az2 = st::dbw<float2>(lds2(YZ - 2 * YW), lds2(YZ - YW), lds2(YZ),
                                             lds2(YZ + YW), ix);
                float2 az3 = st::dfw<float2>(lds2(Cm1), lds2(C0), lds2(Cp1), lds2(Cp2), ix);
#pragma unroll
                for (int l = 0; l < 2; ++l) {
                    if (xs[l] < 0) continue;
                    const float2 h = __ldg(&pmlx[p.nmax + i + l]), w = __ldg(&pmlx[i + l]);
                    float t, d;
                    d = st::cpml_v(qx[l][0], h.x, h.y, lane(ax1, l), t);
                    if (l == 0 || ix1) p.psx[ox[l]] = t;
                    set_lane(ax1, l, d);
                    d = st::cpml_v(qx[l][1], w.x, w.y, lane(ay1, l), t);
                    if (jy1) p.psx[Sxs + ox[l]] = t;
                    set_lane(ay1, l, d);
                    d = st::cpml_v(qx[l][2], w.x, w.y, lane(az1, l), t);
                    if (kz1) p.psx[2 * Sxs + ox[l]] = t;
                    set_lane(az1, l, d);
                }
                if (ys >= 0) {
                    const float2 h = __ldg(&pmly[p.nmax + j]), w = __ldg(&pmly[j]);
                    float2 t;
                    ax2 = st::cpml_v(qy[0], splat<float2>(w.x), splat<float2>(w.y), ax2, t);
                    st::st2_or_1(p.psy + oy, t, ix1);
                    ay2 = st::cpml_v(qy[1], splat<float2>(h.x), splat<float2>(h.y), ay2, t);
                    if (jy1) st::st2(p.psy + Sys + oy, t);
                    az2 = st::cpml_v(qy[2], splat<float2>(w.x), splat<float2>(w.y), az2, t);
                    if (kz1) st::st2(p.psy + 2 * Sys + oy, t);
                }
                if (zs >= 0) {
                    const float2 h = __ldg(&pmlz[p.nmax + k]), w = __ldg(&pmlz[k]);
                    float2 t;
                    ax3 = st::cpml_v(qz[0], splat<float2>(w.x), splat<float2>(w.y), ax3, t);
                    st::st2_or_1(p.psz + oz, t, ix1);
                    ay3 = st::cpml_v(qz[1], splat<float2>(w.x), splat<float2>(w.y), ay3, t);
                    if (jy1) st::st2(p.psz + Szs + oz, t);
                    az3 = st::cpml_v(qz[2], splat<float2>(h.x), splat<float2>(h.y), az3, t);
                    if (kz1) st::st2(p.psz + 2 * Szs + oz, t);
                }
                // buoyancy of each voxel's velocity point from the two cells'
                // materials: (i, i+1), (j, j+1), (k, k+1)
                const int nm = p.n_mat;
                const int ma = I0[0], mb = I0[1];
                const float2 bxv = pair(st::buoyancy(p.buoy, nm, ma, mb),
                                        st::buoyancy(p.buoy, nm, mb, I0[2]));
                const float2 byv = pair(st::buoyancy(p.buoy, nm, ma, I0[IW]),
                                        st::buoyancy(p.buoy, nm, mb, I0[IW + 1]));
                const float2 bzv = pair(st::buoyancy(p.buoy, nm, ma, I1[0]),
                                        st::buoyancy(p.buoy, nm, mb, I1[1]));
                st::st2_or_1(vxg + q, st::vel_step(dt, bxv, ux, ax1, ax2, ax3), ix1);
                if (jy1) st::st2(vyg + q, st::vel_step(dt, byv, uy, ay1, ay2, ay3));
                if (kz1) st::st2(vzg + q, st::vel_step(dt, bzv, uz, az1, az2, az3));
            }
            ux = nux;
            uy = nuy;
            uz = nuz;
            q += plane;
            ox[0] += dox;
            ox[1] += dox;
            oy += doy;
        }
    }
    __syncthreads();
    const int ab = *s_abort;
    if (ab >= 0 && tid == 0) drain_after_timeout<2>(bars, ab, 1, k0, k1, p.wait_limit, p.flag);
    if (REUSE) {
        __syncthreads();
        if (tid == 0) {
            tma::mbar_inval(&bars[0]);
            tma::mbar_inval(&bars[1]);
        }
    }
    return ab >= 0;
}

// six resident blocks of 128 threads per SM at the default height (80
// registers); the thread count times blocks per SM is kept for other heights
template <typename T, int TH>
__global__ void __launch_bounds__(PX * TH, 6 * TY / TH)
    k_velocity_tma(const __grid_constant__ AcParams p, int kchunk,
                   const __grid_constant__ VelocityTmaMaps tm)
{
    extern __shared__ __align__(1024) unsigned char smb[];
    velocity_tile<T, false, TH>(p, tm, kchunk, blockIdx.x, blockIdx.y, blockIdx.z, smb);
}

// ------------------------------------------------------------------ stress
// The stencil inputs (velocity tiles with halos, material index) come through
// TMA rings two planes ahead; the per-voxel arrays (stresses, memory
// variables, peak map, FP64 DFT sums) are read straight into registers at the
// top of each plane, so their latency overlaps the ring wait and the
// derivatives, and written back with coalesced stores.
template <int L, typename T, int TH = TY>
struct StressLayout {
    static constexpr int VT = Box<T, TH>::VT, ES = (int)sizeof(T);
    static constexpr int RV = 7, RI = 4;                      // ring depths
    static constexpr int off_v = 0;                           // vx, vy, vz: k-2 .. k+4
    static constexpr int off_i = off_v + RV * 3 * VT * ES;    // index: k .. k+3
    static constexpr int off_bar = off_i + RI * Idx<TH>::SLOT;
    static constexpr int off_abort = off_bar + 24;            // int: plane whose wait ran out
    static constexpr int off_lut = off_bar + 32;
    static size_t bytes(int n_mat) { return off_lut + (size_t)n_mat * sizeof(st::StressCoef); }
    static_assert((VT * ES) % 128 == 0 && off_i % 128 == 0,
                  "TMA destinations must stay 128-byte aligned");
};

// One voxel per thread (block of 32 x 8 threads, 256): the stress update is
// bound by the latency of its per-voxel streams rather than by issue, and
// one voxel per thread keeps 64 registers and 32 resident warps per SM.
constexpr int SNTH = TX * TY;

// One tile (bx, by) over z-chunk bz; REUSE and the result as for velocity_tile.
template <int L, typename T, bool REUSE, int TH = TY>
__device__ __forceinline__ bool stress_tile(const AcParams &p, const StressTmaMaps &tm,
                                            const StepParam &st, int kchunk, int bx, int by,
                                            int bz, unsigned char *smb)
{
    using Lay = StressLayout<L, T, TH>;
    using Bx = Box<T, TH>;
    constexpr int IT = Idx<TH>::BYTES, IT_SLOT = Idx<TH>::SLOT, NT = TX * TH;
    constexpr int VW = Bx::BW, VT = Bx::VT;
    const T *smt = reinterpret_cast<const T *>(smb);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smb + Lay::off_bar);
    volatile int *s_abort = reinterpret_cast<volatile int *>(smb + Lay::off_abort);
    st::StressCoef *s_lut = reinterpret_cast<st::StressCoef *>(smb + Lay::off_lut);

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = bx * TX, y0 = by * TH;
    const int i = x0 + tx, j = y0 + ty;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const bool live = i < nx && j < ny;
    const int k0 = bz * kchunk, k1 = min(nz, k0 + kchunk);
    for (int m = tid; m < p.n_mat; m += NT) s_lut[m] = st::make_stress_coef(p.lut[m], p.Lf);
    if (tid == 0) {
        for (int b = 0; b < 3; ++b) tma::mbar_init(&bars[b], 1);
        tma::mbar_init_fence();
        *s_abort = -1;
    }
    __syncthreads();

    constexpr unsigned VT_BYTES = VT * Lay::ES;
    auto oV = [&](int pl) { return Lay::off_v + ((pl - k0 + 2) % Lay::RV) * 3 * (int)VT_BYTES; };
    auto oI = [&](int pl) { return Lay::off_i + ((pl - k0) % Lay::RI) * IT_SLOT; };   // bytes
    auto issue = [&](int kk, uint64_t *bar, bool first) {
        const unsigned nv = first ? 5 : 1;
        tma::mbar_expect_tx(bar, nv * 3 * VT_BYTES + (first ? 2 : 1) * IT);
        if (p.hold == 2 && kk == p.hold_plane + 2) return;    // test hook: armed, none issued
        for (int pl = first ? kk - 2 : kk + 2; pl <= kk + 2; ++pl)
            for (int a = 0; a < 3; ++a)
                tma::load3d(smb + oV(pl) + a * VT_BYTES, &tm.v[a], x0 - Bx::XO, y0 - 2, pl, bar);
        for (int pl = first ? kk : kk + 1; pl <= kk + 1; ++pl)
            tma::load3d(smb + oI(pl), &tm.idx, x0, y0, pl, bar);
    };
    if (tid == 0) {
        if (REUSE) tma::fence_async_smem();
        issue(k0, &bars[0], true);
        if (k0 + 1 < k1) issue(k0 + 1, &bars[1], false);
    }

    const st::Dx ix = st::make_dx(p.inv_dx);
    const int cv = (ty + 2) * VW + tx + Bx::XO;
    const int ci = ty * IW + tx;
    const int xs = slab_pos(i, nx, p.P), ys = slab_pos(j, ny, p.P);
    const int Sxs = nz * ny * p.W, Sys = nz * p.W * nx, Szs = p.W * ny * nx;
    const float2 *pmlx = p.pml, *pmly = p.pml + 2 * p.nmax, *pmlz = p.pml + 4 * p.nmax;
    T *const gs[6] = {static_cast<T *>(p.sxx), static_cast<T *>(p.syy), static_cast<T *>(p.szz),
                      static_cast<T *>(p.sxy), static_cast<T *>(p.sxz), static_cast<T *>(p.syz)};
    T *__restrict__ mem = static_cast<T *>(p.mem);

    // Ring positions of this thread's column, rotated once per plane: the
    // velocity ring at planes k-2 .. k+2 (element offsets of the vx centre)
    // and the index ring at k, k+1 (bytes).
    const int vbase = Lay::off_v / Lay::ES, vend = vbase + Lay::RV * 3 * VT;
    const int ibase = Lay::off_i, iend = ibase + Lay::RI * IT_SLOT;
    int vM2 = vbase + cv, vM1 = vM2 + 3 * VT, vK = vM1 + 3 * VT, vP1 = vK + 3 * VT,
        vP2 = vP1 + 3 * VT;
    int iK = ibase + ci, iK1 = iK + IT_SLOT;

    // L2 prefetch of the next plane's per-voxel rows.  A tile row of one
    // stream is 32 elements (stresses, the peak map), 32 L (the memory
    // variables of a component, mechanisms adjacent) or 32 doubles (the DFT
    // sums); its 128-byte lines are numbered over all streams and thread
    // (row r, slot a) prefetches line a of row y0 + r.  Every line starts at
    // an element of the row segment, inside its array.  FP32 storage only:
    // with FP16 storage the kernel is bound by issue, not by the latency of
    // its streams, and the prefetch's instructions cost more than it saves.
    constexpr bool PREFETCH = sizeof(T) == 4;
    const int pf_r = tid >> 5, pf_a = tid & 31;
    const bool pk_on = (st.flags & kStepPeak) != 0, dft_on = (st.flags & kStepDft) != 0;
    constexpr int LS = (32 * (int)sizeof(T) + 127) / 128;              // lines of a stress row
    constexpr int LM = (32 * (L > 0 ? L : 1) * (int)sizeof(T) + 127) / 128;   // of a memory row
    const int n_lines = 6 * LS + (L > 0 ? 6 * LM : 0) + (pk_on ? 1 : 0) + (dft_on ? 4 : 0);
    const T *st0 = static_cast<const T *>(p.sxx);     // stresses: consecutive arrays, fstride apart
    auto prefetch_plane = [&](int kp) {
        if (kp >= k1 || y0 + pf_r >= ny || pf_a >= n_lines) return;
        const size_t e = (size_t)kp * nx * ny + (size_t)(y0 + pf_r) * nx + x0;
        int a = pf_a;
        const char *ln;
        if (a < 6 * LS) {
            ln = reinterpret_cast<const char *>(st0 + (size_t)(a / LS) * p.fstride + e) + (a % LS) * 128;
        } else if ((a -= 6 * LS) < (L > 0 ? 6 * LM : 0)) {
            ln = reinterpret_cast<const char *>(mem + mem_index(0, a / LM, e, p.fstride, L)) +
                 (a % LM) * 128;
        } else {
            a -= (L > 0 ? 6 * LM : 0);
            if (pk_on && a == 0) {
                ln = reinterpret_cast<const char *>(p.peak + e);
            } else {
                a -= pk_on ? 1 : 0;                    // 0, 1: dftC lines; 2, 3: dftS lines
                if ((a & 1) && x0 + 16 >= nx) return;
                ln = reinterpret_cast<const char *>(((a >> 1) ? p.dftS : p.dftC) + e) + (a & 1) * 128;
            }
        }
        tma::prefetch_l2(ln);
    };
    if (PREFETCH) prefetch_plane(k0);

    // Blocks whose tile touches no CPML slab in x or y and holds no ghost
    // or out-of-grid point run a copy of the loop without that code.
    const bool edge = !(x0 >= p.P && x0 + TX - 1 < nx - p.P - 1 && y0 >= p.P &&
                        y0 + TH - 1 < ny - p.P - 1);
    auto march = [&](auto edge_tag) {
    constexpr bool EDGE = decltype(edge_tag)::value;
    const bool lv = EDGE ? live : true;
    int it = 0;
    for (int k = k0; k < k1; ++k, ++it) {
        __syncthreads();
        if (*s_abort >= 0) break;        // a wait of the previous plane ran out
        if (tid == 0 && k + 2 < k1) {
            tma::fence_async_smem();
            issue(k + 2, &bars[(it + 2) % 3], false);
        }
        if (PREFETCH) prefetch_plane(k + 1);
        const int q = k * (nx * ny) + j * nx + i;
        // per-voxel loads first, in flight while the ring wait and the
        // derivatives proceed
        float sv[6], rv[L > 0 ? L : 1][6];
        float pk = 0.0f;
        double dC = 0.0, dS = 0.0;
        // CPML memories of this voxel: components 3-5 of each slab it lies in,
        // i.e. [normal, then the two shear derivatives along that axis]
        const int zs = slab_pos(k, nz, p.P);
        const int ox = (k * ny + j) * p.W + xs, oy = (k * p.W + ys) * nx + i,
                  oz = (zs * ny + j) * nx + i;
        float qx[3] = {0.0f, 0.0f, 0.0f}, qy[3] = {0.0f, 0.0f, 0.0f}, qz[3] = {0.0f, 0.0f, 0.0f};
        if (lv) {
            if (EDGE && xs >= 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) qx[c] = p.psx[(3 + c) * Sxs + ox];
            }
            if (EDGE && ys >= 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) qy[c] = p.psy[(3 + c) * Sys + oy];
            }
            if (zs >= 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) qz[c] = p.psz[(3 + c) * Szs + oz];
            }
        }
        if (lv) {
#pragma unroll
            for (int cc = 0; cc < 6; ++cc) sv[cc] = tof(gs[cc][q]);
#pragma unroll
            for (int cc = 0; cc < 6; ++cc) {
                if constexpr (L == 2) {   // the two mechanisms of a component: one paired load
                    const float2 r2 = st::ld2(mem + mem_index(0, cc, q, p.fstride, 2));
                    rv[0][cc] = r2.x;
                    rv[1][cc] = r2.y;
                } else if constexpr (L == 1) {
                    rv[0][cc] = tof(mem[mem_index(0, cc, q, p.fstride, 1)]);
                }
            }
            if (st.flags & kStepPeak) pk = p.peak[q];
            if (st.flags & kStepDft) {
                dC = p.dftC[q];
                dS = p.dftS[q];
            }
        }
        const bool ready = tma::mbar_wait(&bars[it % 3], (it / 3) & 1, p.wait_limit);
        if (!ready) *s_abort = k;
        if (ready && lv) {
            const int vm2 = vM2, vm1 = vM1, vp1 = vP1, vp2 = vP2;
            const unsigned char *I0 = smb + iK;
            const unsigned char *I1 = smb + iK1;
            const bool ix1 = !EDGE || i < nx - 1, jy1 = !EDGE || j < ny - 1, kz1 = k < nz - 1;
            const int m00 = I0[0];
            const st::StressCoef c0 = s_lut[m00];
            const int vx = vK, vy = vK + VT, vz = vK + 2 * VT;

            // ---- normal stresses at (i, j, k)
            float exx = dbw(tof(smt[vx - 2]), tof(smt[vx - 1]), tof(smt[vx]), tof(smt[vx + 1]), ix);
            float eyy = dbw(tof(smt[vy - 2 * VW]), tof(smt[vy - VW]), tof(smt[vy]),
                            tof(smt[vy + VW]), ix);
            float ezz = dbw(tof(smt[vm2 + 2 * VT]), tof(smt[vm1 + 2 * VT]), tof(smt[vz]),
                            tof(smt[vp1 + 2 * VT]), ix);
            if (EDGE && xs >= 0) exx = st::cpml_pre(p.psx + 3 * Sxs + ox, qx[0], __ldg(&pmlx[i]), exx);
            if (EDGE && ys >= 0) eyy = st::cpml_pre(p.psy + 3 * Sys + oy, qy[0], __ldg(&pmly[j]), eyy);
            if (zs >= 0) ezz = st::cpml_pre(p.psz + 3 * Szs + oz, qz[0], __ldg(&pmlz[k]), ezz);
            float srcv = 0.0f;
            if ((st.flags & kStepSource) && k == p.k_src) {
                const float2 a = p.src[j * nx + i];
                srcv = st::source_value<float>(p.src_scale, a.x, a.y, st.src_ws, st.src_wc);
            }
            st::normal_update<L>(p, c0, exx, eyy, ezz, srcv, sv, rv);
            const float pr = st::pressure(sv);
            if (!isfinite(pr)) atomicOr(p.flag, 1);

            // ---- shear stresses (ghost points computed, not stored)
            const bool dxy = ix1 && jy1, dxz = ix1 && kz1, dyz = jy1 && kz1;
            {                                        // sxy at (i+1/2, j+1/2, k)
                float a = dfw(tof(smt[vx - VW]), tof(smt[vx]), tof(smt[vx + VW]),
                              tof(smt[vx + 2 * VW]), ix);
                float b = dfw(tof(smt[vy - 1]), tof(smt[vy]), tof(smt[vy + 1]), tof(smt[vy + 2]), ix);
                if (EDGE && ys >= 0) {
                    const float2 h = __ldg(&pmly[p.nmax + j]);
                    float t;
                    a = st::cpml_v(qy[1], h.x, h.y, a, t);
                    if (dxy) p.psy[4 * Sys + oy] = t;
                }
                if (EDGE && xs >= 0) {
                    const float2 h = __ldg(&pmlx[p.nmax + i]);
                    float t;
                    b = st::cpml_v(qx[1], h.x, h.y, b, t);
                    if (dxy) p.psx[4 * Sxs + ox] = t;
                }
                st::shear_update<L>(p, s_lut, c0, m00, I0[1], I0[IW], I0[IW + 1], st::vadd(a, b), 3, sv, rv);
            }
            {                                        // sxz at (i+1/2, j, k+1/2)
                float a = dfw(tof(smt[vm1]), tof(smt[vx]), tof(smt[vp1]), tof(smt[vp2]), ix);
                float b = dfw(tof(smt[vz - 1]), tof(smt[vz]), tof(smt[vz + 1]), tof(smt[vz + 2]), ix);
                if (zs >= 0) {
                    const float2 h = __ldg(&pmlz[p.nmax + k]);
                    float t;
                    a = st::cpml_v(qz[1], h.x, h.y, a, t);
                    if (dxz) p.psz[4 * Szs + oz] = t;
                }
                if (EDGE && xs >= 0) {
                    const float2 h = __ldg(&pmlx[p.nmax + i]);
                    float t;
                    b = st::cpml_v(qx[2], h.x, h.y, b, t);
                    if (dxz) p.psx[5 * Sxs + ox] = t;
                }
                st::shear_update<L>(p, s_lut, c0, m00, I0[1], I1[0], I1[1], st::vadd(a, b), 4, sv, rv);
            }
            {                                        // syz at (i, j+1/2, k+1/2)
                float a = dfw(tof(smt[vm1 + VT]), tof(smt[vy]), tof(smt[vp1 + VT]),
                              tof(smt[vp2 + VT]), ix);
                float b = dfw(tof(smt[vz - VW]), tof(smt[vz]), tof(smt[vz + VW]),
                              tof(smt[vz + 2 * VW]), ix);
                if (zs >= 0) {
                    const float2 h = __ldg(&pmlz[p.nmax + k]);
                    float t;
                    a = st::cpml_v(qz[2], h.x, h.y, a, t);
                    if (dyz) p.psz[5 * Szs + oz] = t;
                }
                if (EDGE && ys >= 0) {
                    const float2 h = __ldg(&pmly[p.nmax + j]);
                    float t;
                    b = st::cpml_v(qy[2], h.x, h.y, b, t);
                    if (dyz) p.psy[5 * Sys + oy] = t;
                }
                st::shear_update<L>(p, s_lut, c0, m00, I0[IW], I1[0], I1[IW], st::vadd(a, b), 5, sv, rv);
            }

            // ---- results (ghost points are not written)
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) st::stv(gs[cc] + q, sv[cc]);
            if (dxy) st::stv(gs[3] + q, sv[3]);
            if (dxz) st::stv(gs[4] + q, sv[4]);
            if (dyz) st::stv(gs[5] + q, sv[5]);
#pragma unroll
            for (int cc = 0; cc < 6; ++cc) {
                const bool w = cc < 3 || (cc == 3 && dxy) || (cc == 4 && dxz) || (cc == 5 && dyz);
                if (!w) continue;
                if constexpr (L == 2)
                    st::st2(mem + mem_index(0, cc, q, p.fstride, 2), pair(rv[0][cc], rv[1][cc]));
                else if constexpr (L == 1)
                    st::stv(mem + mem_index(0, cc, q, p.fstride, 1), rv[0][cc]);
            }
            if (st.flags & kStepPeak) p.peak[q] = fmaxf(pk, fabsf(pr));
            if (st.flags & kStepDft) {
                p.dftC[q] = fma((double)pr, st.cw, dC);
                p.dftS[q] = fma((double)pr, st.sw, dS);
            }
        }
        // rotate the ring positions to plane k+1
        vM2 = vM1; vM1 = vK; vK = vP1; vP1 = vP2;
        vP2 += 3 * VT;
        if (vP2 >= vend) vP2 -= Lay::RV * 3 * VT;
        iK = iK1;
        iK1 += IT_SLOT;
        if (iK1 >= iend) iK1 -= Lay::RI * IT_SLOT;
    }
    };
    if (edge)
        march(std::true_type{});
    else
        march(std::false_type{});
    __syncthreads();
    const int ab = *s_abort;
    if (ab >= 0 && tid == 0) drain_after_timeout<3>(bars, ab, 2, k0, k1, p.wait_limit, p.flag);
    if (REUSE) {
        __syncthreads();
        if (tid == 0)
            for (int b = 0; b < 3; ++b) tma::mbar_inval(&bars[b]);
    }
    return ab >= 0;
}

// ------------------------------------------------ stress, FP16 storage, pairs
// With FP16 storage the stress update is bound by issue, so it takes the
// velocity kernel's layout instead: 16 x 8 threads, thread (tx, ty) owns the
// voxel pair (x0 + 2 tx, x0 + 2 tx + 1) of row y0 + ty.  The pair's streams
// stay packed as loaded (a half2 per stress, the four halves of a
// component's two memory variables as one 8-byte word) and are unpacked
// where they are used, so two voxels' streams take the registers one voxel's
// take in FP32.  The rings, the copies and every arithmetic step are those of
// stress_tile on FP32x2 pairs (bit for bit the same results).
constexpr int kStressH2Blocks = 5;   // resident blocks of 128 threads per SM (96 registers)

__device__ __forceinline__ float2 h2f(__half2 v) { return __half22float2(v); }
__device__ __forceinline__ __half2 f2h(float2 v) { return __floats2half2_rn(v.x, v.y); }

// the two mechanisms of a component for both voxels: halves
// (q, 0), (q, 1), (q + 1, 0), (q + 1, 1) of one 8-byte word
__device__ __forceinline__ void unpack_mem2(uint2 w, float2 &r0, float2 &r1)
{
    const float2 a = h2f(*reinterpret_cast<const __half2 *>(&w.x));   // (q,0), (q,1)
    const float2 b = h2f(*reinterpret_cast<const __half2 *>(&w.y));   // (q+1,0), (q+1,1)
    r0 = make_float2(a.x, b.x);
    r1 = make_float2(a.y, b.y);
}
__device__ __forceinline__ uint2 pack_mem2(float2 r0, float2 r1)
{
    const __half2 a = __floats2half2_rn(r0.x, r1.x), b = __floats2half2_rn(r0.y, r1.y);
    uint2 w;
    w.x = *reinterpret_cast<const unsigned *>(&a);
    w.y = *reinterpret_cast<const unsigned *>(&b);
    return w;
}

template <int L, bool REUSE, int TH = TY>
__device__ __forceinline__ bool stress_tile_h2(const AcParams &p, const StressTmaMaps &tm,
                                               const StepParam &st, int kchunk, int bx, int by,
                                               int bz, unsigned char *smb)
{
    using T = __half;
    using Lay = StressLayout<L, T, TH>;
    using Bx = Box<T, TH>;
    constexpr int IT = Idx<TH>::BYTES, IT_SLOT = Idx<TH>::SLOT, NT = PX * TH;
    constexpr int VW = Bx::BW, VT = Bx::VT;
    const T *smt = reinterpret_cast<const T *>(smb);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smb + Lay::off_bar);
    volatile int *s_abort = reinterpret_cast<volatile int *>(smb + Lay::off_abort);
    st::StressCoef *s_lut = reinterpret_cast<st::StressCoef *>(smb + Lay::off_lut);

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * PX + tx;
    const int x0 = bx * TX, y0 = by * TH;
    const int i = x0 + 2 * tx, j = y0 + ty;           // the pair (i, i+1) of row j
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const bool live = i < nx && j < ny;                // nx is even: i + 1 < nx as well
    const int k0 = bz * kchunk, k1 = min(nz, k0 + kchunk);
    for (int m = tid; m < p.n_mat; m += NT) s_lut[m] = st::make_stress_coef(p.lut[m], p.Lf);
    if (tid == 0) {
        for (int b = 0; b < 3; ++b) tma::mbar_init(&bars[b], 1);
        tma::mbar_init_fence();
        *s_abort = -1;
    }
    __syncthreads();

    constexpr unsigned VT_BYTES = VT * Lay::ES;
    auto oV = [&](int pl) { return Lay::off_v + ((pl - k0 + 2) % Lay::RV) * 3 * (int)VT_BYTES; };
    auto oI = [&](int pl) { return Lay::off_i + ((pl - k0) % Lay::RI) * IT_SLOT; };   // bytes
    auto issue = [&](int kk, uint64_t *bar, bool first) {
        const unsigned nv = first ? 5 : 1;
        tma::mbar_expect_tx(bar, nv * 3 * VT_BYTES + (first ? 2 : 1) * IT);
        if (p.hold == 2 && kk == p.hold_plane + 2) return;    // test hook: armed, none issued
        for (int pl = first ? kk - 2 : kk + 2; pl <= kk + 2; ++pl)
            for (int a = 0; a < 3; ++a)
                tma::load3d(smb + oV(pl) + a * VT_BYTES, &tm.v[a], x0 - Bx::XO, y0 - 2, pl, bar);
        for (int pl = first ? kk : kk + 1; pl <= kk + 1; ++pl)
            tma::load3d(smb + oI(pl), &tm.idx, x0, y0, pl, bar);
    };
    if (tid == 0) {
        if (REUSE) tma::fence_async_smem();
        issue(k0, &bars[0], true);
        if (k0 + 1 < k1) issue(k0 + 1, &bars[1], false);
    }

    const st::Dx ix = st::make_dx(p.inv_dx);
    const int cv = (ty + 2) * VW + 2 * tx + Bx::XO;    // even: every pair read is aligned
    const int ci = ty * IW + 2 * tx;
    const int xs[2] = {slab_pos(i, nx, p.P), slab_pos(i + 1, nx, p.P)};
    const int ys = slab_pos(j, ny, p.P);
    const int Sxs = nz * ny * p.W, Sys = nz * p.W * nx, Szs = p.W * ny * nx;
    const float2 *pmlx = p.pml, *pmly = p.pml + 2 * p.nmax, *pmlz = p.pml + 4 * p.nmax;
    T *const gs[6] = {static_cast<T *>(p.sxx), static_cast<T *>(p.syy), static_cast<T *>(p.szz),
                      static_cast<T *>(p.sxy), static_cast<T *>(p.sxz), static_cast<T *>(p.syz)};
    T *__restrict__ mem = static_cast<T *>(p.mem);
    // the pair's second voxel is not the last point in x (the first never is)
    const bool ix1 = i + 1 < nx - 1;

    const int vbase = Lay::off_v / Lay::ES, vend = vbase + Lay::RV * 3 * VT;
    const int ibase = Lay::off_i, iend = ibase + Lay::RI * IT_SLOT;
    int vM2 = vbase + cv, vM1 = vM2 + 3 * VT, vK = vM1 + 3 * VT, vP1 = vK + 3 * VT,
        vP2 = vP1 + 3 * VT;
    int iK = ibase + ci, iK1 = iK + IT_SLOT;

    // one copy of the plane loop for every tile: the paired tile's code is
    // large, and an interior-tile copy without the CPML code costs more in
    // instruction fetch than the CPML branches it saves
    auto march = [&](auto edge_tag) {
    constexpr bool EDGE = decltype(edge_tag)::value;
    const bool lv = EDGE ? live : true;
    int it = 0;
    for (int k = k0; k < k1; ++k, ++it) {
        __syncthreads();
        if (*s_abort >= 0) break;        // a wait of the previous plane ran out
        if (tid == 0 && k + 2 < k1) {
            tma::fence_async_smem();
            issue(k + 2, &bars[(it + 2) % 3], false);
        }
        const int q = k * (nx * ny) + j * nx + i;
        // the pair's streams, packed, in flight while the ring wait and the
        // derivatives proceed
        __half2 sp[6];
        [[maybe_unused]] uint2 rp[6];      // L = 2: one word per component
        [[maybe_unused]] __half2 rp1[6];   // L = 1
        float2 pk = make_float2(0.0f, 0.0f);
        double2 dC = make_double2(0.0, 0.0), dS = dC;
        const int zs = slab_pos(k, nz, p.P);
        const int ox[2] = {(k * ny + j) * p.W + xs[0], (k * ny + j) * p.W + xs[1]};
        const int oy = (k * p.W + ys) * nx + i, oz = (zs * ny + j) * nx + i;
        float qx[2][3] = {{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};
        float2 qy[3] = {pair(0.0f, 0.0f), pair(0.0f, 0.0f), pair(0.0f, 0.0f)};
        float2 qz[3] = {qy[0], qy[0], qy[0]};
        if (lv) {
            if (EDGE) {
#pragma unroll
                for (int l = 0; l < 2; ++l)
                    if (xs[l] >= 0) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) qx[l][c] = p.psx[(3 + c) * Sxs + ox[l]];
                    }
                if (ys >= 0) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) qy[c] = st::ld2(p.psy + (3 + c) * Sys + oy);
                }
            }
            if (zs >= 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) qz[c] = st::ld2(p.psz + (3 + c) * Szs + oz);
            }
#pragma unroll
            for (int cc = 0; cc < 6; ++cc) sp[cc] = *reinterpret_cast<const __half2 *>(gs[cc] + q);
#pragma unroll
            for (int cc = 0; cc < 6; ++cc) {
                if constexpr (L == 2)
                    rp[cc] = *reinterpret_cast<const uint2 *>(mem + mem_index(0, cc, q, p.fstride, 2));
                else if constexpr (L == 1)
                    rp1[cc] = *reinterpret_cast<const __half2 *>(mem + mem_index(0, cc, q, p.fstride, 1));
            }
            if (st.flags & kStepPeak) pk = *reinterpret_cast<const float2 *>(p.peak + q);
            if (st.flags & kStepDft) {
                dC = *reinterpret_cast<const double2 *>(p.dftC + q);
                dS = *reinterpret_cast<const double2 *>(p.dftS + q);
            }
        }
        const bool ready = tma::mbar_wait(&bars[it % 3], (it / 3) & 1, p.wait_limit);
        if (!ready) *s_abort = k;
        if (ready && lv) {
            const int vm2 = vM2, vm1 = vM1, vp1 = vP1, vp2 = vP2;
            const unsigned char *I0 = smb + iK;
            const unsigned char *I1 = smb + iK1;
            const bool jy1 = !EDGE || j < ny - 1, kz1 = k < nz - 1;
            const int ma = I0[0], mb = I0[1];
            const st::StressCoef &ca = s_lut[ma], &cb = s_lut[mb];
            const int vx = vK, vy = vK + VT, vz = vK + 2 * VT;
            // a component's stress and memory variables are unpacked just
            // before its update and stored right after it
            float2 sv[6], rv[L > 0 ? L : 1][6];
            auto unpack = [&](int cc) {
                sv[cc] = h2f(sp[cc]);
                if constexpr (L == 2)
                    unpack_mem2(rp[cc], rv[0][cc], rv[1][cc]);
                else if constexpr (L == 1)
                    rv[0][cc] = h2f(rp1[cc]);
            };
            auto put_s = [&](int cc, bool both) {
                if (both)
                    *reinterpret_cast<__half2 *>(gs[cc] + q) = f2h(sv[cc]);
                else
                    gs[cc][q] = __float2half_rn(sv[cc].x);
            };
            auto put_r = [&](int cc, bool both) {
                if constexpr (L == 2) {
                    const uint2 w = pack_mem2(rv[0][cc], rv[1][cc]);
                    T *r = mem + mem_index(0, cc, q, p.fstride, 2);
                    if (both)
                        *reinterpret_cast<uint2 *>(r) = w;
                    else
                        *reinterpret_cast<unsigned *>(r) = w.x;
                } else if constexpr (L == 1) {
                    T *r = mem + mem_index(0, cc, q, p.fstride, 1);
                    if (both)
                        *reinterpret_cast<__half2 *>(r) = f2h(rv[0][cc]);
                    else
                        *r = __float2half_rn(rv[0][cc].x);
                }
            };

            // ---- normal stresses at (i, j, k), (i + 1, j, k)
            float2 exx = dbw_x(lds2(smt + vx - 2), lds2(smt + vx), lds2(smt + vx + 2), ix);
            float2 eyy = st::dbw<float2>(lds2(smt + vy - 2 * VW), lds2(smt + vy - VW),
                                         lds2(smt + vy), lds2(smt + vy + VW), ix);
            float2 ezz = st::dbw<float2>(lds2(smt + vm2 + 2 * VT), lds2(smt + vm1 + 2 * VT),
                                         lds2(smt + vz), lds2(smt + vp1 + 2 * VT), ix);
            if (EDGE) {
#pragma unroll
                for (int l = 0; l < 2; ++l)
                    if (xs[l] >= 0)
                        set_lane(exx, l, st::cpml_pre(p.psx + 3 * Sxs + ox[l], qx[l][0],
                                                      __ldg(&pmlx[i + l]), lane(exx, l)));
                if (ys >= 0) {
                    const float2 w = __ldg(&pmly[j]);
                    float2 t;
                    eyy = st::cpml_v(qy[0], splat<float2>(w.x), splat<float2>(w.y), eyy, t);
                    st::st2(p.psy + 3 * Sys + oy, t);
                }
            }
            if (zs >= 0) {
                const float2 w = __ldg(&pmlz[k]);
                float2 t;
                ezz = st::cpml_v(qz[0], splat<float2>(w.x), splat<float2>(w.y), ezz, t);
                st::st2(p.psz + 3 * Szs + oz, t);
            }
            float2 srcv = pair(0.0f, 0.0f);
            if ((st.flags & kStepSource) && k == p.k_src) {
                const float4 a = *reinterpret_cast<const float4 *>(p.src + j * nx + i);
                srcv = st::source_value<float2>(p.src_scale, pair(a.x, a.z), pair(a.y, a.w),
                                                st.src_ws, st.src_wc);
            }
            unpack(0);
            unpack(1);
            unpack(2);
            st::normal_update<L, float2>(p, pair(ca.piU, cb.piU), pair(ca.piT, cb.piT),
                                         pair(ca.nmu2U, cb.nmu2U), pair(ca.nmu2T, cb.nmu2T), exx,
                                         eyy, ezz, srcv, sv, rv);
            const float2 pr = st::pressure(sv);
            if (!isfinite(pr.x) || !isfinite(pr.y)) atomicOr(p.flag, 1);
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
                put_s(cc, true);
                put_r(cc, true);
            }

            // ---- shear stresses (ghost points computed, not stored)
            auto coef = [&](int mb0, int md0, int mf0, int mb1, int md1, int mf1, float2 &psic,
                            float2 &thec) {
                st::shear_coef(s_lut, ca, ma, mb0, md0, mf0, p.Lf, psic.x, thec.x);
                st::shear_coef(s_lut, cb, mb, mb1, md1, mf1, p.Lf, psic.y, thec.y);
            };
            {                                        // sxy at (i+1/2, j+1/2, k)
                float2 a = st::dfw<float2>(lds2(smt + vx - VW), lds2(smt + vx),
                                           lds2(smt + vx + VW), lds2(smt + vx + 2 * VW), ix);
                float2 b = dfw_x(lds2(smt + vy - 2), lds2(smt + vy), lds2(smt + vy + 2), ix);
                if (EDGE && ys >= 0) {
                    const float2 h = __ldg(&pmly[p.nmax + j]);
                    float2 t;
                    a = st::cpml_v(qy[1], splat<float2>(h.x), splat<float2>(h.y), a, t);
                    if (jy1) st::st2_or_1(p.psy + 4 * Sys + oy, t, ix1);
                }
                if (EDGE) {
#pragma unroll
                    for (int l = 0; l < 2; ++l) {
                        if (xs[l] < 0) continue;
                        const float2 h = __ldg(&pmlx[p.nmax + i + l]);
                        float t;
                        set_lane(b, l, st::cpml_v(qx[l][1], h.x, h.y, lane(b, l), t));
                        if (jy1 && (l == 0 || ix1)) p.psx[4 * Sxs + ox[l]] = t;
                    }
                }
                float2 psic, thec;
                coef(mb, I0[IW], I0[IW + 1], I0[2], I0[IW + 1], I0[IW + 2], psic, thec);
                unpack(3);
                st::shear_update<L, float2>(p, psic, thec, st::vadd(a, b), 3, sv, rv);
                if (jy1) {
                    put_s(3, ix1);
                    put_r(3, ix1);
                }
            }
            {                                        // sxz at (i+1/2, j, k+1/2)
                float2 a = st::dfw<float2>(lds2(smt + vm1), lds2(smt + vx), lds2(smt + vp1),
                                           lds2(smt + vp2), ix);
                float2 b = dfw_x(lds2(smt + vz - 2), lds2(smt + vz), lds2(smt + vz + 2), ix);
                if (zs >= 0) {
                    const float2 h = __ldg(&pmlz[p.nmax + k]);
                    float2 t;
                    a = st::cpml_v(qz[1], splat<float2>(h.x), splat<float2>(h.y), a, t);
                    if (kz1) st::st2_or_1(p.psz + 4 * Szs + oz, t, ix1);
                }
                if (EDGE) {
#pragma unroll
                    for (int l = 0; l < 2; ++l) {
                        if (xs[l] < 0) continue;
                        const float2 h = __ldg(&pmlx[p.nmax + i + l]);
                        float t;
                        set_lane(b, l, st::cpml_v(qx[l][2], h.x, h.y, lane(b, l), t));
                        if (kz1 && (l == 0 || ix1)) p.psx[5 * Sxs + ox[l]] = t;
                    }
                }
                float2 psic, thec;
                coef(mb, I1[0], I1[1], I0[2], I1[1], I1[2], psic, thec);
                unpack(4);
                st::shear_update<L, float2>(p, psic, thec, st::vadd(a, b), 4, sv, rv);
                if (kz1) {
                    put_s(4, ix1);
                    put_r(4, ix1);
                }
            }
            {                                        // syz at (i, j+1/2, k+1/2)
                float2 a = st::dfw<float2>(lds2(smt + vm1 + VT), lds2(smt + vy),
                                           lds2(smt + vp1 + VT), lds2(smt + vp2 + VT), ix);
                float2 b = st::dfw<float2>(lds2(smt + vz - VW), lds2(smt + vz),
                                           lds2(smt + vz + VW), lds2(smt + vz + 2 * VW), ix);
                if (zs >= 0) {
                    const float2 h = __ldg(&pmlz[p.nmax + k]);
                    float2 t;
                    a = st::cpml_v(qz[2], splat<float2>(h.x), splat<float2>(h.y), a, t);
                    if (jy1 && kz1) st::st2(p.psz + 5 * Szs + oz, t);
                }
                if (EDGE && ys >= 0) {
                    const float2 h = __ldg(&pmly[p.nmax + j]);
                    float2 t;
                    b = st::cpml_v(qy[2], splat<float2>(h.x), splat<float2>(h.y), b, t);
                    if (jy1 && kz1) st::st2(p.psy + 5 * Sys + oy, t);
                }
                float2 psic, thec;
                coef(I0[IW], I1[0], I1[IW], I0[IW + 1], I1[1], I1[IW + 1], psic, thec);
                unpack(5);
                st::shear_update<L, float2>(p, psic, thec, st::vadd(a, b), 5, sv, rv);
                if (jy1 && kz1) {
                    put_s(5, true);
                    put_r(5, true);
                }
            }

            // ---- capture (ghost points are not written above)
            if (st.flags & kStepPeak)
                *reinterpret_cast<float2 *>(p.peak + q) =
                    make_float2(fmaxf(pk.x, fabsf(pr.x)), fmaxf(pk.y, fabsf(pr.y)));
            if (st.flags & kStepDft) {
                *reinterpret_cast<double2 *>(p.dftC + q) =
                    make_double2(fma((double)pr.x, st.cw, dC.x), fma((double)pr.y, st.cw, dC.y));
                *reinterpret_cast<double2 *>(p.dftS + q) =
                    make_double2(fma((double)pr.x, st.sw, dS.x), fma((double)pr.y, st.sw, dS.y));
            }
        }
        // rotate the ring positions to plane k+1
        vM2 = vM1; vM1 = vK; vK = vP1; vP1 = vP2;
        vP2 += 3 * VT;
        if (vP2 >= vend) vP2 -= Lay::RV * 3 * VT;
        iK = iK1;
        iK1 += IT_SLOT;
        if (iK1 >= iend) iK1 -= Lay::RI * IT_SLOT;
    }
    };
    march(std::true_type{});
    __syncthreads();
    const int ab = *s_abort;
    if (ab >= 0 && tid == 0) drain_after_timeout<3>(bars, ab, 2, k0, k1, p.wait_limit, p.flag);
    if (REUSE) {
        __syncthreads();
        if (tid == 0)
            for (int b = 0; b < 3; ++b) tma::mbar_inval(&bars[b]);
    }
    return ab >= 0;
}

template <int L, int MINB, int TH>
__global__ void __launch_bounds__(PX * TH, MINB)
    k_stress_tma_h2(const __grid_constant__ AcParams p, int kchunk,
                    const __grid_constant__ StressTmaMaps tm)
{
    extern __shared__ __align__(1024) unsigned char smb[];
    stress_tile_h2<L, false, TH>(p, tm, p.st, kchunk, blockIdx.x, blockIdx.y, blockIdx.z, smb);
}

template <int L, int MINB, typename T, int TH>
__global__ void __launch_bounds__(TX * TH, MINB)
    k_stress_tma(const __grid_constant__ AcParams p, int kchunk,
                 const __grid_constant__ StressTmaMaps tm)
{
    extern __shared__ __align__(1024) unsigned char smb[];
    stress_tile<L, T, false, TH>(p, tm, p.st, kchunk, blockIdx.x, blockIdx.y, blockIdx.z, smb);
}

// ------------------------------------------------------------------ batch
// Persistent kernels over a work list spanning several domains: block b takes
// items b, b + gridDim.x, ...; an item is one tile and z-chunk of one domain.
// The domain's parameters are copied to shared memory and the tile runs the
// same code as the single-domain kernels.  Domains whose run has ended by
// this step are skipped.

// Per-block walk over the work list, kept in shared memory so that nothing
// but the tile's own state is live in registers during a tile.  A block's
// items ascend, so its domain index only moves forward: thread 0 scans on
// from the previous domain and skips items of domains that have finished.
struct WalkState {
    int w, d, loaded, step;
    int fresh;          // the item's domain differs from the previous item's
};

__device__ __forceinline__ void walk_begin(WalkState &ws, const int *step_ctr, int tid)
{
    if (tid == 0) {
        ws.w = (int)blockIdx.x - (int)gridDim.x;
        ws.d = 0;
        ws.loaded = -1;
        ws.step = *step_ctr;
    }
}

// thread 0: move to the next item of an unfinished domain (w = -1 at the end)
__device__ __forceinline__ void walk_next(WalkState &ws, const BatchParams &bp)
{
    int w = ws.w, d = ws.d;
    for (;;) {
        w += gridDim.x;
        if (w >= bp.total) {
            w = -1;
            break;
        }
        while (d + 1 < bp.n_dom && bp.block0[d + 1] <= w) ++d;
        if (ws.step < bp.n_steps[d]) break;
    }
    ws.w = w;
    ws.d = d;
    ws.fresh = (w >= 0 && d != ws.loaded) ? 1 : 0;
    if (ws.fresh) ws.loaded = d;
}

template <typename T>
__global__ void __launch_bounds__(NTH, 6)
    k_velocity_batch(const __grid_constant__ BatchParams bp, const int *step_ctr)
{
    extern __shared__ __align__(1024) unsigned char smb[];
    __shared__ WalkState ws;
    const int tid = threadIdx.y * PX + threadIdx.x;
    walk_begin(ws, step_ctr, tid);
    for (;;) {
        __syncthreads();
        if (tid == 0) walk_next(ws, bp);
        __syncthreads();
        if (ws.w < 0) break;
        const int d = ws.d;
        if (tid == 0 && ws.fresh) {
            // tensor maps in device memory, written before the launch
            for (int g = 0; g < 6; ++g) tma::tensormap_acquire(&bp.vm[d].sg[g]);
            tma::tensormap_acquire(&bp.vm[d].idx);
        }
        const int li = ws.w - bp.block0[d], tx_ = bp.tiles_x[d], txy = tx_ * bp.tiles_y[d];
        if (velocity_tile<T, true>(bp.p[d], bp.vm[d], bp.kchunk[d], li % tx_, (li % txy) / tx_,
                                   li / txy, smb))
            break;
    }
}

template <int L, int MINB, typename T>
__global__ void __launch_bounds__(SNTH, MINB)
    k_stress_batch(const __grid_constant__ BatchParams bp, const int *step_ctr)
{
    extern __shared__ __align__(1024) unsigned char smb[];
    __shared__ WalkState ws;
    __shared__ StepParam sq;
    const int tid = threadIdx.y * TX + threadIdx.x;
    walk_begin(ws, step_ctr, tid);
    for (;;) {
        __syncthreads();
        if (tid == 0) walk_next(ws, bp);
        __syncthreads();
        if (ws.w < 0) break;
        const int d = ws.d;
        if (ws.fresh) {      // the same value for every thread (set before the barrier)
            if (tid == 0) {
                sq = bp.steps[bp.step_off[d] + ws.step];
                for (int g = 0; g < 3; ++g) tma::tensormap_acquire(&bp.sm[d].v[g]);
                tma::tensormap_acquire(&bp.sm[d].idx);
            }
            __syncthreads();
        }
        const int li = ws.w - bp.block0[d], tx_ = bp.tiles_x[d], txy = tx_ * bp.tiles_y[d];
        if (stress_tile<L, T, true>(bp.p[d], bp.sm[d], sq, bp.kchunk[d], li % tx_,
                                    (li % txy) / tx_, li / txy, smb))
            break;
    }
}

__global__ void k_step_advance(int *ctr) { *ctr += 1; }

}  // namespace

template <int TH = TY>
static dim3 grid_tma(const AcParams &p, int kc)
{
    return dim3((p.nx + TX - 1) / TX, (p.ny + TH - 1) / TH, (p.nz + kc - 1) / kc);
}

// The dynamic shared-memory limit of a kernel, raised once per process to the
// largest size any launch asks for (the material table at its maximum), so
// that launches make no other runtime call (they may be captured in a graph).
template <typename K>
static cudaError_t raise_smem_once(K kernel, size_t bytes, std::atomic<int> &done)
{
    if (done.load(std::memory_order_acquire)) return cudaSuccess;
    const cudaError_t e =
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done.store(1, std::memory_order_release);
    return e;
}

static int chunk_of(const AcParams &p, int th)
{
    return p.kchunk > 0 ? p.kchunk : default_kchunk_tma(p.nx, p.ny, p.nz, th);
}

template <typename T, int TH>
static cudaError_t launch_velocity_tma_t(const AcParams &p, const VelocityTmaMaps &tm,
                                         cudaStream_t s)
{
    const int kc = chunk_of(p, TH);
    const size_t sm = VelLayout<T, TH>::bytes(p.n_mat);
    static std::atomic<int> done{0};
    cudaError_t e = raise_smem_once(k_velocity_tma<T, TH>,
                                    VelLayout<T, TH>::bytes(BVF_MAX_MATERIALS), done);
    if (e != cudaSuccess) return e;
    k_velocity_tma<T, TH><<<grid_tma<TH>(p, kc), dim3(PX, TH, 1), sm, s>>>(p, kc, tm);
    return cudaGetLastError();
}

// tile heights other than TY are built for L = 2 (the method's two
// mechanisms); other L take TY
template <typename T>
static cudaError_t launch_velocity_tma_h(const AcParams &p, const VelocityTmaMaps &tm,
                                         cudaStream_t s)
{
    if (p.L == 2 && p.tile_yv == 4) return launch_velocity_tma_t<T, 4>(p, tm, s);
    if (p.L == 2 && p.tile_yv == 16) return launch_velocity_tma_t<T, 16>(p, tm, s);
    return launch_velocity_tma_t<T, TY>(p, tm, s);
}

cudaError_t launch_velocity_tma(const AcParams &p, const VelocityTmaMaps &tm, cudaStream_t s)
{
    return p.h16 ? launch_velocity_tma_h<__half>(p, tm, s) : launch_velocity_tma_h<float>(p, tm, s);
}

// Resident blocks per SM at height TH: the thread count times blocks per SM
// of the default height (four blocks of 256 threads for the scalar tile, five
// of 128 for the paired FP16 tile) is kept, so are the registers per thread.
template <int L, typename T, int TH>
static cudaError_t launch_stress_tma_t(const AcParams &p, const StressTmaMaps &tm, cudaStream_t s)
{
    const int kc = chunk_of(p, TH);
    const size_t sm = StressLayout<L, T, TH>::bytes(p.n_mat);
    static std::atomic<int> done{0};
    if constexpr (std::is_same<T, __half>::value && L > 0) {
        // FP16 storage: the paired tile (see stress_tile_h2)
        constexpr int MB = kStressH2Blocks * TY / TH > 0 ? kStressH2Blocks * TY / TH : 1;
        cudaError_t e = raise_smem_once(k_stress_tma_h2<L, MB, TH>,
                                        StressLayout<L, T, TH>::bytes(BVF_MAX_MATERIALS), done);
        if (e != cudaSuccess) return e;
        k_stress_tma_h2<L, MB, TH><<<grid_tma<TH>(p, kc), dim3(PX, TH, 1), sm, s>>>(p, kc, tm);
    } else {
        constexpr int MB = 4 * TY / TH;
        cudaError_t e = raise_smem_once(k_stress_tma<L, MB, T, TH>,
                                        StressLayout<L, T, TH>::bytes(BVF_MAX_MATERIALS), done);
        if (e != cudaSuccess) return e;
        k_stress_tma<L, MB, T, TH><<<grid_tma<TH>(p, kc), dim3(TX, TH, 1), sm, s>>>(p, kc, tm);
    }
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_stress_tma_l(const AcParams &p, const StressTmaMaps &tm, cudaStream_t s)
{
    switch (p.L) {
    case 0: return launch_stress_tma_t<0, T, TY>(p, tm, s);
    case 1: return launch_stress_tma_t<1, T, TY>(p, tm, s);
    case 2:
        if (p.tile_y == 4) return launch_stress_tma_t<2, T, 4>(p, tm, s);
        if (p.tile_y == 16) return launch_stress_tma_t<2, T, 16>(p, tm, s);
        return launch_stress_tma_t<2, T, TY>(p, tm, s);
    default: return cudaErrorInvalidValue;
    }
}

// Four resident blocks of 256 threads per SM (64 registers, about 46 KB of
// shared memory each in FP32 storage).
cudaError_t launch_stress_tma(const AcParams &p, const StressTmaMaps &tm, cudaStream_t s)
{
    return p.h16 ? launch_stress_tma_l<__half>(p, tm, s) : launch_stress_tma_l<float>(p, tm, s);
}

template <int L, typename T>
static cudaError_t batch_prepare_t(int n_mat_max, int *gv, int *gs)
{
    const size_t smv = VelLayout<T>::bytes(n_mat_max), sms = StressLayout<L, T>::bytes(n_mat_max);
    cudaError_t e = cudaFuncSetAttribute(k_velocity_batch<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smv);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_stress_batch<L, 4, T>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sms);
    int dev = 0, sm_count = 0, bv = 0, bs = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bv, k_velocity_batch<T>, NTH, smv);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs, k_stress_batch<L, 4, T>, SNTH, sms);
    if (e != cudaSuccess) return e;
    *gv = sm_count * (bv > 0 ? bv : 1);
    *gs = sm_count * (bs > 0 ? bs : 1);
    return cudaSuccess;
}

template <int L, typename T>
static cudaError_t launch_batch_t(const BatchParams &bp, int n_mat_max, int *d_step, int gv, int gs,
                                  cudaStream_t s)
{
    const size_t smv = VelLayout<T>::bytes(n_mat_max), sms = StressLayout<L, T>::bytes(n_mat_max);
    k_velocity_batch<T><<<gv, dim3(PX, TY, 1), smv, s>>>(bp, d_step);
    k_stress_batch<L, 4, T><<<gs, dim3(TX, TY, 1), sms, s>>>(bp, d_step);
    k_step_advance<<<1, 1, 0, s>>>(d_step);
    return cudaGetLastError();
}

cudaError_t batch_prepare(int L, int h16, int n_mat_max, int *gv, int *gs)
{
    switch (L * 2 + (h16 ? 1 : 0)) {
    case 0: return batch_prepare_t<0, float>(n_mat_max, gv, gs);
    case 1: return batch_prepare_t<0, __half>(n_mat_max, gv, gs);
    case 2: return batch_prepare_t<1, float>(n_mat_max, gv, gs);
    case 3: return batch_prepare_t<1, __half>(n_mat_max, gv, gs);
    case 4: return batch_prepare_t<2, float>(n_mat_max, gv, gs);
    case 5: return batch_prepare_t<2, __half>(n_mat_max, gv, gs);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch_step(const BatchParams &bp, int L, int h16, int n_mat_max, int *d_step,
                              int gv, int gs, cudaStream_t s)
{
    switch (L * 2 + (h16 ? 1 : 0)) {
    case 0: return launch_batch_t<0, float>(bp, n_mat_max, d_step, gv, gs, s);
    case 1: return launch_batch_t<0, __half>(bp, n_mat_max, d_step, gv, gs, s);
    case 2: return launch_batch_t<1, float>(bp, n_mat_max, d_step, gv, gs, s);
    case 3: return launch_batch_t<1, __half>(bp, n_mat_max, d_step, gv, gs, s);
    case 4: return launch_batch_t<2, float>(bp, n_mat_max, d_step, gv, gs, s);
    case 5: return launch_batch_t<2, __half>(bp, n_mat_max, d_step, gv, gs, s);
    default: return cudaErrorInvalidValue;
    }
}

// z-chunk length of the TMA kernels: about six waves of four resident blocks
// per SM on 152 SMs (13 planes on the 240 x 240 x 200 grid; 8 to 16 measure
// within 3 % of each other there, 25 is 13 % slower).
int default_kchunk_tma(int nx, int ny, int nz, int tile_y)
{
    const int th = tile_y > 0 ? tile_y : TY;
    const long long tiles = (long long)((nx + TX - 1) / TX) * ((ny + th - 1) / th);
    const long long target = 152LL * 4 * 6;
    long long chunks = (target + tiles - 1) / tiles;
    if (chunks < 1) chunks = 1;
    int kc = (int)((nz + chunks - 1) / chunks);
    if (kc < 8) kc = 8;
    return kc > nz ? nz : kc;
}

}  // namespace bvf
