// TMA-fed acoustic kernels (arXiv 2301.12727, Sec. 2.3, Eq. 1; Sec. 3.2, Eq. 3).
//
// Same arithmetic as the direct kernels in bvf_acoustic.cu, but every array
// moves between HBM and shared memory through the tensor-memory accelerator:
//   * a block of 32 x 8 threads owns one x-y tile and walks a chunk of z;
//   * stencil inputs arrive as 40 x 12 boxes (the tile plus a 4-column /
//     2-row halo; out-of-range elements zero-filled by the TMA, which gives
//     the zero ghosts) held in per-array rings of z-planes that serve the
//     4-point z-stencils as well;
//   * the 1-byte material index arrives as 48 x 9 boxes (planes k and k+1);
//   * velocity kernel: each stress array arrives in a box with exactly the
//     halo its stencil needs; the velocities go straight to registers and
//     back; copies for plane k+1 are issued while plane k is computed;
//   * stress kernel: the velocity and index rings run two planes ahead; the
//     per-voxel arrays (stresses, memory variables, peak map, FP64 DFT sums)
//     go straight to registers with loads issued at the top of each plane and
//     back with coalesced stores, which keeps shared memory small enough for
//     four resident blocks per SM;
//   * one thread issues every copy; one __syncthreads and one bounded mbarrier
//     wait per plane.
// Used when rows are whole multiples of 16 bytes of the index (nx % 16 == 0)
// and L <= 2.
#include "bvf_stencil.cuh"
#include "bvf_tma.cuh"

namespace bvf {

namespace {

using st::dbw;
using st::dfw;
using st::slab_pos;

constexpr int TX = 32, TY = 8, NTH = TX * TY;
constexpr int VW = 40, VH = 12, VT = VW * VH;       // halo'd box: x0-4 .. x0+35, y0-2 .. y0+9
constexpr unsigned VT_BYTES = VT * 4;               // 1920 = 15 * 128
constexpr int IW = 48, IH = 9, IT = IW * IH;        // index box: x0 .. x0+47, y0 .. y0+8
constexpr int IT_SLOT = 512;                        // bytes per index slot

// ---------------------------------------------------------------- velocity
// Each stress array arrives in a box holding exactly the halo its stencil
// reads: sxx 40 x 8 (x-halo), syy 32 x 12 (y-halo), sxy 40 x 12, sxz 40 x 8,
// syz 32 x 12, szz 32 x 8 (z only).  The velocities go straight to registers
// and back.  Loads for plane k+1 are issued while plane k is computed.
//
// The plane loop is unrolled by the ring period R = 6 (every ring depth
// divides it), so each unrolled copy reads fixed ring slots: every shared
// memory access is one of five per-thread centres plus a constant.
constexpr int XW = 40, XH = 8, YW = 32, YH = 12;             // x-halo / y-halo boxes
constexpr int TXX = XW * XH, TYY = YW * YH, TXY = VW * VH, TZZ = TX * TY;
struct VelLayout {
    static constexpr int R = 6;                               // ring period = unroll
    static constexpr int RA = 2, RB = 6, RC = 6, RI = 3;      // ring depths (divide R)
    static constexpr int SA = TXX + TYY + TXY;                // floats per A slot (sxx, syy, sxy)
    static constexpr int SB = TXX + TYY;                      // B slot (sxz, syz)
    static constexpr int off_a = 0;                           // plane k, k+1
    static constexpr int off_b = off_a + RA * SA * 4;         // k-2 .. k+2 (+1 spare)
    static constexpr int off_c = off_b + RB * SB * 4;         // szz: k-1 .. k+3 (+1 spare)
    static constexpr int off_i = off_c + RC * TZZ * 4;        // index: k .. k+2
    static constexpr int off_bar = off_i + RI * IT_SLOT;
    static constexpr int off_lut = off_bar + 16;
    static size_t bytes(int n_mat) { return off_lut + (size_t)n_mat * sizeof(float); }
};
static_assert(VelLayout::R % VelLayout::RA == 0 && VelLayout::R % VelLayout::RB == 0 &&
                  VelLayout::R % VelLayout::RC == 0 && VelLayout::R % VelLayout::RI == 0,
              "ring depths must divide the unroll period");
static_assert(VelLayout::off_b % 128 == 0 && VelLayout::off_c % 128 == 0 &&
                  VelLayout::off_i % 128 == 0 && (VelLayout::SA * 4) % 128 == 0 &&
                  (VelLayout::SB * 4) % 128 == 0 && (TXX * 4) % 128 == 0 &&
                  (TYY * 4) % 128 == 0,
              "TMA destinations must stay 128-byte aligned");

__global__ void __launch_bounds__(NTH, 5)
    k_velocity_tma(const __grid_constant__ AcParams p, int kchunk,
                   const __grid_constant__ VelocityTmaMaps tm)
{
    using Lay = VelLayout;
    extern __shared__ __align__(1024) float smf[];
    unsigned char *smb = reinterpret_cast<unsigned char *>(smf);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smb + Lay::off_bar);
    float *s_rho = smf + Lay::off_lut / 4;

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int i = x0 + tx, j = y0 + ty;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const bool live = i < nx && j < ny;
    const int k0 = blockIdx.z * kchunk, k1 = min(nz, k0 + kchunk);
    for (int m = tid; m < p.n_mat; m += NTH) s_rho[m] = p.lut[m].rho;
    if (tid == 0) {
        tma::mbar_init(&bars[0], 1);
        tma::mbar_init(&bars[1], 1);
        tma::mbar_init_fence();
    }
    __syncthreads();

    // ring slots: A holds plane pl in slot (pl-k0)%2, B in (pl-k0+2)%6,
    // C in (pl-k0+1)%6, the index in (pl-k0)%3
    constexpr unsigned A_BYTES = Lay::SA * 4, B_BYTES = Lay::SB * 4, C_BYTES = TZZ * 4;
    auto ldA = [&](int pl, int slot, uint64_t *bar) {
        float *d = smf + Lay::off_a / 4 + slot * Lay::SA;
        tma::load3d(d, &tm.sg[0], x0 - 4, y0, pl, bar);                    // sxx
        tma::load3d(d + TXX, &tm.sg[1], x0, y0 - 2, pl, bar);              // syy
        tma::load3d(d + TXX + TYY, &tm.sg[3], x0 - 4, y0 - 2, pl, bar);    // sxy
    };
    auto ldB = [&](int pl, int slot, uint64_t *bar) {
        float *d = smf + Lay::off_b / 4 + slot * Lay::SB;
        tma::load3d(d, &tm.sg[4], x0 - 4, y0, pl, bar);                    // sxz
        tma::load3d(d + TXX, &tm.sg[5], x0, y0 - 2, pl, bar);              // syz
    };
    auto ldC = [&](int pl, int slot, uint64_t *bar) {
        tma::load3d(smf + Lay::off_c / 4 + slot * TZZ, &tm.sg[2], x0, y0, pl, bar);
    };
    auto ldI = [&](int pl, int slot, uint64_t *bar) {
        tma::load3d(smb + Lay::off_i + slot * IT_SLOT, &tm.idx, x0, y0, pl, bar);
    };

    if (tid == 0) {
        tma::mbar_expect_tx(&bars[0], A_BYTES + 4 * B_BYTES + 4 * C_BYTES + 2 * IT);
        ldA(k0, 0, &bars[0]);
        for (int d = 0; d < 4; ++d) ldB(k0 - 2 + d, d, &bars[0]);
        for (int d = 0; d < 4; ++d) ldC(k0 - 1 + d, d, &bars[0]);
        ldI(k0, 0, &bars[0]);
        ldI(k0 + 1, 1, &bars[0]);
    }

    const st::Dx ix = st::make_dx(p.inv_dx);
    const float dt = p.dt;
    // per-thread centres inside a slot: x-halo box, y-halo box, full-halo box,
    // plain box, index box
    const int cx = ty * XW + tx + 4;
    const int cy = (ty + 2) * YW + tx;
    const int cxy = (ty + 2) * VW + tx + 4;
    const int cI = ty * IW + tx;
    const int xs = slab_pos(i, nx, p.P), ys = slab_pos(j, ny, p.P);
    const int Sxs = nz * ny * p.W, Sys = nz * p.W * nx, Szs = p.W * ny * nx;
    const float2 *pmlx = p.pml, *pmly = p.pml + 2 * p.nmax, *pmlz = p.pml + 4 * p.nmax;
    float *__restrict__ vxg = p.vx;
    float *__restrict__ vyg = p.vy;
    float *__restrict__ vzg = p.vz;
    const bool ix1 = i < nx - 1, jy1 = j < ny - 1;
    const int plane = nx * ny, col = j * nx + i;
    // velocities of the plane being computed, loaded one plane ahead
    float ux = 0.0f, uy = 0.0f, uz = 0.0f;
    if (live) {
        ux = vxg[k0 * plane + col];
        uy = vyg[k0 * plane + col];
        uz = vzg[k0 * plane + col];
    }
    int q = k0 * plane + col;                       // this voxel in plane k
    int ox = (k0 * ny + j) * p.W + xs;              // in the x-slab (xs >= 0)
    int oy = (k0 * p.W + ys) * nx + i;              // in the y-slab (ys >= 0)
    const int dox = ny * p.W, doy = p.W * nx;

    unsigned mpar = 0;                              // parity of (k - k0) / R
    for (int kb = k0; kb < k1; kb += Lay::R, mpar ^= 1u) {
#pragma unroll
        for (int u = 0; u < Lay::R; ++u) {
            const int k = kb + u;
            if (k >= k1) break;
            __syncthreads();
            if (tid == 0 && k + 1 < k1) {
                tma::fence_async_smem();
                uint64_t *bar = &bars[(u + 1) & 1];
                tma::mbar_expect_tx(bar, A_BYTES + B_BYTES + C_BYTES + IT);
                ldA(k + 1, (u + 1) % Lay::RA, bar);
                ldB(k + 2, (u + 4) % Lay::RB, bar);
                ldC(k + 3, (u + 4) % Lay::RC, bar);
                ldI(k + 2, (u + 2) % Lay::RI, bar);
            }
            float nux = 0.0f, nuy = 0.0f, nuz = 0.0f;
            if (live && k + 1 < k1) {
                nux = vxg[q + plane];
                nuy = vyg[q + plane];
                nuz = vzg[q + plane];
            }
            // CPML memories of this voxel (components 0-2 of each slab it lies
            // in), all loads issued together before the ring wait
            const int zs = slab_pos(k, nz, p.P);
            const int oz = zs * plane + col;
            float qx[3] = {0.0f, 0.0f, 0.0f}, qy[3] = {0.0f, 0.0f, 0.0f},
                  qz[3] = {0.0f, 0.0f, 0.0f};
            if (live) {
                if (xs >= 0) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) qx[c] = p.psx[c * Sxs + ox];
                }
                if (ys >= 0) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) qy[c] = p.psy[c * Sys + oy];
                }
                if (zs >= 0) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) qz[c] = p.psz[c * Szs + oz];
                }
            }
            const bool ready = tma::mbar_wait(&bars[u & 1], mpar ^ ((u >> 1) & 1u), p.flag);
            if (ready && live) {
                // fixed slots of this unrolled copy
                const float *A = smf + Lay::off_a / 4 + (u % Lay::RA) * Lay::SA;
                const float *XX = A + cx, *YY = A + TXX + cy, *XY = A + TXX + TYY + cxy;
                const float *Bm2 = smf + Lay::off_b / 4 + ((u + 0) % Lay::RB) * Lay::SB;
                const float *Bm1 = smf + Lay::off_b / 4 + ((u + 1) % Lay::RB) * Lay::SB;
                const float *B0 = smf + Lay::off_b / 4 + ((u + 2) % Lay::RB) * Lay::SB;
                const float *Bp1 = smf + Lay::off_b / 4 + ((u + 3) % Lay::RB) * Lay::SB;
                const float *Cm1 = smf + Lay::off_c / 4 + ((u + 0) % Lay::RC) * TZZ + tid;
                const float *C0 = smf + Lay::off_c / 4 + ((u + 1) % Lay::RC) * TZZ + tid;
                const float *Cp1 = smf + Lay::off_c / 4 + ((u + 2) % Lay::RC) * TZZ + tid;
                const float *Cp2 = smf + Lay::off_c / 4 + ((u + 3) % Lay::RC) * TZZ + tid;
                const unsigned char *I0 = smb + Lay::off_i + (u % Lay::RI) * IT_SLOT + cI;
                const unsigned char *I1 = smb + Lay::off_i + ((u + 1) % Lay::RI) * IT_SLOT + cI;
                const float *XZ = B0 + cx, *YZ = B0 + TXX + cy;
                const bool kz1 = k < nz - 1;

                // all three components are computed; ghost points (the last
                // half point of each axis) are simply not stored
                float ax1 = dfw(XX[-1], XX[0], XX[1], XX[2], ix);
                float ax2 = dbw(XY[-2 * VW], XY[-VW], XY[0], XY[VW], ix);
                float ax3 = dbw(Bm2[cx], Bm1[cx], XZ[0], Bp1[cx], ix);
                float ay1 = dbw(XY[-2], XY[-1], XY[0], XY[1], ix);
                float ay2 = dfw(YY[-YW], YY[0], YY[YW], YY[2 * YW], ix);
                float ay3 = dbw(Bm2[TXX + cy], Bm1[TXX + cy], YZ[0], Bp1[TXX + cy], ix);
                float az1 = dbw(XZ[-2], XZ[-1], XZ[0], XZ[1], ix);
                float az2 = dbw(YZ[-2 * YW], YZ[-YW], YZ[0], YZ[YW], ix);
                float az3 = dfw(*Cm1, *C0, *Cp1, *Cp2, ix);
                if (xs >= 0) {
                    const float2 h = __ldg(&pmlx[p.nmax + i]), w = __ldg(&pmlx[i]);
                    float t = fmaf(h.x, ax1, h.y * qx[0]);
                    if (ix1) p.psx[ox] = t;
                    ax1 += t;
                    t = fmaf(w.x, ay1, w.y * qx[1]);
                    if (jy1) p.psx[Sxs + ox] = t;
                    ay1 += t;
                    t = fmaf(w.x, az1, w.y * qx[2]);
                    if (kz1) p.psx[2 * Sxs + ox] = t;
                    az1 += t;
                }
                if (ys >= 0) {
                    const float2 h = __ldg(&pmly[p.nmax + j]), w = __ldg(&pmly[j]);
                    float t = fmaf(w.x, ax2, w.y * qy[0]);
                    if (ix1) p.psy[oy] = t;
                    ax2 += t;
                    t = fmaf(h.x, ay2, h.y * qy[1]);
                    if (jy1) p.psy[Sys + oy] = t;
                    ay2 += t;
                    t = fmaf(w.x, az2, w.y * qy[2]);
                    if (kz1) p.psy[2 * Sys + oy] = t;
                    az2 += t;
                }
                if (zs >= 0) {
                    const float2 h = __ldg(&pmlz[p.nmax + k]), w = __ldg(&pmlz[k]);
                    float t = fmaf(w.x, ax3, w.y * qz[0]);
                    if (ix1) p.psz[oz] = t;
                    ax3 += t;
                    t = fmaf(w.x, ay3, w.y * qz[1]);
                    if (jy1) p.psz[Szs + oz] = t;
                    ay3 += t;
                    t = fmaf(h.x, az3, h.y * qz[2]);
                    if (kz1) p.psz[2 * Szs + oz] = t;
                    az3 += t;
                }
                const float rho0 = s_rho[I0[0]];
                const float nvx = ux + st::vel_increment(dt, rho0, s_rho[I0[1]], ax1, ax2, ax3);
                const float nvy = uy + st::vel_increment(dt, rho0, s_rho[I0[IW]], ay1, ay2, ay3);
                const float nvz = uz + st::vel_increment(dt, rho0, s_rho[I1[0]], az1, az2, az3);
                if (ix1) vxg[q] = nvx;
                if (jy1) vyg[q] = nvy;
                if (kz1) vzg[q] = nvz;
            }
            ux = nux;
            uy = nuy;
            uz = nuz;
            q += plane;
            ox += dox;
            oy += doy;
        }
    }
}

// ------------------------------------------------------------------ stress
// The stencil inputs (velocity tiles with halos, material index) come through
// TMA rings two planes ahead; the per-voxel arrays (stresses, memory
// variables, peak map, FP64 DFT sums) are read straight into registers at the
// top of each plane, so their latency overlaps the ring wait and the
// derivatives, and written back with coalesced stores.
template <int L>
struct StressLayout {
    static constexpr int RV = 7, RI = 4;                      // ring depths
    static constexpr int off_v = 0;                           // vx, vy, vz: k-2 .. k+4
    static constexpr int off_i = off_v + RV * 3 * VT * 4;     // index: k .. k+3
    static constexpr int off_bar = off_i + RI * IT_SLOT;
    static constexpr int off_lut = off_bar + 32;
    static size_t bytes(int n_mat) { return off_lut + (size_t)n_mat * sizeof(st::StressCoef); }
};

template <int L, int MINB>
__global__ void __launch_bounds__(NTH, MINB)
    k_stress_tma(const __grid_constant__ AcParams p, int kchunk,
                 const __grid_constant__ StressTmaMaps tm)
{
    using Lay = StressLayout<L>;
    extern __shared__ __align__(1024) float smf[];
    unsigned char *smb = reinterpret_cast<unsigned char *>(smf);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smb + Lay::off_bar);
    st::StressCoef *s_lut = reinterpret_cast<st::StressCoef *>(smb + Lay::off_lut);

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int i = x0 + tx, j = y0 + ty;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const bool live = i < nx && j < ny;
    const int k0 = blockIdx.z * kchunk, k1 = min(nz, k0 + kchunk);
    for (int m = tid; m < p.n_mat; m += NTH) s_lut[m] = st::make_stress_coef(p.lut[m], p.Lf);
    if (tid == 0) {
        for (int b = 0; b < 3; ++b) tma::mbar_init(&bars[b], 1);
        tma::mbar_init_fence();
    }
    __syncthreads();

    auto oV = [&](int pl) { return Lay::off_v / 4 + ((pl - k0 + 2) % Lay::RV) * 3 * VT; };
    auto oI = [&](int pl) { return Lay::off_i + ((pl - k0) % Lay::RI) * IT_SLOT; };   // bytes
    auto issue = [&](int kk, uint64_t *bar, bool first) {
        const unsigned nv = first ? 5 : 1;
        tma::mbar_expect_tx(bar, nv * 3 * VT_BYTES + (first ? 2 : 1) * IT);
        for (int pl = first ? kk - 2 : kk + 2; pl <= kk + 2; ++pl)
            for (int a = 0; a < 3; ++a)
                tma::load3d(smf + oV(pl) + a * VT, &tm.v[a], x0 - 4, y0 - 2, pl, bar);
        for (int pl = first ? kk : kk + 1; pl <= kk + 1; ++pl)
            tma::load3d(smb + oI(pl), &tm.idx, x0, y0, pl, bar);
    };
    if (tid == 0) {
        issue(k0, &bars[0], true);
        if (k0 + 1 < k1) issue(k0 + 1, &bars[1], false);
    }

    const st::Dx ix = st::make_dx(p.inv_dx);
    const int cv = (ty + 2) * VW + tx + 4;
    const int ci = ty * IW + tx;
    const int xs = slab_pos(i, nx, p.P), ys = slab_pos(j, ny, p.P);
    const int Sxs = nz * ny * p.W, Sys = nz * p.W * nx, Szs = p.W * ny * nx;
    const float2 *pmlx = p.pml, *pmly = p.pml + 2 * p.nmax, *pmlz = p.pml + 4 * p.nmax;
    float *const gs[6] = {p.sxx, p.syy, p.szz, p.sxy, p.sxz, p.syz};
    float *__restrict__ mem = p.mem;

    // Ring positions of this thread's column, rotated once per plane: the
    // velocity ring at planes k-2 .. k+2 (float offsets of the vx centre) and
    // the index ring at k, k+1 (bytes).
    const int vbase = Lay::off_v / 4, vend = vbase + Lay::RV * 3 * VT;
    const int ibase = Lay::off_i, iend = ibase + Lay::RI * IT_SLOT;
    int vM2 = vbase + cv, vM1 = vM2 + 3 * VT, vK = vM1 + 3 * VT, vP1 = vK + 3 * VT,
        vP2 = vP1 + 3 * VT;
    int iK = ibase + ci, iK1 = iK + IT_SLOT;

    int it = 0;
    for (int k = k0; k < k1; ++k, ++it) {
        __syncthreads();
        if (tid == 0 && k + 2 < k1) {
            tma::fence_async_smem();
            issue(k + 2, &bars[(it + 2) % 3], false);
        }
        const int q = k * (nx * ny) + j * nx + i;
        // per-voxel loads first, in flight while the ring wait and the
        // derivatives proceed
        float sv[6], rv[L > 0 ? L : 1][6];
        float pk = 0.0f;
        double dC = 0.0, dS = 0.0;
        // CPML memories of this voxel (components 3-5 of each slab it lies in)
        const int zs = slab_pos(k, nz, p.P);
        const int ox = (k * ny + j) * p.W + xs, oy = (k * p.W + ys) * nx + i,
                  oz = (zs * ny + j) * nx + i;
        float qx[3] = {0.0f, 0.0f, 0.0f}, qy[3] = {0.0f, 0.0f, 0.0f}, qz[3] = {0.0f, 0.0f, 0.0f};
        if (live) {
            if (xs >= 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) qx[c] = p.psx[(3 + c) * Sxs + ox];
            }
            if (ys >= 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) qy[c] = p.psy[(3 + c) * Sys + oy];
            }
            if (zs >= 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) qz[c] = p.psz[(3 + c) * Szs + oz];
            }
        }
        if (live) {
#pragma unroll
            for (int cc = 0; cc < 6; ++cc) sv[cc] = gs[cc][q];
#pragma unroll
            for (int l = 0; l < L; ++l)
#pragma unroll
                for (int cc = 0; cc < 6; ++cc) rv[l][cc] = mem[(size_t)(l * 6 + cc) * p.fstride + q];
            if (p.do_peak) pk = p.peak[q];
            if (p.do_dft) {
                dC = p.dftC[q];
                dS = p.dftS[q];
            }
        }
        const bool ready = tma::mbar_wait(&bars[it % 3], (it / 3) & 1, p.flag);
        if (ready && live) {
            const int vm2 = vM2, vm1 = vM1, vp1 = vP1, vp2 = vP2;
            const unsigned char *I0 = smb + iK;
            const unsigned char *I1 = smb + iK1;
            const bool ix1 = i < nx - 1, jy1 = j < ny - 1, kz1 = k < nz - 1;
            const int m00 = I0[0];
            const st::StressCoef c0 = s_lut[m00];
            const int vx = vK, vy = vK + VT, vz = vK + 2 * VT;

            // ---- normal stresses at (i, j, k)
            float exx = dbw(smf[vx - 2], smf[vx - 1], smf[vx], smf[vx + 1], ix);
            float eyy = dbw(smf[vy - 2 * VW], smf[vy - VW], smf[vy], smf[vy + VW], ix);
            float ezz = dbw(smf[vm2 + 2 * VT], smf[vm1 + 2 * VT], smf[vz], smf[vp1 + 2 * VT], ix);
            if (xs >= 0) exx = st::cpml_pre(p.psx + 3 * Sxs + ox, qx[0], __ldg(&pmlx[i]), exx);
            if (ys >= 0) eyy = st::cpml_pre(p.psy + 3 * Sys + oy, qy[0], __ldg(&pmly[j]), eyy);
            if (zs >= 0) ezz = st::cpml_pre(p.psz + 3 * Szs + oz, qz[0], __ldg(&pmlz[k]), ezz);
            float srcv = 0.0f;
            if (p.src_on && k == p.k_src) {
                const float2 a = p.src[j * nx + i];
                srcv = p.src_scale * fmaf(a.x, p.src_ws, a.y * p.src_wc);
            }
            st::normal_update<L>(p, c0, exx, eyy, ezz, srcv, sv, rv);
            const float pr = st::pressure(sv);
            if (!isfinite(pr)) atomicOr(p.flag, 1);

            // ---- shear stresses
            const bool dxy = ix1 && jy1, dxz = ix1 && kz1, dyz = jy1 && kz1;
            if (dxy) {                               // sxy at (i+1/2, j+1/2, k)
                float a = dfw(smf[vx - VW], smf[vx], smf[vx + VW], smf[vx + 2 * VW], ix);
                float b = dfw(smf[vy - 1], smf[vy], smf[vy + 1], smf[vy + 2], ix);
                if (ys >= 0) a = st::cpml_pre(p.psy + 4 * Sys + oy, qy[1], __ldg(&pmly[p.nmax + j]), a);
                if (xs >= 0) b = st::cpml_pre(p.psx + 4 * Sxs + ox, qx[1], __ldg(&pmlx[p.nmax + i]), b);
                st::shear_update<L>(p, s_lut, c0, m00, I0[1], I0[IW], I0[IW + 1], a + b, 3, sv, rv);
            }
            if (dxz) {                               // sxz at (i+1/2, j, k+1/2)
                float a = dfw(smf[vm1], smf[vx], smf[vp1], smf[vp2], ix);
                float b = dfw(smf[vz - 1], smf[vz], smf[vz + 1], smf[vz + 2], ix);
                if (zs >= 0) a = st::cpml_pre(p.psz + 4 * Szs + oz, qz[1], __ldg(&pmlz[p.nmax + k]), a);
                if (xs >= 0) b = st::cpml_pre(p.psx + 5 * Sxs + ox, qx[2], __ldg(&pmlx[p.nmax + i]), b);
                st::shear_update<L>(p, s_lut, c0, m00, I0[1], I1[0], I1[1], a + b, 4, sv, rv);
            }
            if (dyz) {                               // syz at (i, j+1/2, k+1/2)
                float a = dfw(smf[vm1 + VT], smf[vy], smf[vp1 + VT], smf[vp2 + VT], ix);
                float b = dfw(smf[vz - VW], smf[vz], smf[vz + VW], smf[vz + 2 * VW], ix);
                if (zs >= 0) a = st::cpml_pre(p.psz + 5 * Szs + oz, qz[2], __ldg(&pmlz[p.nmax + k]), a);
                if (ys >= 0) b = st::cpml_pre(p.psy + 5 * Sys + oy, qy[2], __ldg(&pmly[p.nmax + j]), b);
                st::shear_update<L>(p, s_lut, c0, m00, I0[IW], I1[0], I1[IW], a + b, 5, sv, rv);
            }

            // ---- results (ghost points are not written)
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) gs[cc][q] = sv[cc];
            if (dxy) gs[3][q] = sv[3];
            if (dxz) gs[4][q] = sv[4];
            if (dyz) gs[5][q] = sv[5];
#pragma unroll
            for (int l = 0; l < L; ++l)
#pragma unroll
                for (int cc = 0; cc < 6; ++cc) {
                    const bool w = cc < 3 || (cc == 3 && dxy) || (cc == 4 && dxz) || (cc == 5 && dyz);
                    if (w) mem[(size_t)(l * 6 + cc) * p.fstride + q] = rv[l][cc];
                }
            if (p.do_peak) p.peak[q] = fmaxf(pk, fabsf(pr));
            if (p.do_dft) {
                p.dftC[q] = fma((double)pr, p.cw, dC);
                p.dftS[q] = fma((double)pr, p.sw, dS);
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
}

}  // namespace

static dim3 grid_tma(const AcParams &p, int kc)
{
    return dim3((p.nx + TX - 1) / TX, (p.ny + TY - 1) / TY, (p.nz + kc - 1) / kc);
}

cudaError_t launch_velocity_tma(const AcParams &p, const VelocityTmaMaps &tm, cudaStream_t s)
{
    const int kc = p.kchunk > 0 ? p.kchunk : default_kchunk_tma(p.nx, p.ny, p.nz);
    const size_t sm = VelLayout::bytes(p.n_mat);
    cudaError_t e = cudaFuncSetAttribute(k_velocity_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    k_velocity_tma<<<grid_tma(p, kc), dim3(TX, TY, 1), sm, s>>>(p, kc, tm);
    return cudaGetLastError();
}

template <int L, int MINB>
static cudaError_t launch_stress_tma_t(const AcParams &p, const StressTmaMaps &tm, cudaStream_t s)
{
    const int kc = p.kchunk > 0 ? p.kchunk : default_kchunk_tma(p.nx, p.ny, p.nz);
    const size_t sm = StressLayout<L>::bytes(p.n_mat);
    cudaError_t e = cudaFuncSetAttribute(k_stress_tma<L, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_stress_tma<L, MINB><<<grid_tma(p, kc), dim3(TX, TY, 1), sm, s>>>(p, kc, tm);
    return cudaGetLastError();
}

// Four resident blocks per SM (64 registers, about 46 KB of shared memory).
cudaError_t launch_stress_tma(const AcParams &p, const StressTmaMaps &tm, cudaStream_t s)
{
    switch (p.L) {
    case 0: return launch_stress_tma_t<0, 4>(p, tm, s);
    case 1: return launch_stress_tma_t<1, 4>(p, tm, s);
    case 2: return launch_stress_tma_t<2, 4>(p, tm, s);
    default: return cudaErrorInvalidValue;
    }
}

// z-chunk length of the TMA kernels: about six waves of four resident blocks
// per SM on 152 SMs (13 planes on the 240 x 240 x 200 grid; 8 to 16 measure
// within 3 % of each other there, 25 is 13 % slower).
int default_kchunk_tma(int nx, int ny, int nz)
{
    const long long tiles = (long long)((nx + TX - 1) / TX) * ((ny + TY - 1) / TY);
    const long long target = 152LL * 4 * 6;
    long long chunks = (target + tiles - 1) / tiles;
    if (chunks < 1) chunks = 1;
    int kc = (int)((nz + chunks - 1) / chunks);
    if (kc < 8) kc = 8;
    return kc > nz ? nz : kc;
}

}  // namespace bvf
