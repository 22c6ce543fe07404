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
//   * velocity kernel: the velocities are staged per plane, updated in place
//     and written back with TMA stores; copies for plane k+1 are issued while
//     plane k is computed (four resident blocks per SM);
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
using st::cpml;
using st::slab_pos;

constexpr int TX = 32, TY = 8, NTH = TX * TY;
constexpr int VW = 40, VH = 12, VT = VW * VH;       // halo'd box: x0-4 .. x0+35, y0-2 .. y0+9
constexpr unsigned VT_BYTES = VT * 4;               // 1920 = 15 * 128
constexpr int IW = 48, IH = 9, IT = IW * IH;        // index box: x0 .. x0+47, y0 .. y0+8
constexpr int IT_SLOT = 512;                        // bytes per index slot

// ---------------------------------------------------------------- velocity
// Shared-memory layout (bytes) for loads issued D planes ahead; every TMA
// destination is 128-byte aligned.
template <int D>
struct VelLayout {
    static constexpr int NS = 2 + D;                          // stages (vx, vy, vz)
    static constexpr int RA = 1 + D, RB = 4 + D, RC = 4 + D, RI = 2 + D;   // ring depths
    static constexpr int STAGE_F = 3 * NTH;                   // floats per stage
    static constexpr int off_s = 0;
    static constexpr int off_a = off_s + NS * STAGE_F * 4;    // sxx, syy, sxy: k .. k+D
    static constexpr int off_b = off_a + RA * 3 * VT * 4;     // sxz, syz: k-2 .. k+1+D
    static constexpr int off_c = off_b + RB * 2 * VT * 4;     // szz: k-1 .. k+2+D
    static constexpr int off_i = off_c + RC * VT * 4;         // index: k .. k+1+D
    static constexpr int off_bar = off_i + RI * IT_SLOT;
    static constexpr int off_lut = off_bar + 32;
    static size_t bytes(int n_mat) { return off_lut + (size_t)n_mat * sizeof(float); }
};

template <int D>
__global__ void __launch_bounds__(NTH, D == 1 ? 4 : 3)
    k_velocity_tma(const __grid_constant__ AcParams p, int kchunk,
                   const __grid_constant__ VelocityTmaMaps tm)
{
    using Lay = VelLayout<D>;
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
        for (int b = 0; b <= D; ++b) tma::mbar_init(&bars[b], 1);
        tma::mbar_init_fence();
    }
    __syncthreads();

    // float offsets of ring slots / stages for plane pl
    auto oA = [&](int pl) { return Lay::off_a / 4 + ((pl - k0) % Lay::RA) * 3 * VT; };
    auto oB = [&](int pl) { return Lay::off_b / 4 + ((pl - k0 + 2) % Lay::RB) * 2 * VT; };
    auto oC = [&](int pl) { return Lay::off_c / 4 + ((pl - k0 + 1) % Lay::RC) * VT; };
    auto oI = [&](int pl) { return Lay::off_i + ((pl - k0) % Lay::RI) * IT_SLOT; };   // bytes
    auto oS = [&](int pl) { return Lay::off_s / 4 + ((pl - k0) % Lay::NS) * Lay::STAGE_F; };
    // loads that plane kk needs first (everything for kk = k0)
    auto issue = [&](int kk, uint64_t *bar, bool first) {
        const unsigned nb = first ? 4 : 1;   // new B planes
        const unsigned nc = first ? 4 : 1;   // new C planes
        tma::mbar_expect_tx(bar, (3 + 2 * nb + nc) * VT_BYTES + (first ? 2 : 1) * IT +
                                     Lay::STAGE_F * 4);
        tma::load3d(smf + oA(kk), &tm.sg[0], x0 - 4, y0 - 2, kk, bar);            // sxx
        tma::load3d(smf + oA(kk) + VT, &tm.sg[1], x0 - 4, y0 - 2, kk, bar);       // syy
        tma::load3d(smf + oA(kk) + 2 * VT, &tm.sg[3], x0 - 4, y0 - 2, kk, bar);   // sxy
        for (int pl = first ? kk - 2 : kk + 1; pl <= kk + 1; ++pl) {
            tma::load3d(smf + oB(pl), &tm.sg[4], x0 - 4, y0 - 2, pl, bar);        // sxz
            tma::load3d(smf + oB(pl) + VT, &tm.sg[5], x0 - 4, y0 - 2, pl, bar);   // syz
        }
        for (int pl = first ? kk - 1 : kk + 2; pl <= kk + 2; ++pl)
            tma::load3d(smf + oC(pl), &tm.sg[2], x0 - 4, y0 - 2, pl, bar);        // szz
        for (int pl = first ? kk : kk + 1; pl <= kk + 1; ++pl)
            tma::load3d(smb + oI(pl), &tm.idx, x0, y0, pl, bar);
        for (int a = 0; a < 3; ++a) tma::load3d(smf + oS(kk) + a * NTH, &tm.v[a], x0, y0, kk, bar);
    };
    auto store_stage = [&](int kk) {
        for (int a = 0; a < 3; ++a) tma::store3d(&tm.v[a], x0, y0, kk, smf + oS(kk) + a * NTH);
        tma::bulk_commit();
    };
    if (tid == 0) {
        issue(k0, &bars[0], true);
        for (int d = 1; d < D; ++d)
            if (k0 + d < k1) issue(k0 + d, &bars[d], false);
    }

    const st::Dx ix = st::make_dx(p.inv_dx);
    const float dt = p.dt;
    const int cv = (ty + 2) * VW + tx + 4;
    const int ci = ty * IW + tx;
    const int xs = slab_pos(i, nx, p.P), ys = slab_pos(j, ny, p.P);
    const int Sxs = nz * ny * p.W, Sys = nz * p.W * nx, Szs = p.W * ny * nx;
    const float2 *pmlx = p.pml, *pmly = p.pml + 2 * p.nmax, *pmlz = p.pml + 4 * p.nmax;

    int it = 0;
    for (int k = k0; k < k1; ++k, ++it) {
        __syncthreads();
        if (tid == 0) {
            if (it > 0) store_stage(k - 1);
            if (k + D < k1) {
                tma::bulk_wait_read<1>();
                tma::fence_async_smem();
                issue(k + D, &bars[(it + D) % (D + 1)], false);
            }
        }
        const bool ready = tma::mbar_wait(&bars[it % (D + 1)], (it / (D + 1)) & 1, p.flag);
        if (ready && live) {
            const int s = oS(k) + tid;
            const int a = oA(k) + cv;                 // sxx at a, syy at a + VT, sxy at a + 2 VT
            const int bk = oB(k) + cv, bm2 = oB(k - 2) + cv, bm1 = oB(k - 1) + cv,
                      bp1 = oB(k + 1) + cv;           // sxz at +0, syz at +VT
            const unsigned char *I0 = smb + oI(k) + ci;
            const unsigned char *I1 = smb + oI(k + 1) + ci;
            const bool ix1 = i < nx - 1, jy1 = j < ny - 1, kz1 = k < nz - 1;
            const int zs = slab_pos(k, nz, p.P);
            const float rho0 = s_rho[I0[0]];
            if (ix1) {
                float d1 = dfw(smf[a - 1], smf[a], smf[a + 1], smf[a + 2], ix);
                const int xy = a + 2 * VT;
                float d2 = dbw(smf[xy - 2 * VW], smf[xy - VW], smf[xy], smf[xy + VW], ix);
                float d3 = dbw(smf[bm2], smf[bm1], smf[bk], smf[bp1], ix);
                if (xs >= 0) d1 = cpml(p.psx + 0 * Sxs + (k * ny + j) * p.W + xs, pmlx[p.nmax + i], d1);
                if (ys >= 0) d2 = cpml(p.psy + 0 * Sys + (k * p.W + ys) * nx + i, pmly[j], d2);
                if (zs >= 0) d3 = cpml(p.psz + 0 * Szs + (zs * ny + j) * nx + i, pmlz[k], d3);
                smf[s] += st::vel_increment(dt, rho0, s_rho[I0[1]], d1, d2, d3);
            }
            if (jy1) {
                const int xy = a + 2 * VT, yy = a + VT;
                float d1 = dbw(smf[xy - 2], smf[xy - 1], smf[xy], smf[xy + 1], ix);
                float d2 = dfw(smf[yy - VW], smf[yy], smf[yy + VW], smf[yy + 2 * VW], ix);
                float d3 = dbw(smf[bm2 + VT], smf[bm1 + VT], smf[bk + VT], smf[bp1 + VT], ix);
                if (xs >= 0) d1 = cpml(p.psx + 1 * Sxs + (k * ny + j) * p.W + xs, pmlx[i], d1);
                if (ys >= 0) d2 = cpml(p.psy + 1 * Sys + (k * p.W + ys) * nx + i, pmly[p.nmax + j], d2);
                if (zs >= 0) d3 = cpml(p.psz + 1 * Szs + (zs * ny + j) * nx + i, pmlz[k], d3);
                smf[s + NTH] += st::vel_increment(dt, rho0, s_rho[I0[IW]], d1, d2, d3);
            }
            if (kz1) {
                const int xz = bk, yz = bk + VT;
                float d1 = dbw(smf[xz - 2], smf[xz - 1], smf[xz], smf[xz + 1], ix);
                float d2 = dbw(smf[yz - 2 * VW], smf[yz - VW], smf[yz], smf[yz + VW], ix);
                float d3 = dfw(smf[oC(k - 1) + cv], smf[oC(k) + cv], smf[oC(k + 1) + cv],
                               smf[oC(k + 2) + cv], ix);
                if (xs >= 0) d1 = cpml(p.psx + 2 * Sxs + (k * ny + j) * p.W + xs, pmlx[i], d1);
                if (ys >= 0) d2 = cpml(p.psy + 2 * Sys + (k * p.W + ys) * nx + i, pmly[j], d2);
                if (zs >= 0) d3 = cpml(p.psz + 2 * Szs + (zs * ny + j) * nx + i, pmlz[p.nmax + k], d3);
                smf[s + 2 * NTH] += st::vel_increment(dt, rho0, s_rho[I1[0]], d1, d2, d3);
            }
        }
        tma::fence_async_smem();
    }
    __syncthreads();
    if (tid == 0 && it > 0) {
        store_stage(k1 - 1);
        tma::bulk_wait<0>();
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
            const int v0 = oV(k) + cv;                       // vx at v0, vy v0 + VT, vz v0 + 2 VT
            const int vm2 = oV(k - 2) + cv, vm1 = oV(k - 1) + cv, vp1 = oV(k + 1) + cv,
                      vp2 = oV(k + 2) + cv;
            const unsigned char *I0 = smb + oI(k) + ci;
            const unsigned char *I1 = smb + oI(k + 1) + ci;
            const bool ix1 = i < nx - 1, jy1 = j < ny - 1, kz1 = k < nz - 1;
            const int zs = slab_pos(k, nz, p.P);
            const int m00 = I0[0];
            const st::StressCoef c0 = s_lut[m00];
            const int vx = v0, vy = v0 + VT, vz = v0 + 2 * VT;

            // ---- normal stresses at (i, j, k)
            float exx = dbw(smf[vx - 2], smf[vx - 1], smf[vx], smf[vx + 1], ix);
            float eyy = dbw(smf[vy - 2 * VW], smf[vy - VW], smf[vy], smf[vy + VW], ix);
            float ezz = dbw(smf[vm2 + 2 * VT], smf[vm1 + 2 * VT], smf[vz], smf[vp1 + 2 * VT], ix);
            if (xs >= 0) exx = cpml(p.psx + 3 * Sxs + (k * ny + j) * p.W + xs, pmlx[i], exx);
            if (ys >= 0) eyy = cpml(p.psy + 3 * Sys + (k * p.W + ys) * nx + i, pmly[j], eyy);
            if (zs >= 0) ezz = cpml(p.psz + 3 * Szs + (zs * ny + j) * nx + i, pmlz[k], ezz);
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
                if (ys >= 0) a = cpml(p.psy + 4 * Sys + (k * p.W + ys) * nx + i, pmly[p.nmax + j], a);
                if (xs >= 0) b = cpml(p.psx + 4 * Sxs + (k * ny + j) * p.W + xs, pmlx[p.nmax + i], b);
                st::shear_update<L>(p, s_lut, c0, m00, I0[1], I0[IW], I0[IW + 1], a + b, 3, sv, rv);
            }
            if (dxz) {                               // sxz at (i+1/2, j, k+1/2)
                float a = dfw(smf[vm1], smf[vx], smf[vp1], smf[vp2], ix);
                float b = dfw(smf[vz - 1], smf[vz], smf[vz + 1], smf[vz + 2], ix);
                if (zs >= 0) a = cpml(p.psz + 4 * Szs + (zs * ny + j) * nx + i, pmlz[p.nmax + k], a);
                if (xs >= 0) b = cpml(p.psx + 5 * Sxs + (k * ny + j) * p.W + xs, pmlx[p.nmax + i], b);
                st::shear_update<L>(p, s_lut, c0, m00, I0[1], I1[0], I1[1], a + b, 4, sv, rv);
            }
            if (dyz) {                               // syz at (i, j+1/2, k+1/2)
                float a = dfw(smf[vm1 + VT], smf[vy], smf[vp1 + VT], smf[vp2 + VT], ix);
                float b = dfw(smf[vz - VW], smf[vz], smf[vz + VW], smf[vz + 2 * VW], ix);
                if (zs >= 0) a = cpml(p.psz + 5 * Szs + (zs * ny + j) * nx + i, pmlz[p.nmax + k], a);
                if (ys >= 0) b = cpml(p.psy + 5 * Sys + (k * p.W + ys) * nx + i, pmly[p.nmax + j], b);
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
    }
}

}  // namespace

static dim3 grid_tma(const AcParams &p, int kc)
{
    return dim3((p.nx + TX - 1) / TX, (p.ny + TY - 1) / TY, (p.nz + kc - 1) / kc);
}

template <int D>
static cudaError_t launch_velocity_tma_t(const AcParams &p, const VelocityTmaMaps &tm, cudaStream_t s)
{
    const int kc = p.kchunk > 0 ? p.kchunk : default_kchunk_tma(p.nx, p.ny, p.nz);
    const size_t sm = VelLayout<D>::bytes(p.n_mat);
    cudaError_t e = cudaFuncSetAttribute(k_velocity_tma<D>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_velocity_tma<D><<<grid_tma(p, kc), dim3(TX, TY, 1), sm, s>>>(p, kc, tm);
    return cudaGetLastError();
}

// One plane of lead (four resident blocks per SM) measures faster than two
// planes of lead at three blocks per SM.
cudaError_t launch_velocity_tma(const AcParams &p, const VelocityTmaMaps &tm, cudaStream_t s)
{
    return launch_velocity_tma_t<1>(p, tm, s);
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
