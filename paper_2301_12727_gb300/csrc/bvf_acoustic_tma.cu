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
//   * the arrays each voxel reads and rewrites (velocities in the velocity
//     kernel; stresses, memory variables, peak map and FP64 DFT sums in the
//     stress kernel) are staged in a ring of three buffers, updated in place
//     and written back with TMA stores;
//   * one thread issues every copy for plane k+1 while plane k is computed;
//     one __syncthreads and one bounded mbarrier wait per plane.
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
constexpr int NSTG = 3;                             // staging buffers

// ---------------------------------------------------------------- velocity
struct VelLayout {
    static constexpr int STAGE_BYTES = 3 * NTH * 4;        // vx, vy, vz
    static constexpr int RA = 2, RB = 5, RC = 5, RI = 3;  // ring depths
    static constexpr size_t off_a = NSTG * STAGE_BYTES;   // sxx, syy, sxy (plane k, k+1)
    static constexpr size_t off_b = off_a + RA * 3 * VT_BYTES;   // sxz, syz (k-2 .. k+2)
    static constexpr size_t off_c = off_b + RB * 2 * VT_BYTES;   // szz (k-1 .. k+3)
    static constexpr size_t off_i = off_c + RC * VT_BYTES;
    static constexpr size_t off_bar = off_i + RI * IT_SLOT;
    static constexpr size_t off_lut = off_bar + 16;
    static size_t bytes(int n_mat) { return off_lut + (size_t)n_mat * sizeof(float); }
};

__global__ void __launch_bounds__(NTH, 4)
    k_velocity_tma(const __grid_constant__ AcParams p, int kchunk,
                   const __grid_constant__ VelocityTmaMaps tm)
{
    using Lay = VelLayout;
    extern __shared__ __align__(1024) unsigned char sm[];
    float *stages = reinterpret_cast<float *>(sm);
    float *ringA = reinterpret_cast<float *>(sm + Lay::off_a);
    float *ringB = reinterpret_cast<float *>(sm + Lay::off_b);
    float *ringC = reinterpret_cast<float *>(sm + Lay::off_c);
    uint8_t *ringI = sm + Lay::off_i;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + Lay::off_bar);
    float *s_rho = reinterpret_cast<float *>(sm + Lay::off_lut);

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

    auto stage = [&](int it) { return stages + (it % NSTG) * (Lay::STAGE_BYTES / 4); };
    auto tA = [&](int pl, int a) { return ringA + (((pl - k0) & 1) * 3 + a) * VT; };
    auto tB = [&](int pl, int a) { return ringB + (((pl - k0 + 2) % Lay::RB) * 2 + a) * VT; };
    auto tC = [&](int pl) { return ringC + ((pl - k0 + 1) % Lay::RC) * VT; };
    auto tI = [&](int pl) { return ringI + ((pl - k0) % Lay::RI) * IT_SLOT; };
    auto ldA = [&](int pl, uint64_t *bar) {
        tma::load3d(tA(pl, 0), &tm.sg[0], x0 - 4, y0 - 2, pl, bar);   // sxx
        tma::load3d(tA(pl, 1), &tm.sg[1], x0 - 4, y0 - 2, pl, bar);   // syy
        tma::load3d(tA(pl, 2), &tm.sg[3], x0 - 4, y0 - 2, pl, bar);   // sxy
    };
    auto ldB = [&](int pl, uint64_t *bar) {
        tma::load3d(tB(pl, 0), &tm.sg[4], x0 - 4, y0 - 2, pl, bar);   // sxz
        tma::load3d(tB(pl, 1), &tm.sg[5], x0 - 4, y0 - 2, pl, bar);   // syz
    };
    auto ldC = [&](int pl, uint64_t *bar) { tma::load3d(tC(pl), &tm.sg[2], x0 - 4, y0 - 2, pl, bar); };
    auto ldI = [&](int pl, uint64_t *bar) { tma::load3d(tI(pl), &tm.idx, x0, y0, pl, bar); };
    auto ldS = [&](int pl, float *s, uint64_t *bar) {
        for (int a = 0; a < 3; ++a) tma::load3d(s + a * NTH, &tm.v[a], x0, y0, pl, bar);
    };
    auto stS = [&](int pl, const float *s) {
        for (int a = 0; a < 3; ++a) tma::store3d(&tm.v[a], x0, y0, pl, s + a * NTH);
        tma::bulk_commit();
    };

    if (tid == 0) {
        tma::mbar_expect_tx(&bars[0], (3 + 4 * 2 + 4) * VT_BYTES + 2 * IT + Lay::STAGE_BYTES);
        ldA(k0, &bars[0]);
        for (int pl = k0 - 2; pl <= k0 + 1; ++pl) ldB(pl, &bars[0]);
        for (int pl = k0 - 1; pl <= k0 + 2; ++pl) ldC(pl, &bars[0]);
        ldI(k0, &bars[0]);
        ldI(k0 + 1, &bars[0]);
        ldS(k0, stage(0), &bars[0]);
    }

    const st::Dx ix = st::make_dx(p.inv_dx);
    const float dt = p.dt;
    const int cv = (ty + 2) * VW + tx + 4;
    const int ci = ty * IW + tx;
    const int xs = slab_pos(i, nx, p.P), ys = slab_pos(j, ny, p.P);
    const int Sxs = nz * ny * p.W, Sys = nz * p.W * nx, Szs = p.W * ny * nx;
    const float2 *pmlx = p.pml, *pmly = p.pml + 2 * p.nmax, *pmlz = p.pml + 4 * p.nmax;

    // ring slots, rotated once per plane: A holds plane k (slot a0) and k+1;
    // B holds planes k-2 .. k+2 from slot b0; C holds k-1 .. k+3 from slot c0;
    // the index ring holds k, k+1, k+2 from slot i0; stage of plane k: s0.
    int a0 = 0, b0 = 0, c0 = 0, i0 = 0, s0 = 0;
    auto wrap = [](int v, int n) { return v >= n ? v - n : v; };
    int it = 0;
    for (int k = k0; k < k1; ++k, ++it) {
        __syncthreads();
        if (tid == 0) {
            if (it > 0) stS(k - 1, stage(it - 1));
            if (k + 1 < k1) {
                tma::bulk_wait_read<1>();
                tma::fence_async_smem();
                uint64_t *bar = &bars[(it + 1) & 1];
                tma::mbar_expect_tx(bar, 6 * VT_BYTES + IT + Lay::STAGE_BYTES);
                ldA(k + 1, bar);
                ldB(k + 2, bar);
                ldC(k + 3, bar);
                ldI(k + 2, bar);
                ldS(k + 1, stage(it + 1), bar);
            }
        }
        const bool ready = tma::mbar_wait(&bars[it & 1], (it >> 1) & 1, p.flag);
        if (ready && live) {
            float *s = stages + s0 * (Lay::STAGE_BYTES / 4) + tid;
            const float *XX = ringA + (a0 * 3 + 0) * VT + cv;
            const float *YY = ringA + (a0 * 3 + 1) * VT + cv;
            const float *XY = ringA + (a0 * 3 + 2) * VT + cv;
            const int bm2 = b0, bm1 = wrap(b0 + 1, 5), bk = wrap(b0 + 2, 5), bp1 = wrap(b0 + 3, 5);
            const float *XZ = ringB + (bk * 2 + 0) * VT + cv;
            const float *YZ = ringB + (bk * 2 + 1) * VT + cv;
            const uint8_t *I0 = ringI + i0 * IT_SLOT + ci;
            const uint8_t *I1 = ringI + wrap(i0 + 1, 3) * IT_SLOT + ci;
            const bool ix1 = i < nx - 1, jy1 = j < ny - 1, kz1 = k < nz - 1;
            const int zs = slab_pos(k, nz, p.P);
            const float rho0 = s_rho[I0[0]];
            if (ix1) {
                float d1 = dfw(XX[-1], XX[0], XX[1], XX[2], ix);
                float d2 = dbw(XY[-2 * VW], XY[-VW], XY[0], XY[VW], ix);
                float d3 = dbw(ringB[(bm2 * 2) * VT + cv], ringB[(bm1 * 2) * VT + cv], XZ[0],
                               ringB[(bp1 * 2) * VT + cv], ix);
                if (xs >= 0) d1 = cpml(p.psx + 0 * Sxs + (k * ny + j) * p.W + xs, pmlx[p.nmax + i], d1);
                if (ys >= 0) d2 = cpml(p.psy + 0 * Sys + (k * p.W + ys) * nx + i, pmly[j], d2);
                if (zs >= 0) d3 = cpml(p.psz + 0 * Szs + (zs * ny + j) * nx + i, pmlz[k], d3);
                s[0] += st::vel_increment(dt, rho0, s_rho[I0[1]], d1, d2, d3);
            }
            if (jy1) {
                float d1 = dbw(XY[-2], XY[-1], XY[0], XY[1], ix);
                float d2 = dfw(YY[-VW], YY[0], YY[VW], YY[2 * VW], ix);
                float d3 = dbw(ringB[(bm2 * 2 + 1) * VT + cv], ringB[(bm1 * 2 + 1) * VT + cv], YZ[0],
                               ringB[(bp1 * 2 + 1) * VT + cv], ix);
                if (xs >= 0) d1 = cpml(p.psx + 1 * Sxs + (k * ny + j) * p.W + xs, pmlx[i], d1);
                if (ys >= 0) d2 = cpml(p.psy + 1 * Sys + (k * p.W + ys) * nx + i, pmly[p.nmax + j], d2);
                if (zs >= 0) d3 = cpml(p.psz + 1 * Szs + (zs * ny + j) * nx + i, pmlz[k], d3);
                s[NTH] += st::vel_increment(dt, rho0, s_rho[I0[IW]], d1, d2, d3);
            }
            if (kz1) {
                const int cm1 = c0, ck = wrap(c0 + 1, 5), cp1 = wrap(c0 + 2, 5), cp2 = wrap(c0 + 3, 5);
                float d1 = dbw(XZ[-2], XZ[-1], XZ[0], XZ[1], ix);
                float d2 = dbw(YZ[-2 * VW], YZ[-VW], YZ[0], YZ[VW], ix);
                float d3 = dfw(ringC[cm1 * VT + cv], ringC[ck * VT + cv], ringC[cp1 * VT + cv],
                               ringC[cp2 * VT + cv], ix);
                if (xs >= 0) d1 = cpml(p.psx + 2 * Sxs + (k * ny + j) * p.W + xs, pmlx[i], d1);
                if (ys >= 0) d2 = cpml(p.psy + 2 * Sys + (k * p.W + ys) * nx + i, pmly[j], d2);
                if (zs >= 0) d3 = cpml(p.psz + 2 * Szs + (zs * ny + j) * nx + i, pmlz[p.nmax + k], d3);
                s[2 * NTH] += st::vel_increment(dt, rho0, s_rho[I1[0]], d1, d2, d3);
            }
        }
        tma::fence_async_smem();
        a0 ^= 1;
        b0 = wrap(b0 + 1, 5);
        c0 = wrap(c0 + 1, 5);
        i0 = wrap(i0 + 1, 3);
        s0 = wrap(s0 + 1, 3);
    }
    __syncthreads();
    if (tid == 0 && it > 0) {
        stS(k1 - 1, stage(it - 1));
        tma::bulk_wait<0>();
    }
}

// ------------------------------------------------------------------ stress
template <int L>
struct StressLayout {
    static constexpr int NS = 6 + 6 * L + 1;               // staged float arrays
    static constexpr int STAGE_F = NS * NTH;
    static constexpr int STAGE_BYTES = STAGE_F * 4 + 2 * NTH * 8;   // + FP64 C, S
    static constexpr int RV = 6, RI = 3;
    static constexpr size_t off_v = (size_t)NSTG * STAGE_BYTES;     // vx, vy, vz (k-2 .. k+3)
    static constexpr size_t off_i = off_v + (size_t)RV * 3 * VT_BYTES;
    static constexpr size_t off_bar = off_i + RI * IT_SLOT;
    static constexpr size_t off_lut = off_bar + 16;
    static size_t bytes(int n_mat) { return off_lut + (size_t)n_mat * sizeof(st::StressCoef); }
};

template <int L>
__global__ void __launch_bounds__(NTH, 2)
    k_stress_tma(const __grid_constant__ AcParams p, int kchunk,
                 const __grid_constant__ StressTmaMaps tm)
{
    using Lay = StressLayout<L>;
    constexpr int NS = Lay::NS;
    extern __shared__ __align__(1024) unsigned char sm[];
    float *stages = reinterpret_cast<float *>(sm);
    float *ringV = reinterpret_cast<float *>(sm + Lay::off_v);
    uint8_t *ringI = sm + Lay::off_i;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + Lay::off_bar);
    st::StressCoef *s_lut = reinterpret_cast<st::StressCoef *>(sm + Lay::off_lut);

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int i = x0 + tx, j = y0 + ty;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const bool live = i < nx && j < ny;
    const int k0 = blockIdx.z * kchunk, k1 = min(nz, k0 + kchunk);
    for (int m = tid; m < p.n_mat; m += NTH) s_lut[m] = st::make_stress_coef(p.lut[m], p.Lf);
    if (tid == 0) {
        tma::mbar_init(&bars[0], 1);
        tma::mbar_init(&bars[1], 1);
        tma::mbar_init_fence();
    }
    __syncthreads();

    const unsigned sbytes = (NS - 1) * NTH * 4 + (p.do_peak ? NTH * 4 : 0) + (p.do_dft ? 2 * NTH * 8 : 0);
    auto stage = [&](int it) { return stages + (size_t)(it % NSTG) * (Lay::STAGE_BYTES / 4); };
    auto tV = [&](int pl, int a) { return ringV + (((pl - k0 + 2) % Lay::RV) * 3 + a) * VT; };
    auto tI = [&](int pl) { return ringI + ((pl - k0) % Lay::RI) * IT_SLOT; };
    auto ldV = [&](int pl, uint64_t *bar) {
        for (int a = 0; a < 3; ++a) tma::load3d(tV(pl, a), &tm.v[a], x0 - 4, y0 - 2, pl, bar);
    };
    auto ldI = [&](int pl, uint64_t *bar) { tma::load3d(tI(pl), &tm.idx, x0, y0, pl, bar); };
    auto ldS = [&](int pl, float *s, uint64_t *bar) {
        for (int a = 0; a < NS - 1; ++a) tma::load3d(s + a * NTH, &tm.s[a], x0, y0, pl, bar);
        if (p.do_peak) tma::load3d(s + (NS - 1) * NTH, &tm.s[NS - 1], x0, y0, pl, bar);
        if (p.do_dft) {
            double *dd = reinterpret_cast<double *>(s + Lay::STAGE_F);
            tma::load3d(dd, &tm.s[NS], x0, y0, pl, bar);
            tma::load3d(dd + NTH, &tm.s[NS + 1], x0, y0, pl, bar);
        }
    };
    auto stS = [&](int pl, const float *s) {
        for (int a = 0; a < NS - 1; ++a) tma::store3d(&tm.s[a], x0, y0, pl, s + a * NTH);
        if (p.do_peak) tma::store3d(&tm.s[NS - 1], x0, y0, pl, s + (NS - 1) * NTH);
        if (p.do_dft) {
            const double *dd = reinterpret_cast<const double *>(s + Lay::STAGE_F);
            tma::store3d(&tm.s[NS], x0, y0, pl, dd);
            tma::store3d(&tm.s[NS + 1], x0, y0, pl, dd + NTH);
        }
        tma::bulk_commit();
    };

    if (tid == 0) {
        tma::mbar_expect_tx(&bars[0], 5 * 3 * VT_BYTES + 2 * IT + sbytes);
        for (int pl = k0 - 2; pl <= k0 + 2; ++pl) ldV(pl, &bars[0]);
        ldI(k0, &bars[0]);
        ldI(k0 + 1, &bars[0]);
        ldS(k0, stage(0), &bars[0]);
    }

    const st::Dx ix = st::make_dx(p.inv_dx);
    const int cv = (ty + 2) * VW + tx + 4;
    const int ci = ty * IW + tx;
    const int xs = slab_pos(i, nx, p.P), ys = slab_pos(j, ny, p.P);
    const int Sxs = nz * ny * p.W, Sys = nz * p.W * nx, Szs = p.W * ny * nx;
    const float2 *pmlx = p.pml, *pmly = p.pml + 2 * p.nmax, *pmlz = p.pml + 4 * p.nmax;

    // ring slots, rotated once per plane: the v ring holds planes k-2 .. k+3
    // from slot v0; the index ring k .. k+2 from slot i0; stage of plane k: s0.
    int v0 = 0, i0 = 0, s0 = 0;
    auto wrap = [](int v, int n) { return v >= n ? v - n : v; };
    int it = 0;
    for (int k = k0; k < k1; ++k, ++it) {
        __syncthreads();
        if (tid == 0) {
            if (it > 0) stS(k - 1, stage(it - 1));
            if (k + 1 < k1) {
                tma::bulk_wait_read<1>();
                tma::fence_async_smem();
                uint64_t *bar = &bars[(it + 1) & 1];
                tma::mbar_expect_tx(bar, 3 * VT_BYTES + IT + sbytes);
                ldV(k + 3, bar);
                ldI(k + 2, bar);
                ldS(k + 1, stage(it + 1), bar);
            }
        }
        const bool ready = tma::mbar_wait(&bars[it & 1], (it >> 1) & 1, p.flag);
        if (ready && live) {
            float *s = stages + s0 * (Lay::STAGE_BYTES / 4) + tid;
            // plane k-2+r of velocity component a, at this thread's column
            const int r0 = v0, r1 = wrap(v0 + 1, 6), r2 = wrap(v0 + 2, 6), r3 = wrap(v0 + 3, 6),
                      r4 = wrap(v0 + 4, 6);
            const float *VX = ringV + (r2 * 3 + 0) * VT + cv;
            const float *VY = ringV + (r2 * 3 + 1) * VT + cv;
            const float *VZ = ringV + (r2 * 3 + 2) * VT + cv;
            const uint8_t *I0 = ringI + i0 * IT_SLOT + ci;
            const uint8_t *I1 = ringI + wrap(i0 + 1, 3) * IT_SLOT + ci;
            const bool ix1 = i < nx - 1, jy1 = j < ny - 1, kz1 = k < nz - 1;
            const int zs = slab_pos(k, nz, p.P);
            float sv[6], rv[L > 0 ? L : 1][6];
#pragma unroll
            for (int cc = 0; cc < 6; ++cc) sv[cc] = s[cc * NTH];
#pragma unroll
            for (int l = 0; l < L; ++l)
#pragma unroll
                for (int cc = 0; cc < 6; ++cc) rv[l][cc] = s[(6 + 6 * l + cc) * NTH];
            const int m00 = I0[0];
            const st::StressCoef c0 = s_lut[m00];

            // ---- normal stresses at (i, j, k)
            float exx = dbw(VX[-2], VX[-1], VX[0], VX[1], ix);
            float eyy = dbw(VY[-2 * VW], VY[-VW], VY[0], VY[VW], ix);
            float ezz = dbw(ringV[(r0 * 3 + 2) * VT + cv], ringV[(r1 * 3 + 2) * VT + cv], VZ[0],
                            ringV[(r3 * 3 + 2) * VT + cv], ix);
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
                float a = dfw(VX[-VW], VX[0], VX[VW], VX[2 * VW], ix);
                float b = dfw(VY[-1], VY[0], VY[1], VY[2], ix);
                if (ys >= 0) a = cpml(p.psy + 4 * Sys + (k * p.W + ys) * nx + i, pmly[p.nmax + j], a);
                if (xs >= 0) b = cpml(p.psx + 4 * Sxs + (k * ny + j) * p.W + xs, pmlx[p.nmax + i], b);
                st::shear_update<L>(p, s_lut, c0, m00, I0[1], I0[IW], I0[IW + 1], a + b, 3, sv, rv);
            }
            if (dxz) {                               // sxz at (i+1/2, j, k+1/2)
                float a = dfw(ringV[(r1 * 3 + 0) * VT + cv], VX[0], ringV[(r3 * 3 + 0) * VT + cv],
                              ringV[(r4 * 3 + 0) * VT + cv], ix);
                float b = dfw(VZ[-1], VZ[0], VZ[1], VZ[2], ix);
                if (zs >= 0) a = cpml(p.psz + 4 * Szs + (zs * ny + j) * nx + i, pmlz[p.nmax + k], a);
                if (xs >= 0) b = cpml(p.psx + 5 * Sxs + (k * ny + j) * p.W + xs, pmlx[p.nmax + i], b);
                st::shear_update<L>(p, s_lut, c0, m00, I0[1], I1[0], I1[1], a + b, 4, sv, rv);
            }
            if (dyz) {                               // syz at (i, j+1/2, k+1/2)
                float a = dfw(ringV[(r1 * 3 + 1) * VT + cv], VY[0], ringV[(r3 * 3 + 1) * VT + cv],
                              ringV[(r4 * 3 + 1) * VT + cv], ix);
                float b = dfw(VZ[-VW], VZ[0], VZ[VW], VZ[2 * VW], ix);
                if (zs >= 0) a = cpml(p.psz + 5 * Szs + (zs * ny + j) * nx + i, pmlz[p.nmax + k], a);
                if (ys >= 0) b = cpml(p.psy + 5 * Sys + (k * p.W + ys) * nx + i, pmly[p.nmax + j], b);
                st::shear_update<L>(p, s_lut, c0, m00, I0[IW], I1[0], I1[IW], a + b, 5, sv, rv);
            }

            // ---- results back into the stage (ghost points keep their zeros)
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) s[cc * NTH] = sv[cc];
            if (dxy) s[3 * NTH] = sv[3];
            if (dxz) s[4 * NTH] = sv[4];
            if (dyz) s[5 * NTH] = sv[5];
#pragma unroll
            for (int l = 0; l < L; ++l)
#pragma unroll
                for (int cc = 0; cc < 6; ++cc) {
                    const bool w = cc < 3 || (cc == 3 && dxy) || (cc == 4 && dxz) || (cc == 5 && dyz);
                    if (w) s[(6 + 6 * l + cc) * NTH] = rv[l][cc];
                }
            if (p.do_peak) s[(NS - 1) * NTH] = fmaxf(s[(NS - 1) * NTH], fabsf(pr));
            if (p.do_dft) {
                double *dd = reinterpret_cast<double *>(stages + s0 * (Lay::STAGE_BYTES / 4) + Lay::STAGE_F) + tid;
                dd[0] = fma((double)pr, p.cw, dd[0]);
                dd[NTH] = fma((double)pr, p.sw, dd[NTH]);
            }
        }
        tma::fence_async_smem();
        v0 = wrap(v0 + 1, 6);
        i0 = wrap(i0 + 1, 3);
        s0 = wrap(s0 + 1, 3);
    }
    __syncthreads();
    if (tid == 0 && it > 0) {
        stS(k1 - 1, stage(it - 1));
        tma::bulk_wait<0>();
    }
}

}  // namespace

size_t velocity_tma_smem(int n_mat) { return VelLayout::bytes(n_mat); }

size_t stress_tma_smem(int L, int n_mat)
{
    switch (L) {
    case 0: return StressLayout<0>::bytes(n_mat);
    case 1: return StressLayout<1>::bytes(n_mat);
    default: return StressLayout<2>::bytes(n_mat);
    }
}

static dim3 grid_tma(const AcParams &p, int kc)
{
    return dim3((p.nx + TX - 1) / TX, (p.ny + TY - 1) / TY, (p.nz + kc - 1) / kc);
}

cudaError_t launch_velocity_tma(const AcParams &p, const VelocityTmaMaps &tm, cudaStream_t s)
{
    const int kc = p.kchunk > 0 ? p.kchunk : default_kchunk_tma(p.nx, p.ny, p.nz);
    const size_t sm = velocity_tma_smem(p.n_mat);
    cudaError_t e = cudaFuncSetAttribute(k_velocity_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    k_velocity_tma<<<grid_tma(p, kc), dim3(TX, TY, 1), sm, s>>>(p, kc, tm);
    return cudaGetLastError();
}

template <int L>
static cudaError_t launch_stress_tma_t(const AcParams &p, const StressTmaMaps &tm, cudaStream_t s)
{
    const int kc = p.kchunk > 0 ? p.kchunk : default_kchunk_tma(p.nx, p.ny, p.nz);
    const size_t sm = StressLayout<L>::bytes(p.n_mat);
    cudaError_t e = cudaFuncSetAttribute(k_stress_tma<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    k_stress_tma<L><<<grid_tma(p, kc), dim3(TX, TY, 1), sm, s>>>(p, kc, tm);
    return cudaGetLastError();
}

cudaError_t launch_stress_tma(const AcParams &p, const StressTmaMaps &tm, cudaStream_t s)
{
    switch (p.L) {
    case 0: return launch_stress_tma_t<0>(p, tm, s);
    case 1: return launch_stress_tma_t<1>(p, tm, s);
    case 2: return launch_stress_tma_t<2>(p, tm, s);
    default: return cudaErrorInvalidValue;
    }
}

// z-chunk length of the TMA kernels: each chunk pays a prologue of five
// v-planes, so chunks are longer than for the direct kernels; about six waves
// of two resident blocks per SM.
int default_kchunk_tma(int nx, int ny, int nz)
{
    const long long tiles = (long long)((nx + TX - 1) / TX) * ((ny + TY - 1) / TY);
    const long long target = 152LL * 2 * 6;
    long long chunks = (target + tiles - 1) / tiles;
    if (chunks < 1) chunks = 1;
    int kc = (int)((nz + chunks - 1) / chunks);
    if (kc < 8) kc = 8;
    return kc > nz ? nz : kc;
}

}  // namespace bvf
