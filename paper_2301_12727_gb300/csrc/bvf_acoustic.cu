// Direct acoustic step kernels (any grid shape, any L): velocity update, then
// stress + SLS memory variables + source + capture (arXiv 2301.12727,
// Sec. 2.3, Eq. 1; Sec. 3.2, Eq. 3).  Grids whose rows suit the TMA use the
// kernels of bvf_acoustic_tma.cu instead.
//
// Both kernels march along z.  A block of 32 x 8 threads owns one x-y tile and
// walks a chunk of z-planes; every thread owns one column of the tile:
//   * the 4-point z-stencils come from per-thread register queues, so each
//     plane of a z-differenced array is read from memory once;
//   * the x- and y-stencils of the current plane come from a shared-memory
//     tile with a 2-cell halo (strips only: the stencils never touch corners),
//     double-buffered so one barrier per plane suffices;
//   * the next plane's queue tails and halo values are loaded one iteration
//     ahead of use.
// Zero ghosts (points outside the grid) are produced when the tiles and queues
// are filled, so the arithmetic has no bounds tests.  The last half-grid point
// of each axis is a ghost that is never written.  CPML memories exist only in
// the edge slabs.
#include "bvf_stencil.cuh"

namespace bvf {

namespace {

using st::cpml;
using st::slab_pos;

__device__ __forceinline__ float dfw(float a, float b, float c, float d, st::Dx x)
{
    return st::dfw<float>(a, b, c, d, x);
}
__device__ __forceinline__ float dbw(float a, float b, float c, float d, st::Dx x)
{
    return st::dbw<float>(a, b, c, d, x);
}

constexpr int TX = 32, TY = 8, H = 2;
constexpr int SW = TX + 2 * H;           // tile row length (36)
constexpr int SH = TY + 2 * H;           // tile rows (12)
constexpr int TILE = SW * SH;
constexpr int NTH = TX * TY;
constexpr int NX_HALO = 4 * TY;          // x-strips: 2 columns each side of the TY rows
constexpr int NHALO = NX_HALO + 4 * TX;  // + y-strips: 2 rows above and below the TX columns

// Tile coordinates (hx, hy) of halo element t: t < NX_HALO are the x-strips,
// the rest the y-strips.
__device__ __forceinline__ void halo_coord(int t, int &hx, int &hy)
{
    if (t < NX_HALO) {
        const int r = t >> 2, c = t & 3;
        hy = H + r;
        hx = (c < 2) ? c : TX + c;
    } else {
        t -= NX_HALO;
        const int r = t / TX, c = t % TX;
        hx = H + c;
        hy = (r < 2) ? r : TY + r;
    }
}

struct Geo {
    int nx, ny, nz;
    int SZ;
    int i, j, tx, ty, tid;
    bool live;
    int col;            // j*nx + i
    bool hal, hin;      // this thread fills a halo element / it lies inside the grid
    int hslot;          // its index in the tile
    bool hxstrip;       // the element belongs to an x-strip
    int hcol;           // its gy*nx + gx
};

__device__ __forceinline__ Geo make_geo(int nx, int ny, int nz)
{
    Geo g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.SZ = nx * ny;
    g.tx = threadIdx.x;
    g.ty = threadIdx.y;
    g.tid = g.ty * TX + g.tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    g.i = x0 + g.tx;
    g.j = y0 + g.ty;
    g.live = g.i < nx && g.j < ny;
    g.col = g.j * nx + g.i;
    g.hal = g.tid < NHALO;
    int hx = 0, hy = 0;
    if (g.hal) halo_coord(g.tid, hx, hy);
    g.hxstrip = g.tid < NX_HALO;
    const int gx = x0 - H + hx, gy = y0 - H + hy;
    g.hin = g.hal && gx >= 0 && gx < nx && gy >= 0 && gy < ny;
    g.hslot = hy * SW + hx;
    g.hcol = gy * nx + gx;
    return g;
}

// column value f(i, j, k), zero outside the grid
template <typename T>
__device__ __forceinline__ float colv(const T *__restrict__ f, const Geo &g, int k)
{
    return (g.live && k >= 0 && k < g.nz) ? st::tof(__ldg(f + k * g.SZ + g.col)) : 0.0f;
}
// halo value of this thread's halo element at plane k, zero outside the grid
template <typename T>
__device__ __forceinline__ float halv(const T *__restrict__ f, const Geo &g, int k, bool want)
{
    return (want && g.hin && k >= 0 && k < g.nz) ? st::tof(__ldg(f + k * g.SZ + g.hcol)) : 0.0f;
}

template <typename T>
__global__ void __launch_bounds__(NTH, 3) k_velocity(AcParams p, int kchunk)
{
    extern __shared__ __align__(16) float sm_v[];
    float *tiles = sm_v;                               // [2 buffers][5 arrays][TILE]
    const Geo g = make_geo(p.nx, p.ny, p.nz);

    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int k0 = blockIdx.z * kchunk, k1 = min(nz, k0 + kchunk);
    const st::Dx ix = st::make_dx(p.inv_dx);
    const float dt = p.dtv;
    const int c = (g.ty + H) * SW + (g.tx + H);
    const int xs = slab_pos(g.i, nx, p.P), ys = slab_pos(g.j, ny, p.P);
    const int Sxs = nz * ny * p.W, Sys = nz * p.W * nx, Szs = p.W * ny * nx;
    const float2 *pmlx = p.pml, *pmly = p.pml + 2 * p.nmax, *pmlz = p.pml + 4 * p.nmax;
    const bool hx_ = g.hxstrip, hy_ = !g.hxstrip;
    const uint8_t *__restrict__ idx = p.idx;
    T *__restrict__ vx = static_cast<T *>(p.vx);
    T *__restrict__ vy = static_cast<T *>(p.vy);
    T *__restrict__ vz = static_cast<T *>(p.vz);
    const T *sxx = static_cast<const T *>(p.sxx), *syy = static_cast<const T *>(p.syy);
    const T *szz = static_cast<const T *>(p.szz), *sxy = static_cast<const T *>(p.sxy);
    const T *sxz = static_cast<const T *>(p.sxz), *syz = static_cast<const T *>(p.syz);

    // z-queues: sxz, syz at k-2 .. k+1 ; szz at k-1 .. k+2
    float bz0 = colv(sxz, g, k0 - 2), bz1 = colv(sxz, g, k0 - 1);
    float bz2 = colv(sxz, g, k0), bz3 = colv(sxz, g, k0 + 1);
    float cz0 = colv(syz, g, k0 - 2), cz1 = colv(syz, g, k0 - 1);
    float cz2 = colv(syz, g, k0), cz3 = colv(syz, g, k0 + 1);
    float dz0 = colv(szz, g, k0 - 1), dz1 = colv(szz, g, k0);
    float dz2 = colv(szz, g, k0 + 1), dz3 = colv(szz, g, k0 + 2);
    // plane-k centres of the x/y-differenced arrays and this thread's halo values
    float cxx = colv(sxx, g, k0), cyy = colv(syy, g, k0), cxy = colv(sxy, g, k0);
    float hxx = halv(sxx, g, k0, hx_), hyy = halv(syy, g, k0, hy_);
    float hxy = halv(sxy, g, k0, true), hxz = halv(sxz, g, k0, hx_);
    float hyz = halv(syz, g, k0, hy_);
    __syncthreads();

    for (int k = k0; k < k1; ++k) {
        float *t = tiles + (k & 1) * 5 * TILE;
        float *txx = t, *tyy = t + TILE, *txy = t + 2 * TILE, *txz = t + 3 * TILE, *tyz = t + 4 * TILE;
        txx[c] = cxx; tyy[c] = cyy; txy[c] = cxy; txz[c] = bz2; tyz[c] = cz2;
        if (g.hal) {
            txx[g.hslot] = hxx; tyy[g.hslot] = hyy; txy[g.hslot] = hxy;
            txz[g.hslot] = hxz; tyz[g.hslot] = hyz;
        }
        __syncthreads();
        // loads for plane k+1, consumed in the next iteration
        const float nbz = colv(sxz, g, k + 2), ncz = colv(syz, g, k + 2);
        const float ndz = colv(szz, g, k + 3);
        const float nxx = colv(sxx, g, k + 1), nyy = colv(syy, g, k + 1);
        const float nxy = colv(sxy, g, k + 1);
        const float nhxx = halv(sxx, g, k + 1, hx_), nhyy = halv(syy, g, k + 1, hy_);
        const float nhxy = halv(sxy, g, k + 1, true), nhxz = halv(sxz, g, k + 1, hx_);
        const float nhyz = halv(syz, g, k + 1, hy_);

        if (g.live) {
            const int q = k * g.SZ + g.col;
            const int zs = slab_pos(k, nz, p.P);
            const int qx = (k * ny + g.j) * p.W + xs;
            const int qy = (k * p.W + ys) * nx + g.i;
            const int qz = (zs * ny + g.j) * nx + g.i;
            const bool ix1 = g.i < nx - 1, jy1 = g.j < ny - 1, kz1 = k < nz - 1;
            // every global load of this voxel first
            const int m0 = __ldg(idx + q), mx = __ldg(idx + q + (ix1 ? 1 : 0));
            const int my = __ldg(idx + q + (jy1 ? nx : 0)), mz = __ldg(idx + q + (kz1 ? g.SZ : 0));
            float ux = st::tof(vx[q]), uy = st::tof(vy[q]), uz = st::tof(vz[q]);
            if (ix1) {
                float d1 = dfw(txx[c - 1], txx[c], txx[c + 1], txx[c + 2], ix);
                float d2 = dbw(txy[c - 2 * SW], txy[c - SW], txy[c], txy[c + SW], ix);
                float d3 = dbw(bz0, bz1, bz2, bz3, ix);
                if (xs >= 0) d1 = cpml(p.psx + 0 * Sxs + qx, pmlx[p.nmax + g.i], d1);
                if (ys >= 0) d2 = cpml(p.psy + 0 * Sys + qy, pmly[g.j], d2);
                if (zs >= 0) d3 = cpml(p.psz + 0 * Szs + qz, pmlz[k], d3);
                ux = st::vel_step(dt, st::buoyancy(p.buoy, p.n_mat, m0, mx), ux, d1, d2, d3);
                st::stv(vx + q, ux);
            }
            if (jy1) {
                float d1 = dbw(txy[c - 2], txy[c - 1], txy[c], txy[c + 1], ix);
                float d2 = dfw(tyy[c - SW], tyy[c], tyy[c + SW], tyy[c + 2 * SW], ix);
                float d3 = dbw(cz0, cz1, cz2, cz3, ix);
                if (xs >= 0) d1 = cpml(p.psx + 1 * Sxs + qx, pmlx[g.i], d1);
                if (ys >= 0) d2 = cpml(p.psy + 1 * Sys + qy, pmly[p.nmax + g.j], d2);
                if (zs >= 0) d3 = cpml(p.psz + 1 * Szs + qz, pmlz[k], d3);
                uy = st::vel_step(dt, st::buoyancy(p.buoy, p.n_mat, m0, my), uy, d1, d2, d3);
                st::stv(vy + q, uy);
            }
            if (kz1) {
                float d1 = dbw(txz[c - 2], txz[c - 1], txz[c], txz[c + 1], ix);
                float d2 = dbw(tyz[c - 2 * SW], tyz[c - SW], tyz[c], tyz[c + SW], ix);
                float d3 = dfw(dz0, dz1, dz2, dz3, ix);
                if (xs >= 0) d1 = cpml(p.psx + 2 * Sxs + qx, pmlx[g.i], d1);
                if (ys >= 0) d2 = cpml(p.psy + 2 * Sys + qy, pmly[g.j], d2);
                if (zs >= 0) d3 = cpml(p.psz + 2 * Szs + qz, pmlz[p.nmax + k], d3);
                uz = st::vel_step(dt, st::buoyancy(p.buoy, p.n_mat, m0, mz), uz, d1, d2, d3);
                st::stv(vz + q, uz);
            }
        }
        bz0 = bz1; bz1 = bz2; bz2 = bz3; bz3 = nbz;
        cz0 = cz1; cz1 = cz2; cz2 = cz3; cz3 = ncz;
        dz0 = dz1; dz1 = dz2; dz2 = dz3; dz3 = ndz;
        cxx = nxx; cyy = nyy; cxy = nxy;
        hxx = nhxx; hyy = nhyy; hxy = nhxy; hxz = nhxz; hyz = nhyz;
    }
}

template <int L, typename T>
__global__ void __launch_bounds__(NTH, L <= 2 ? 3 : 2) k_stress(AcParams p, int kchunk)
{
    extern __shared__ __align__(16) float sm_s[];
    st::StressCoef *s_lut = reinterpret_cast<st::StressCoef *>(sm_s);
    float *tiles = sm_s + p.n_mat * (sizeof(st::StressCoef) / sizeof(float));   // [2][3][TILE]
    const Geo g = make_geo(p.nx, p.ny, p.nz);
    for (int m = g.tid; m < p.n_mat; m += NTH) s_lut[m] = st::make_stress_coef(p.lut[m], p.Lf);

    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int k0 = blockIdx.z * kchunk, k1 = min(nz, k0 + kchunk);
    const st::Dx ix = st::make_dx(p.inv_dx);
    const int c = (g.ty + H) * SW + (g.tx + H);
    const int xs = slab_pos(g.i, nx, p.P), ys = slab_pos(g.j, ny, p.P);
    const int Sxs = nz * ny * p.W, Sys = nz * p.W * nx, Szs = p.W * ny * nx;
    const float2 *pmlx = p.pml, *pmly = p.pml + 2 * p.nmax, *pmlz = p.pml + 4 * p.nmax;
    const uint8_t *__restrict__ idx = p.idx;
    T *__restrict__ mem = static_cast<T *>(p.mem);
    const T *vxg = static_cast<const T *>(p.vx), *vyg = static_cast<const T *>(p.vy);
    const T *vzg = static_cast<const T *>(p.vz);
    float *__restrict__ peak = p.peak;
    T *const sig[6] = {static_cast<T *>(p.sxx), static_cast<T *>(p.syy), static_cast<T *>(p.szz),
                       static_cast<T *>(p.sxy), static_cast<T *>(p.sxz), static_cast<T *>(p.syz)};

    // z-queues: vx, vy at k-1 .. k+2 ; vz at k-2 .. k+1
    float ax0 = colv(vxg, g, k0 - 1), ax1 = colv(vxg, g, k0);
    float ax2 = colv(vxg, g, k0 + 1), ax3 = colv(vxg, g, k0 + 2);
    float ay0 = colv(vyg, g, k0 - 1), ay1 = colv(vyg, g, k0);
    float ay2 = colv(vyg, g, k0 + 1), ay3 = colv(vyg, g, k0 + 2);
    float az0 = colv(vzg, g, k0 - 2), az1 = colv(vzg, g, k0 - 1);
    float az2 = colv(vzg, g, k0), az3 = colv(vzg, g, k0 + 1);
    float hvx = halv(vxg, g, k0, true), hvy = halv(vyg, g, k0, true);
    float hvz = halv(vzg, g, k0, true);
    __syncthreads();

    for (int k = k0; k < k1; ++k) {
        float *t = tiles + (k & 1) * 3 * TILE;
        float *tvx = t, *tvy = t + TILE, *tvz = t + 2 * TILE;
        tvx[c] = ax1; tvy[c] = ay1; tvz[c] = az2;
        if (g.hal) { tvx[g.hslot] = hvx; tvy[g.hslot] = hvy; tvz[g.hslot] = hvz; }
        __syncthreads();
        const float nax = colv(vxg, g, k + 3), nay = colv(vyg, g, k + 3);
        const float naz = colv(vzg, g, k + 2);
        const float nhx = halv(vxg, g, k + 1, true), nhy = halv(vyg, g, k + 1, true);
        const float nhz = halv(vzg, g, k + 1, true);

        if (g.live) {
            const int q = k * g.SZ + g.col;
            const int zs = slab_pos(k, nz, p.P);
            const int qx = (k * ny + g.j) * p.W + xs;
            const int qy = (k * p.W + ys) * nx + g.i;
            const int qz = (zs * ny + g.j) * nx + g.i;
            // ---- every global load of this voxel first (independent, in flight together)
            const bool ix1 = g.i < nx - 1, jy1 = g.j < ny - 1, kz1 = k < nz - 1;
            const int o1 = ix1 ? 1 : 0, oy = jy1 ? nx : 0, oz = kz1 ? g.SZ : 0;
            const int m00 = __ldg(idx + q), m10 = __ldg(idx + q + o1);
            const int m01 = __ldg(idx + q + oy), m11 = __ldg(idx + q + o1 + oy);
            const int mz0 = __ldg(idx + q + oz), mz1 = __ldg(idx + q + o1 + oz);
            const int mzy = __ldg(idx + q + oy + oz);
            float sv[6], rv[L > 0 ? L : 1][6];
#pragma unroll
            for (int cc = 0; cc < 6; ++cc) sv[cc] = st::tof(sig[cc][q]);
#pragma unroll
            for (int l = 0; l < L; ++l)
#pragma unroll
                for (int cc = 0; cc < 6; ++cc)
                    rv[l][cc] = st::tof(mem[mem_index(l, cc, q, p.fstride, L)]);
            const float pk = (p.st.flags & kStepPeak) ? peak[q] : 0.0f;
            double dC = 0.0, dS = 0.0;
            if (p.st.flags & kStepDft) { dC = p.dftC[q]; dS = p.dftS[q]; }
            const st::StressCoef c0 = s_lut[m00];

            // ---- normal stresses at (i, j, k)
            float exx = dbw(tvx[c - 2], tvx[c - 1], tvx[c], tvx[c + 1], ix);
            float eyy = dbw(tvy[c - 2 * SW], tvy[c - SW], tvy[c], tvy[c + SW], ix);
            float ezz = dbw(az0, az1, az2, az3, ix);
            if (xs >= 0) exx = cpml(p.psx + 3 * Sxs + qx, pmlx[g.i], exx);
            if (ys >= 0) eyy = cpml(p.psy + 3 * Sys + qy, pmly[g.j], eyy);
            if (zs >= 0) ezz = cpml(p.psz + 3 * Szs + qz, pmlz[k], ezz);
            float srcv = 0.0f;
            if ((p.st.flags & kStepSource) && k == p.k_src) {
                const float2 a = p.src[g.col];
                srcv = st::source_value<float>(p.src_scale, a.x, a.y, p.st.src_ws, p.st.src_wc);
            }
            st::normal_update<L>(p, c0, exx, eyy, ezz, srcv, sv, rv);
            const float pr = st::pressure(sv);
            if (!isfinite(pr)) atomicOr(p.flag, 1);

            // ---- shear stresses
            auto shear = [&](int cc, int mb, int md, int mf, float e) {
                st::shear_update<L>(p, s_lut, c0, m00, mb, md, mf, e, cc, sv, rv);
            };
            const bool dxy = ix1 && jy1, dxz = ix1 && kz1, dyz = jy1 && kz1;
            if (dxy) {                               // sxy at (i+1/2, j+1/2, k)
                float a = dfw(tvx[c - SW], tvx[c], tvx[c + SW], tvx[c + 2 * SW], ix);
                float b = dfw(tvy[c - 1], tvy[c], tvy[c + 1], tvy[c + 2], ix);
                if (ys >= 0) a = cpml(p.psy + 4 * Sys + qy, pmly[p.nmax + g.j], a);
                if (xs >= 0) b = cpml(p.psx + 4 * Sxs + qx, pmlx[p.nmax + g.i], b);
                shear(3, m10, m01, m11, st::vadd(a, b));
            }
            if (dxz) {                               // sxz at (i+1/2, j, k+1/2)
                float a = dfw(ax0, ax1, ax2, ax3, ix);
                float b = dfw(tvz[c - 1], tvz[c], tvz[c + 1], tvz[c + 2], ix);
                if (zs >= 0) a = cpml(p.psz + 4 * Szs + qz, pmlz[p.nmax + k], a);
                if (xs >= 0) b = cpml(p.psx + 5 * Sxs + qx, pmlx[p.nmax + g.i], b);
                shear(4, m10, mz0, mz1, st::vadd(a, b));
            }
            if (dyz) {                               // syz at (i, j+1/2, k+1/2)
                float a = dfw(ay0, ay1, ay2, ay3, ix);
                float b = dfw(tvz[c - SW], tvz[c], tvz[c + SW], tvz[c + 2 * SW], ix);
                if (zs >= 0) a = cpml(p.psz + 5 * Szs + qz, pmlz[p.nmax + k], a);
                if (ys >= 0) b = cpml(p.psy + 5 * Sys + qy, pmly[p.nmax + g.j], b);
                shear(5, m01, mz0, mzy, st::vadd(a, b));
            }

            // ---- stores
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) st::stv(sig[cc] + q, sv[cc]);
            if (dxy) st::stv(sig[3] + q, sv[3]);
            if (dxz) st::stv(sig[4] + q, sv[4]);
            if (dyz) st::stv(sig[5] + q, sv[5]);
#pragma unroll
            for (int l = 0; l < L; ++l)
#pragma unroll
                for (int cc = 0; cc < 6; ++cc) {
                    const bool w = cc < 3 || (cc == 3 && dxy) || (cc == 4 && dxz) || (cc == 5 && dyz);
                    if (w) st::stv(mem + mem_index(l, cc, q, p.fstride, L), rv[l][cc]);
                }
            if (p.st.flags & kStepPeak) peak[q] = fmaxf(pk, fabsf(pr));
            if (p.st.flags & kStepDft) {
                p.dftC[q] = fma((double)pr, p.st.cw, dC);
                p.dftS[q] = fma((double)pr, p.st.sw, dS);
            }
        }
        ax0 = ax1; ax1 = ax2; ax2 = ax3; ax3 = nax;
        ay0 = ay1; ay1 = ay2; ay2 = ay3; ay3 = nay;
        az0 = az1; az1 = az2; az2 = az3; az3 = naz;
        hvx = nhx; hvy = nhy; hvz = nhz;
    }
}

}  // namespace

// z-chunk length: about two waves of four resident blocks per SM on 152 SMs,
// at least 8 planes per chunk (queue start-up costs 3 planes).
int default_kchunk(int nx, int ny, int nz)
{
    const long long tiles = (long long)((nx + TX - 1) / TX) * ((ny + TY - 1) / TY);
    const long long target = 152LL * 4 * 2;
    long long chunks = (target + tiles - 1) / tiles;
    if (chunks < 1) chunks = 1;
    int kc = (int)((nz + chunks - 1) / chunks);
    if (kc < 8) kc = 8;
    return kc > nz ? nz : kc;
}

static dim3 grid_of(const AcParams &p, int kchunk)
{
    return dim3((p.nx + TX - 1) / TX, (p.ny + TY - 1) / TY, (p.nz + kchunk - 1) / kchunk);
}

cudaError_t launch_velocity(const AcParams &p, cudaStream_t s)
{
    const int kc = p.kchunk > 0 ? p.kchunk : default_kchunk(p.nx, p.ny, p.nz);
    const size_t sm = 2 * 5 * TILE * sizeof(float);
    if (p.h16)
        k_velocity<__half><<<grid_of(p, kc), dim3(TX, TY, 1), sm, s>>>(p, kc);
    else
        k_velocity<float><<<grid_of(p, kc), dim3(TX, TY, 1), sm, s>>>(p, kc);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_stress_t(const AcParams &p, int kc, dim3 grd, dim3 blk, size_t sm,
                                   cudaStream_t s)
{
    switch (p.L) {
    case 0: k_stress<0, T><<<grd, blk, sm, s>>>(p, kc); break;
    case 1: k_stress<1, T><<<grd, blk, sm, s>>>(p, kc); break;
    case 2: k_stress<2, T><<<grd, blk, sm, s>>>(p, kc); break;
    case 3: k_stress<3, T><<<grd, blk, sm, s>>>(p, kc); break;
    case 4: k_stress<4, T><<<grd, blk, sm, s>>>(p, kc); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_stress(const AcParams &p, cudaStream_t s)
{
    const int kc = p.kchunk > 0 ? p.kchunk : default_kchunk(p.nx, p.ny, p.nz);
    const size_t sm = p.n_mat * sizeof(st::StressCoef) + 2 * 3 * TILE * sizeof(float);
    const dim3 grd = grid_of(p, kc), blk(TX, TY, 1);
    return p.h16 ? launch_stress_t<__half>(p, kc, grd, blk, sm, s)
                 : launch_stress_t<float>(p, kc, grd, blk, sm, s);
}

}  // namespace bvf
