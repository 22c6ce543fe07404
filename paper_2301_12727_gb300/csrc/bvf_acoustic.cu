// Acoustic step kernels: velocity update, then stress + SLS memory variables +
// source + capture (arXiv 2301.12727, Sec. 2.3, Eq. 1; Sec. 3.2, Eq. 3).
//
// One thread per voxel, blocks of 32 x 8 (x, y) on one z-plane.  Neighbours
// are read through the read-only path; points outside the grid read as zero
// (two ghost layers), and the last half-grid point of each axis is a ghost
// that is never written.  CPML memories exist only in the edge slabs.
#include "bvf_internal.cuh"

namespace bvf {

namespace {

constexpr float kC1 = 1.125f;            // 9/8
constexpr float kC2 = -1.0f / 24.0f;     // -1/24

// D+ : integer-point field -> derivative at s + 1/2
__device__ __forceinline__ float dfw(float fm1, float f0, float f1, float f2, float ix)
{
    return fmaf(kC2, f2 - fm1, kC1 * (f1 - f0)) * ix;
}
// D- : half-point field -> derivative at s
__device__ __forceinline__ float dbw(float fm2, float fm1, float f0, float f1, float ix)
{
    return fmaf(kC2, f1 - fm2, kC1 * (f0 - fm1)) * ix;
}

// zero-ghost load of f at linear index q + d * stride, coordinate c + d in [0, n)
__device__ __forceinline__ float ldg0(const float *__restrict__ f, long long q, int c, int d,
                                      int n, long long stride)
{
    int cc = c + d;
    return (cc >= 0 && cc < n) ? __ldg(f + q + (long long)d * stride) : 0.0f;
}

// position of coordinate c in its axis' CPML slab (-1 outside):
// [0, P) on the low side, [n-P-1, n) on the high side.
__device__ __forceinline__ int slab_pos(int c, int n, int P)
{
    if (P <= 0) return -1;
    if (c < P) return c;
    if (c >= n - P - 1) return c - (n - P - 1) + P;
    return -1;
}

// CPML recursion psi <- b psi + a d; the derivative used is d + psi.
__device__ __forceinline__ float cpml(float *__restrict__ psi, float2 ab, float d)
{
    float v = fmaf(ab.x, d, ab.y * *psi);
    *psi = v;
    return d + v;
}

__global__ void __launch_bounds__(256) k_velocity(AcParams p)
{
    extern __shared__ float s_rho[];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int m = tid; m < p.n_mat; m += blockDim.x * blockDim.y) s_rho[m] = p.lut[m].rho;
    __syncthreads();

    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    if (i >= nx || j >= ny) return;
    const long long SX = 1, SY = nx, SZ = (long long)nx * ny;
    const long long q = k * SZ + j * SY + i;
    const float ix = p.inv_dx, dt = p.dt;
    const float rho0 = s_rho[p.idx[q]];
    const int xs = slab_pos(i, nx, p.P), ys = slab_pos(j, ny, p.P), zs = slab_pos(k, nz, p.P);
    const long long Sxs = (long long)nz * ny * p.W, Sys = (long long)nz * p.W * nx,
                    Szs = (long long)p.W * ny * nx;
    const long long qx = ((long long)k * ny + j) * p.W + xs;
    const long long qy = ((long long)k * p.W + ys) * nx + i;
    const long long qz = ((long long)zs * ny + j) * nx + i;
    const float2 *pmlx = p.pml, *pmly = p.pml + 2 * p.nmax, *pmlz = p.pml + 4 * p.nmax;

#define LX(f, d) ldg0(f, q, i, d, nx, SX)
#define LY(f, d) ldg0(f, q, j, d, ny, SY)
#define LZ(f, d) ldg0(f, q, k, d, nz, SZ)
    if (i < nx - 1) {
        const float b = 2.0f / (rho0 + s_rho[p.idx[q + SX]]);
        float d1 = dfw(LX(p.sxx, -1), LX(p.sxx, 0), LX(p.sxx, 1), LX(p.sxx, 2), ix);
        float d2 = dbw(LY(p.sxy, -2), LY(p.sxy, -1), LY(p.sxy, 0), LY(p.sxy, 1), ix);
        float d3 = dbw(LZ(p.sxz, -2), LZ(p.sxz, -1), LZ(p.sxz, 0), LZ(p.sxz, 1), ix);
        if (xs >= 0) d1 = cpml(p.psx + 0 * Sxs + qx, pmlx[p.nmax + i], d1);
        if (ys >= 0) d2 = cpml(p.psy + 0 * Sys + qy, pmly[j], d2);
        if (zs >= 0) d3 = cpml(p.psz + 0 * Szs + qz, pmlz[k], d3);
        p.vx[q] += dt * b * (d1 + d2 + d3);
    }
    if (j < ny - 1) {
        const float b = 2.0f / (rho0 + s_rho[p.idx[q + SY]]);
        float d1 = dbw(LX(p.sxy, -2), LX(p.sxy, -1), LX(p.sxy, 0), LX(p.sxy, 1), ix);
        float d2 = dfw(LY(p.syy, -1), LY(p.syy, 0), LY(p.syy, 1), LY(p.syy, 2), ix);
        float d3 = dbw(LZ(p.syz, -2), LZ(p.syz, -1), LZ(p.syz, 0), LZ(p.syz, 1), ix);
        if (xs >= 0) d1 = cpml(p.psx + 1 * Sxs + qx, pmlx[i], d1);
        if (ys >= 0) d2 = cpml(p.psy + 1 * Sys + qy, pmly[p.nmax + j], d2);
        if (zs >= 0) d3 = cpml(p.psz + 1 * Szs + qz, pmlz[k], d3);
        p.vy[q] += dt * b * (d1 + d2 + d3);
    }
    if (k < nz - 1) {
        const float b = 2.0f / (rho0 + s_rho[p.idx[q + SZ]]);
        float d1 = dbw(LX(p.sxz, -2), LX(p.sxz, -1), LX(p.sxz, 0), LX(p.sxz, 1), ix);
        float d2 = dbw(LY(p.syz, -2), LY(p.syz, -1), LY(p.syz, 0), LY(p.syz, 1), ix);
        float d3 = dfw(LZ(p.szz, -1), LZ(p.szz, 0), LZ(p.szz, 1), LZ(p.szz, 2), ix);
        if (xs >= 0) d1 = cpml(p.psx + 2 * Sxs + qx, pmlx[i], d1);
        if (ys >= 0) d2 = cpml(p.psy + 2 * Sys + qy, pmly[j], d2);
        if (zs >= 0) d3 = cpml(p.psz + 2 * Szs + qz, pmlz[p.nmax + k], d3);
        p.vz[q] += dt * b * (d1 + d2 + d3);
    }
}

// Memory-variable update of one stress component (Crank-Nicolson):
// r_l <- ca_l r_l - cb_l Theta ; returns sum_l (r_l^{n+1} + r_l^n).
template <int L>
__device__ __forceinline__ float sls_update(const AcParams &p, long long q, int c, float The)
{
    float sum = 0.0f;
#pragma unroll
    for (int l = 0; l < L; ++l) {
        float *r = p.mem + (size_t)(l * 6 + c) * p.fstride + q;
        float r0 = *r;
        float rn = p.ca[l] * r0 - p.cb[l] * The;
        sum += rn + r0;
        *r = rn;
    }
    return sum;
}

template <int L>
__global__ void __launch_bounds__(256) k_stress(AcParams p)
{
    extern __shared__ MatCoef s_lut[];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int m = tid; m < p.n_mat; m += blockDim.x * blockDim.y) s_lut[m] = p.lut[m];
    __syncthreads();

    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    if (i >= nx || j >= ny) return;
    const long long SX = 1, SY = nx, SZ = (long long)nx * ny;
    const long long q = k * SZ + j * SY + i;
    const float ix = p.inv_dx, dt = p.dt;
    const int xs = slab_pos(i, nx, p.P), ys = slab_pos(j, ny, p.P), zs = slab_pos(k, nz, p.P);
    const long long Sxs = (long long)nz * ny * p.W, Sys = (long long)nz * p.W * nx,
                    Szs = (long long)p.W * ny * nx;
    const long long qx = ((long long)k * ny + j) * p.W + xs;
    const long long qy = ((long long)k * p.W + ys) * nx + i;
    const long long qz = ((long long)zs * ny + j) * nx + i;
    const float2 *pmlx = p.pml, *pmly = p.pml + 2 * p.nmax, *pmlz = p.pml + 4 * p.nmax;
    const int m00 = p.idx[q];
    const MatCoef c0 = s_lut[m00];

    // ---- normal stresses at (i, j, k)
    float exx = dbw(LX(p.vx, -2), LX(p.vx, -1), LX(p.vx, 0), LX(p.vx, 1), ix);
    float eyy = dbw(LY(p.vy, -2), LY(p.vy, -1), LY(p.vy, 0), LY(p.vy, 1), ix);
    float ezz = dbw(LZ(p.vz, -2), LZ(p.vz, -1), LZ(p.vz, 0), LZ(p.vz, 1), ix);
    if (xs >= 0) exx = cpml(p.psx + 3 * Sxs + qx, pmlx[i], exx);
    if (ys >= 0) eyy = cpml(p.psy + 3 * Sys + qy, pmly[j], eyy);
    if (zs >= 0) ezz = cpml(p.psz + 3 * Szs + qz, pmlz[k], ezz);
    const float th = exx + eyy + ezz;

    float srcv = 0.0f;
    if (p.src_on && k == p.k_src) {
        const float2 a = p.src[(long long)j * nx + i];
        srcv = p.src_scale * fmaf(a.x, p.src_ws, a.y * p.src_wc);
    }
    float snew[3];
    const float ev[3] = {exx, eyy, ezz};
    float *sig[3] = {p.sxx, p.syy, p.szz};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float dev = th - ev[c];
        const float Psi = c0.piU * th - c0.mu2U * dev;
        const float The = c0.piT * th - c0.mu2T * dev;
        const float sum = sls_update<L>(p, q, c, The);
        float s = sig[c][q] + dt * (Psi + 0.5f * sum);
        s -= srcv;
        sig[c][q] = s;
        snew[c] = s;
    }

    // ---- capture: p = -(sxx + syy + szz) / 3
    const float pr = -(snew[0] + snew[1] + snew[2]) / 3.0f;
    if (!isfinite(pr)) atomicOr(p.flag, 1);
    if (p.do_peak) p.peak[q] = fmaxf(p.peak[q], fabsf(pr));
    if (p.do_dft) {
        p.dftC[q] += (double)pr * p.cw;
        p.dftS[q] += (double)pr * p.sw;
    }

    // ---- shear stresses: harmonic-mean mu and mean tau_S of the four cells
    // (pairs along the first axis summed first, to keep mirror symmetry)
    auto shear = [&](float *s, int c, long long o1, long long o2, float e) {
        const MatCoef a = s_lut[m00], b = s_lut[p.idx[q + o1]];
        const MatCoef cc = s_lut[p.idx[q + o2]], d = s_lut[p.idx[q + o1 + o2]];
        const float muh = 4.0f / ((a.inv_mu + b.inv_mu) + (cc.inv_mu + d.inv_mu));
        const float tsh = 0.25f * ((a.tauS + b.tauS) + (cc.tauS + d.tauS));
        const float Psi = muh * (1.0f + p.Lf * tsh) * e;
        const float The = muh * tsh * e;
        const float sum = sls_update<L>(p, q, c, The);
        s[q] += dt * (Psi + 0.5f * sum);
    };
    if (i < nx - 1 && j < ny - 1) {     // sxy at (i+1/2, j+1/2, k)
        float a = dfw(LY(p.vx, -1), LY(p.vx, 0), LY(p.vx, 1), LY(p.vx, 2), ix);
        float b = dfw(LX(p.vy, -1), LX(p.vy, 0), LX(p.vy, 1), LX(p.vy, 2), ix);
        if (ys >= 0) a = cpml(p.psy + 4 * Sys + qy, pmly[p.nmax + j], a);
        if (xs >= 0) b = cpml(p.psx + 4 * Sxs + qx, pmlx[p.nmax + i], b);
        shear(p.sxy, 3, SX, SY, a + b);
    }
    if (i < nx - 1 && k < nz - 1) {     // sxz at (i+1/2, j, k+1/2)
        float a = dfw(LZ(p.vx, -1), LZ(p.vx, 0), LZ(p.vx, 1), LZ(p.vx, 2), ix);
        float b = dfw(LX(p.vz, -1), LX(p.vz, 0), LX(p.vz, 1), LX(p.vz, 2), ix);
        if (zs >= 0) a = cpml(p.psz + 4 * Szs + qz, pmlz[p.nmax + k], a);
        if (xs >= 0) b = cpml(p.psx + 5 * Sxs + qx, pmlx[p.nmax + i], b);
        shear(p.sxz, 4, SX, SZ, a + b);
    }
    if (j < ny - 1 && k < nz - 1) {     // syz at (i, j+1/2, k+1/2)
        float a = dfw(LZ(p.vy, -1), LZ(p.vy, 0), LZ(p.vy, 1), LZ(p.vy, 2), ix);
        float b = dfw(LY(p.vz, -1), LY(p.vz, 0), LY(p.vz, 1), LY(p.vz, 2), ix);
        if (zs >= 0) a = cpml(p.psz + 5 * Szs + qz, pmlz[p.nmax + k], a);
        if (ys >= 0) b = cpml(p.psy + 5 * Sys + qy, pmly[p.nmax + j], b);
        shear(p.syz, 5, SY, SZ, a + b);
    }
#undef LX
#undef LY
#undef LZ
}

}  // namespace

static dim3 grid_of(const AcParams &p, dim3 blk)
{
    return dim3((p.nx + blk.x - 1) / blk.x, (p.ny + blk.y - 1) / blk.y, p.nz);
}

cudaError_t launch_velocity(const AcParams &p, cudaStream_t s)
{
    dim3 blk(32, 8, 1);
    k_velocity<<<grid_of(p, blk), blk, p.n_mat * sizeof(float), s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_stress(const AcParams &p, cudaStream_t s)
{
    dim3 blk(32, 8, 1);
    size_t sm = p.n_mat * sizeof(MatCoef);
    switch (p.L) {
    case 0: k_stress<0><<<grid_of(p, blk), blk, sm, s>>>(p); break;
    case 1: k_stress<1><<<grid_of(p, blk), blk, sm, s>>>(p); break;
    case 2: k_stress<2><<<grid_of(p, blk), blk, sm, s>>>(p); break;
    case 3: k_stress<3><<<grid_of(p, blk), blk, sm, s>>>(p); break;
    case 4: k_stress<4><<<grid_of(p, blk), blk, sm, s>>>(p); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace bvf
