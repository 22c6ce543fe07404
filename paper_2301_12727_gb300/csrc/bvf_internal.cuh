// Internal declarations of libbvf (not part of the public ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/bvf.h"

namespace bvf {

// Per-material coefficients of the acoustic kernels (FP32, derived in FP64 on
// the host).  Normal stress:  Psi = piU th - mu2U (th - e_ii),
//                             Theta = piT th - mu2T (th - e_ii);
// shear points combine inv_mu (harmonic mean) and tauS (arithmetic mean),
// stored next to each other so one 8-byte load fetches both.
struct MatCoef {
    float rho;     // density (buoyancy at v-points: 2 / (rho_a + rho_b))
    float piU;     // pi_R (1 + L tau_P)
    float piT;     // pi_R tau_P
    float mu2U;    // 2 mu_R (1 + L tau_S)
    float inv_mu;  // 1 / mu_R  (+inf for fluids, so the harmonic mean is 0)
    float tauS;    // tau_S
    float mu2T;    // 2 mu_R tau_S
    float pad;
};

// Per-material constants of the BHTE kernel.
struct ThermCoef {
    float k;         // face conductivity between two cells of this material: the
                     // diagonal entry of the BHTE pair table (the harmonic mean of k_th
                     // with itself, derived in FP64 and rounded once)
    float inv_rhoc;  // 1 / (rho c_th)
    float perfw;     // perf * rhob_cb
    float qfac;      // heat_frac * alphaL / (rho cL)
};

constexpr int kNumCpmlSlots = 6;   // CPML memories per slab (see ctx layout)

// Memory variable of mechanism l for stress component c at voxel q: the L
// mechanisms of one component and voxel are adjacent (one paired access for
// L = 2), components are fstride * L elements apart.
__host__ __device__ __forceinline__ size_t mem_index(int l, int c, size_t q, size_t fstride, int L)
{
    return ((size_t)c * fstride + q) * (size_t)L + (size_t)l;
}

// Source and capture parameters of one step (the update n -> n+1):
struct StepParam {
    double cw, sw;          // DFT weights cos / sin(w t) of the captured step
    float src_ws, src_wc;   // source envelope times sin / cos(w t)
    int flags;              // 1: source on, 2: peak capture, 4: DFT capture
    int pad;
};
enum { kStepSource = 1, kStepPeak = 2, kStepDft = 4 };

// The state (v, sigma, memory variables) is stored as float, or as FP16
// scaled so that stored values stay well inside FP16's range: v / S_v,
// sigma / S_sigma and r / S_r.  The equations are linear in the state, so the
// scales fold into the constants below and the kernels run the same FP32
// arithmetic on the stored values (all scales 1 for float storage):
//   velocity  dtv = dt S_sigma / S_v
//   stress    dt (the stress step) = dt S_v / S_sigma, memory-variable sum
//             weight rh = S_r / (2 S_v), cb_l divided by S_r / S_v (held
//             negated: ncb_l = -cb_l)
//   source    src_scale divided by S_sigma
// Captured p (peak map, DFT sums) is in units of S_sigma.
struct AcParams {
    int nx, ny, nz;
    int P, W;            // CPML cells per face; slab width 2P+1 (0 if no CPML)
    int L;               // SLS mechanisms
    int n_mat;
    int h16;             // state stored as scaled FP16
    float dt, dtv, inv_dx, Lf, rh;
    float ca[BVF_MAX_SLS], ncb[BVF_MAX_SLS];
    const uint8_t *idx;
    const MatCoef *lut;
    const float *buoy;   // 2 / (rho_a + rho_b) of every material pair, [a * n_mat + b]
    void *vx, *vy, *vz, *sxx, *syy, *szz, *sxy, *sxz, *syz;   // float or __half
    void *mem;           // memory variables, element mem_index(l, c, q)
    size_t fstride;
    float *psx, *psy, *psz;   // CPML slabs: x [6][nz][ny][W], y [6][nz][W][nx], z [6][W][ny][nx]
    const float2 *pml;   // (a, b) at [axis][h][s], h = 0 integer / 1 half point
    int nmax;
    // source plane
    const float2 *src;
    int k_src;
    float src_scale;     // 2 c0 dt / dx (over the stress storage scale)
    // capture
    float *peak;
    double *dftC, *dftS;
    StepParam st;        // this step's source and capture parameters
    int *flag;
    int kchunk;          // z-planes per block (0 = default_kchunk)
    // bounded TMA waits: polls per mbarrier wait before a block gives up
    // (sets bit 2 of *flag, issues no further copies, drains the copies it
    // has issued, and stops).  hold = 1 (velocity) or 2 (stress) makes that
    // kernel arm the barrier of its look-ahead copies at plane hold_plane but
    // issue none of them, so the wait that follows runs out with nothing in
    // flight: the test hook of the time-out path (0 = off).
    unsigned wait_limit;
    int hold, hold_plane;
    // rows of an x-y tile of the TMA-fed stress and velocity kernels: 4, 8 or
    // 16 (heights other than 8 with L = 2 only)
    int tile_y, tile_yv;
};

// Tensor maps of the TMA-fed acoustic kernels (x-y boxes of one z-plane).
// Stress kernel: the velocities with (32 + 2 XO) x 12 halo boxes and the
// material index with 48 x 9 boxes.  Velocity kernel: the six stresses (sxx,
// syy, szz, sxy, sxz, syz), each with a box holding the halo its stencil
// reads: (32 + 2 XO) x 8, 32 x 12, 32 x 8, (32 + 2 XO) x 12, (32 + 2 XO) x 8,
// 32 x 12; the material index.  XO = 16 bytes of the storage type.
struct StressTmaMaps {
    CUtensorMap v[3];
    CUtensorMap idx;
};
struct VelocityTmaMaps {
    CUtensorMap sg[6];
    CUtensorMap idx;
};

// Batched runs: up to kMaxBatch contexts advanced in lockstep by persistent
// kernels that take their work from a list of (domain, tile, z-chunk) items.
// Everything per domain travels in the kernel parameter (read-only constant
// space, so the compiler reloads instead of spilling); the tensor maps and the
// per-step tables sit in device memory.
constexpr int kMaxBatch = 64;
struct BatchParams {
    AcParams p[kMaxBatch];
    const StressTmaMaps *sm;     // [n_dom]
    const VelocityTmaMaps *vm;   // [n_dom]
    const StepParam *steps;      // domain d, step s: steps[step_off[d] + s]
    int step_off[kMaxBatch];
    int block0[kMaxBatch];       // first work item of each domain (ascending)
    int tiles_x[kMaxBatch], tiles_y[kMaxBatch], kchunk[kMaxBatch];
    int n_steps[kMaxBatch];      // steps of this run; later steps skip the domain
    int n_dom, total;            // domains, work items
};
static_assert(sizeof(BatchParams) <= 32000, "batch parameters must fit a kernel parameter");

// One BHTE step.  The CEM43 increments of consecutive steps are summed in an
// FP32 partial (cemf) and added to the FP64 dose on `flush` steps (every 32
// steps and the last), which keeps FP64 arithmetic out of most steps.
// The BHTE kernels advance the rise theta = T - T_a (the arterial
// temperature), not T: near 37 C an FP32 T carries 3.8e-6 C ulps, against
// which the per-step increments round; the rise is small and keeps ~2^10
// times finer resolution.  bvf_run_thermal converts on entry and exit.
struct ThParams {
    int nx, ny, nz;
    float dt, inv_dx2, dc, dt60;
    float rise43;            // 43 C - T_a: the CEM43 threshold as a rise
    const uint8_t *idx;
    const ThermCoef *lut;
    const float *kface;      // [n_mat][n_mat] harmonic-mean face conductivity (FP64-derived)
    int n_mat;
    const float *T;
    float *Tn;
    const float *Q;
    float *Tmax;
    float *cemf;
    double *cem;
    int flush;
    int kz;                  // z-planes per block (thermal_kchunk)
    // bounded waits of the TMA-fed step: polls per wait; hold_plane >= 0 makes
    // the kernel arm that plane's barrier but issue none of its copies (the
    // test hook of the time-out path; negative = off: plane -1, the one below
    // the grid, is loaded as zeros by the first z-chunk)
    unsigned wait_limit;
    int hold_plane;
};

// message returned by bvf_last_error(NULL) for a failed context-free call
void set_context_free_error(const char *msg);

// z-planes per block of the z-marching acoustic kernels for a grid
int default_kchunk(int nx, int ny, int nz);
int default_kchunk_tma(int nx, int ny, int nz, int tile_y = 8);

// Persistent batch kernels: one velocity and one stress launch advance every
// domain of `dom` by one step (the step number is read from *d_step, which a
// third one-thread kernel then increments).  batch_prepare sets the kernels'
// shared-memory limits and returns the persistent grid sizes.
cudaError_t batch_prepare(int L, int h16, int n_mat_max, int *grid_vel, int *grid_str);
cudaError_t launch_batch_step(const BatchParams &bp, int L, int h16, int n_mat_max, int *d_step,
                              int grid_vel, int grid_str, cudaStream_t s);

// kernel launchers (bvf_acoustic.cu / bvf_aux.cu); return cudaGetLastError()
cudaError_t launch_velocity(const AcParams &p, cudaStream_t s);
cudaError_t launch_stress(const AcParams &p, cudaStream_t s);
cudaError_t launch_velocity_tma(const AcParams &p, const VelocityTmaMaps &tm, cudaStream_t s);
cudaError_t launch_stress_tma(const AcParams &p, const StressTmaMaps &tm, cudaStream_t s);
cudaError_t launch_index_max(const uint8_t *idx, size_t n, unsigned *d_out, cudaStream_t s);
cudaError_t launch_pressure(const void *sxx, const void *syy, const void *szz, int h16,
                            float scale, float *out, size_t n, cudaStream_t s);
cudaError_t launch_field_out(const void *f, int h16, size_t stride, float scale, float *out,
                             size_t n, cudaStream_t s);
cudaError_t launch_field_in(const float *in, int h16, size_t stride, float inv_scale, void *f,
                            size_t n, cudaStream_t s);
cudaError_t launch_scale_copy(const float *in, float scale, float *out, size_t n, cudaStream_t s);
cudaError_t launch_fill(float *out, float value, size_t n, cudaStream_t s);
// x[i] += c (round to nearest)
cudaError_t launch_add_const(float *x, float c, size_t n, cudaStream_t s);
cudaError_t launch_amp_phase(const double *C, const double *S, size_t n, int count, double scale,
                             double *amp, double *ph, cudaStream_t s);
cudaError_t launch_rs(const float4 *el, int ne, int nx, int ny, float dx, float zp, float k_over_pi,
                      double pref, float2 *out, cudaStream_t s);
cudaError_t launch_rs_weighted(const float4 *el, const float2 *wt, int ne, int nx, int ny,
                               float dx, float zp, float k_over_pi, double pref, float2 *out,
                               cudaStream_t s);
cudaError_t launch_conj_plane(const double *C, const double *S, size_t n,
                              unsigned long long *d_max, float2 *out, cudaStream_t s);
cudaError_t launch_heat_source(const uint8_t *idx, const ThermCoef *lut, int n_mat,
                               const double *amp, double p_scale, float *Q, size_t n,
                               cudaStream_t s);
// Tensor maps of the TMA-fed BHTE step: the input temperature (40 x 18 x 1
// float box), the material index (64 x 18 x 1 byte box), and the heat
// source, T_max and the FP32 dose partial (32 x 16 x 1 float boxes).
struct ThermTmaMaps {
    CUtensorMap T, idx, Q, Tmax, cemf;
};
// z-planes per block of the BHTE kernels for a grid (tma: the TMA-fed kernel)
int thermal_kchunk(int nx, int ny, int nz, bool tma, int n_mat);
// one BHTE step; tm == NULL takes the direct kernel
cudaError_t launch_thermal_step(const ThParams &p, const ThermTmaMaps *tm, int *flag,
                               cudaStream_t s);
cudaError_t launch_intensity_argmax(const uint8_t *idx, const double *zw, const double *amp,
                                    size_t n, unsigned long long *d_best, cudaStream_t s);
cudaError_t launch_intensity_argmin_index(const uint8_t *idx, const double *zw,
                                          const double *amp, size_t n,
                                          const unsigned long long *d_best,
                                          unsigned long long *d_idx, cudaStream_t s);
cudaError_t launch_plane_sums(const uint8_t *idx_a, const double *za, const double *amp_a,
                              const uint8_t *idx_w, const double *zw, const double *amp_w,
                              int nx, int ny, int nz, const unsigned long long *d_idx,
                              double *d_sums, cudaStream_t s);

}  // namespace bvf
