/*
 * bvf.h -- C ABI of libbvf, a GB300 (sm_103a) implementation of the hot path of
 * the transcranial focused-ultrasound pipeline of arXiv 2301.12727 (BabelBrain):
 *
 *   1. material table -> viscoelastic coefficients (Sec. 2.2 Table 1; Sec. 3.2
 *      Eq. 3, Q = omega / (2 c alpha) with Q = Q0 q_c);
 *   2. Rayleigh-Sommerfeld field of a focused bowl on the entry plane
 *      (Sec. 2.3, last paragraph: elements of area lambda^2/16);
 *   3. viscoelastic velocity-stress FDTD, 4th order in space, 2nd in time, on a
 *      staggered grid (Sec. 2.3, Eq. 1), with standard-linear-solid memory
 *      variables matched to Q, CPML absorbing slabs, a stress source on the
 *      entry plane and running peak-pressure / amplitude-phase capture;
 *   4. Pennes bioheat (BHTE) FDTD with 37 C borders, duty cycle and CEM43 dose
 *      (Sec. 2.4);
 *   5. energy-loss factor E_L over the plane of maximal water intensity and
 *      T_S = sqrt(E_L) (Sec. 2.4, Eq. 2; Sec. 3.2).
 *
 * Conventions shared by every entry point
 *   - Grid: nx * ny * nz cells, spacing dx (m), CPML cells included.  Arrays are
 *     C order with x fastest: idx = (k*ny + j)*nx + i.  Grid point (i,j,k) sits
 *     at (i dx, j dx, k dx).
 *   - Staggering: sxx, syy, szz, p at (i,j,k); vx at (i+1/2,j,k); vy at
 *     (i,j+1/2,k); vz at (i,j,k+1/2); sxy at (i+1/2,j+1/2,k); sxz at
 *     (i+1/2,j,k+1/2); syz at (i,j+1/2,k+1/2).  Stresses and pressure at step n
 *     are at t = n dt, velocities at (n + 1/2) dt.  The last half-grid point of
 *     each axis (position n - 1/2) is a ghost held at zero, and points outside
 *     the array are zero.
 *   - Pointers named d_* are DEVICE memory owned by the caller; h_* are host
 *     memory.  The library never frees caller memory.  A context owns its field,
 *     CPML and capture buffers and frees them in bvf_destroy.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls enqueue work on it and return without waiting unless stated.
 *   - Every call returns an int status: BVF_OK (0) or a negative BVF_E_* code.
 *     Argument and material validation happens on the host, synchronously,
 *     before anything is enqueued.  No exception or device trap crosses the ABI.
 *     bvf_last_error() gives a one-line description of the last failure.
 */
#ifndef BVF_H
#define BVF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BVF_VERSION 3

#define BVF_OK 0
#define BVF_E_ARG (-1)        /* NULL pointer, bad size, bad option, call order */
#define BVF_E_CFL (-2)        /* dt above the O(4) 3-D stability limit           */
#define BVF_E_MATERIAL (-3)   /* unphysical material, Q out of reach, bad index  */
#define BVF_E_NOMEM (-4)      /* device allocation failed                        */
#define BVF_E_CUDA (-5)       /* a CUDA runtime call failed                      */
#define BVF_E_UNSTABLE (-6)   /* a non-finite pressure was detected              */
#define BVF_E_TIMEOUT (-7)    /* the call's wall-clock budget was spent          */

#define BVF_ENV_NONE 0        /* no source                                       */
#define BVF_ENV_BURST 1       /* rectangular burst of n_cycles                   */
#define BVF_ENV_RAMP_CW 2     /* one-cycle raised-cosine ramp, then CW           */

#define BVF_MAX_MATERIALS 256
#define BVF_MAX_SLS 4

/* Field ids for bvf_get_field / bvf_set_field.  Memory variable of mechanism l
 * for stress component c (0 xx, 1 yy, 2 zz, 3 xy, 4 xz, 5 yz) has id
 * BVF_FIELD_MEM0 + 6*l + c. */
enum {
    BVF_FIELD_VX = 0, BVF_FIELD_VY, BVF_FIELD_VZ,
    BVF_FIELD_SXX, BVF_FIELD_SYY, BVF_FIELD_SZZ,
    BVF_FIELD_SXY, BVF_FIELD_SXZ, BVF_FIELD_SYZ,
    BVF_FIELD_MEM0
};

typedef struct bvf_ctx bvf_ctx;

/* Grid and time step (Sec. 2.2: resolution from frequency and points per
 * wavelength; Sec. 2.3: time step).  n_pml CPML cells on every face
 * (0 = closed box with zero ghosts); pml_R is the CPML's nominal normal-incidence
 * reflection (e.g. 1e-4).  Requires nx, ny, nz >= 2 n_pml + 2. */
typedef struct {
    int nx, ny, nz;
    double dx;        /* m */
    double dt;        /* s */
    int n_pml;
    double pml_R;
} bvf_grid;

/* One row of the property table (Sec. 2.2, Table 1).  Attenuations are in Np/m
 * at the drive frequency.  Thermal constants feed the BHTE (Sec. 2.4):
 * conductivity k_th (W/m/K), specific heat c_th (J/kg/K), blood perfusion
 * rate perf (1/s), and the fraction heat_frac of alphaL turned into heat
 * (0.16 for bone in the paper). */
typedef struct {
    double rho, cL, cS, alphaL, alphaS;
    double k_th, c_th, perf, heat_frac;
} bvf_material;

/* Drive frequency f0 (Hz), attenuation correction q_c (Q = Q0 q_c, Sec. 3.2)
 * and number of SLS mechanisms (0 .. BVF_MAX_SLS; 0 = lossless).
 *
 * storage selects how the acoustic state (velocities, stresses, memory
 * variables) is held between steps; the arithmetic is FP32 either way.
 * BVF_STORAGE_F16 halves the state's bytes: stresses are stored as
 * sigma / p_ref, velocities as v rho_w c_w / p_ref (rho_w c_w = 1.5e6 Pa s/m),
 * memory variables in matching units, each rounded to FP16.  p_ref (Pa, 0 =
 * 1e5) should be near the largest pressure expected; FP16 keeps 11
 * significant bits from 6e-5 p_ref to 6.5e4 p_ref.  Every accessor returns
 * and takes physical units in FP32/FP64 regardless of storage.  FP16 storage
 * is an extension beyond the paper, whose solvers run in FP32. */
enum { BVF_STORAGE_F32 = 0, BVF_STORAGE_F16 = 1 };
typedef struct {
    double f0;
    double qc;
    int n_sls;
    int storage;
    double p_ref;
} bvf_physics;

/* Single-element spherical bowl (Sec. 2, "Single"): aperture diameter and
 * radius of curvature (m), apex position (m, grid frame) and unit acoustic
 * axis.  p0 = rho0 c0 u0 is the surface pressure (Pa); c0 the coupling
 * medium's speed (water).  ds_over_lambda sets the element size (0.25 gives
 * the paper's lambda^2/16 area; 0 selects 0.25). */
typedef struct {
    double aperture, roc;
    double apex[3];
    double dir[3];
    double p0;
    double c0;
    double ds_over_lambda;
} bvf_bowl;

/* Capture window, counted in completed steps (step s holds p at t = s dt).
 * peak_from: first step entering the max |p| map (negative = off).
 * dft_start, dft_steps: steps entering C += p cos(w t), S += p sin(w t) in FP64
 * (dft_steps = 0: off).  dft_steps should span whole periods. */
typedef struct {
    int peak_from;
    int dft_start;
    int dft_steps;
} bvf_capture;

/* BHTE regime (Sec. 2.4; Sec. 4.1.1: 40 s on at 30 % duty cycle, 80 s off).
 * dt (s) must satisfy dt <= dx^2 min(rho c_th / k_th) / 6.  n_on steps with
 * the time-averaged source duty * Q, then n_off steps with none.  T_a is the
 * initial, border and arterial temperature (37 C).  rhob_cb is the blood's
 * volumetric heat capacity (J/m^3/K).  The heat source is
 * Q = heat_frac * alphaL * (p_scale * amp)^2 / (rho cL). */
typedef struct {
    double dt;
    int n_on, n_off;
    double duty;
    double T_a;
    double rhob_cb;
    double p_scale;
} bvf_thermal;

/* Device time of the acoustic kernels, from CUDA events recorded around each
 * launch on the launching stream while timing is enabled. */
typedef struct {
    long long velocity_launches, stress_launches;
    double velocity_ms, stress_ms;   /* summed event durations */
} bvf_kernel_times;

/* Counters of one context. */
typedef struct {
    long long steps;             /* acoustic steps advanced since creation/reset */
    long long kernel_launches;   /* kernels this context enqueued (all calls)    */
    long long thermal_steps;
    double courant;              /* c_max(unrelaxed) dt / dx of the material set */
    double bytes_per_voxel_step; /* algorithmic bytes of one acoustic step       */
} bvf_stats;

/* ---- library ---------------------------------------------------------- */

/* BVF_VERSION of the loaded library. */
int bvf_version(void);

/* Stability limit of the O(4) staggered leapfrog in 3-D (Sec. 2.3 scheme):
 * c dt / dx <= 6 / (7 sqrt 3). */
double bvf_courant_limit(void);

/* Text for a status code (static storage). */
const char *bvf_strerror(int code);

/* ---- context ------------------------------------------------------------ */

/* Allocate a context and its device state (fields, memory variables, CPML
 * slabs, peak map) on the current device, all zero.  Errors: BVF_E_ARG for
 * bad sizes or options, BVF_E_NOMEM.  *out is NULL on failure. */
int bvf_create(const bvf_grid *grid, const bvf_physics *phys, bvf_ctx **out);

/* Release everything the context owns (NULL is accepted). */
void bvf_destroy(bvf_ctx *ctx);

/* Description of the last failure on this context (or of the last failed
 * bvf_create / context-free call when ctx is NULL). */
const char *bvf_last_error(const bvf_ctx *ctx);

/* Material-index volume and property table (Sec. 2.2; Table 1).
 * d_index: nx*ny*nz uint8 on the device (copied; the caller may free it after
 * the call returns).  h_table: n_mat rows (copied).  Derives per material the
 * relaxed moduli and SLS strengths matched to Q = q_c w / (2 c alpha) at f0,
 * the CPML profile, and checks: rho > 0, cL > 0, 0 <= cS, Poisson ratio in
 * [-1, 0.5] (Sec. 3.2), Q reachable by the mechanisms, every index < n_mat
 * (a synchronous device scan), and the CFL limit against the fastest unrelaxed
 * wave speed.  Errors: BVF_E_ARG, BVF_E_MATERIAL, BVF_E_CFL, BVF_E_CUDA. */
int bvf_set_materials(bvf_ctx *ctx, const uint8_t *d_index, const bvf_material *h_table,
                      int n_mat);

/* Rayleigh-Sommerfeld incident field of a bowl on the plane z = z_plane
 * (Sec. 2.3, last paragraph):  p = (i k p0 / 2 pi) sum_e dA_e exp(-i k r_e) / r_e
 * over elements of size ds_over_lambda * lambda in water (c0).  Output d_out:
 * nx*ny complex values as interleaved float pairs (re, im), x fastest, grid
 * point (i,j) at (i dx, j dx).  Every element must lie below the plane
 * (z < z_plane); otherwise BVF_E_ARG.  Context-free; asynchronous on `stream`. */
int bvf_rs_plane(const bvf_bowl *bowl, int nx, int ny, double dx, double z_plane, double f0,
                 float *d_out, void *stream);

/* Source on plane k_plane (Sec. 2.3: the incident field forward-propagated as
 * a stress source perpendicular to the acoustic axis).  d_plane holds nx*ny
 * complex amplitudes A e^{i phi} (interleaved float pairs, copied).  At the
 * update from step n to n+1 every normal stress of the plane receives
 * -(2 c0 dt / dx) * env(t) * A sin(w t + phi), t = (n + 1/2) dt, with env given
 * by `envelope` (BVF_ENV_*) and n_cycles for bursts.  Errors: BVF_E_ARG. */
int bvf_set_source(bvf_ctx *ctx, int k_plane, const float *d_plane, double c0, int envelope,
                   int n_cycles, void *stream);

/* Zero the fields, memory variables, CPML memories, captures and step count. */
int bvf_reset(bvf_ctx *ctx, void *stream);

/* Advance n_steps acoustic steps (velocity, then stress + memory variables +
 * source + capture per step) on `stream`.  Requires bvf_set_materials.  The
 * capture window (NULL = none) refers to the context's absolute step count.
 * Non-finite pressure sets a device flag reported by bvf_synchronize.  With a
 * time budget (bvf_set_time_budget) the call may return BVF_E_TIMEOUT after
 * fewer steps, having waited for them (bvf_get_stats gives the count). */
int bvf_run_acoustic(bvf_ctx *ctx, int n_steps, const bvf_capture *cap, void *stream);

/* Tiles of the TMA-fed acoustic kernels (no counterpart in the paper: how the
 * grid is cut into blocks, which changes no result, bit for bit).  A block
 * owns an x-y tile 32 voxels wide and stress_rows (stress kernel) or
 * velocity_rows (velocity kernel) rows high, 4, 8 or 16, and marches kchunk
 * z-planes.  0 selects the default: 8 rows for the stress and 16 for the
 * velocity kernel, and a z-chunk that fills the GPU about six times.  Heights
 * other than 8 apply to contexts with two SLS mechanisms (n_sls = 2, the
 * method's); other contexts use 8.  bvf_set_tile keeps the choice for later
 * bvf_run_acoustic calls; bvf_get_tile reports the heights and the stress
 * kernel's z-chunk the kernels use.  Errors: BVF_E_ARG. */
typedef struct bvf_tile {
    int stress_rows;
    int velocity_rows;
    int kchunk;
} bvf_tile;
int bvf_set_tile(bvf_ctx *ctx, const bvf_tile *tile);
int bvf_get_tile(const bvf_ctx *ctx, bvf_tile *out);

/* Wall-clock budget (seconds, 0 = none, the default) of each later
 * bvf_run_acoustic and bvf_run_thermal call on this context: failure
 * detection for planning services, which must not wait without bound on one
 * plan (the paper's pipeline runs each step to completion).  Every 32 steps
 * the call compares the time since it began with the budget, keeping at most
 * two such chunks queued ahead of the host; once the budget is spent it waits
 * for the queued steps and returns BVF_E_TIMEOUT.  The context then holds the
 * state after every step that ran (consistent and resumable: a later call
 * continues from it; an acoustic run continues bit for bit, a thermal run to
 * within one FP32 rounding of T at the stop, since the call hands T back in
 * C, see bvf_run_thermal).  Work already on the GPU is never cancelled, so a
 * call can overrun its budget by up to two chunks of steps. */
int bvf_set_time_budget(bvf_ctx *ctx, double seconds);

/* Wait for `stream` and report: BVF_E_UNSTABLE if a non-finite pressure was
 * seen since the last reset; BVF_E_CUDA on an asynchronous CUDA error, or when
 * a TMA copy of an acoustic kernel did not complete within its wait bound
 * (the blocks concerned stop after draining the copies they issued; their
 * results are incomplete, the context stays usable, and bvf_reset clears the
 * report). */
int bvf_synchronize(bvf_ctx *ctx, void *stream);

/* Size in bytes of a snapshot of the context's acoustic state. */
int bvf_state_bytes(const bvf_ctx *ctx, size_t *out);

/* Snapshot of everything an acoustic run continues from: the velocities,
 * stresses and memory variables, the CPML memories, the peak map, the FP64 DFT
 * sums, the step counter, the number of captured DFT steps and the
 * non-finite / time-out flag (checkpoint and resume of a long run; the paper
 * runs each simulation in one go).  Not included: materials, source and
 * capture settings, which the caller sets again before loading.  d_buf: device
 * memory of at least bvf_state_bytes bytes, caller-owned; the layout is a
 * 256-byte header (library version, grid, time step, frequency, SLS count,
 * storage, counters) then the arrays.  bvf_state_save is stream-ordered and
 * asynchronous.  bvf_state_load first waits for `stream` to read the header,
 * rejects (BVF_E_ARG) a snapshot of another library version, grid, time step,
 * frequency, SLS count or storage, then enqueues the copies; a run continued
 * from a loaded snapshot equals the uninterrupted run bit for bit. */
int bvf_state_save(bvf_ctx *ctx, void *d_buf, size_t bytes, void *stream);
int bvf_state_load(bvf_ctx *ctx, const void *d_buf, size_t bytes, void *stream);

/* Test hook of the bounded TMA waits (the paper has no counterpart).  Arms the
 * next acoustic step so that `kernel` (1 = velocity, 2 = stress) of the
 * TMA-fed pair arms the mbarrier of the look-ahead copies it would issue at
 * plane `plane` of its z-chunk but issues none of them, or (kernel = 3) the
 * first step of the next bvf_run_thermal so that the TMA-fed BHTE kernel arms
 * plane `plane`'s barrier but issues none of its copies; the waits for that
 * data then run out after wait_limit polls (0: the library's bound of 2^22).
 * The blocks concerned stop after draining every copy they did issue, so no
 * copy is left in flight, and bvf_synchronize reports BVF_E_CUDA; after
 * bvf_reset the context runs normally.  kernel = 0 disarms.  BVF_E_ARG if the
 * context does not use that TMA-fed kernel (nx % 8 != 0, or more than 2 SLS
 * mechanisms for kernels 1 and 2) or the plane is outside the grid. */
int bvf_test_withhold_copy(bvf_ctx *ctx, int kernel, int plane, unsigned wait_limit);

/* Copy one state array (BVF_FIELD_* id, nx*ny*nz floats) out of / into the
 * context.  Used to start from a prescribed state and to inspect every field. */
int bvf_get_field(bvf_ctx *ctx, int which, float *d_out, void *stream);
int bvf_set_field(bvf_ctx *ctx, int which, const float *d_in, void *stream);

/* p = -(sxx + syy + szz)/3 at the current step (nx*ny*nz floats). */
int bvf_get_pressure(bvf_ctx *ctx, float *d_out, void *stream);

/* Running max |p| map (nx*ny*nz floats). */
int bvf_get_peak(bvf_ctx *ctx, float *d_out, void *stream);

/* Amplitude 2 sqrt(C^2 + S^2) / N and phase atan2(-S, C) from the FP64 DFT
 * sums of the capture window (N = steps captured so far), nx*ny*nz doubles
 * each; either pointer may be NULL.  BVF_E_ARG if nothing was captured. */
int bvf_get_amp_phase(bvf_ctx *ctx, double *d_amp, double *d_phase, void *stream);

/* Pennes BHTE + CEM43 (Sec. 2.4) on the context's grid and materials:
 * rho c_th dT/dt = div(k grad T) - perf rhob_cb (T - T_a) + Q, forward Euler,
 * 7-point stencil with harmonic-mean face conductivity, border voxels at T_a.
 * d_amp: nx*ny*nz pressure amplitudes (Pa, FP64, e.g. from bvf_get_amp_phase;
 * NULL = no heating).  d_T (in/out, float) holds the starting temperature and
 * receives the final one; d_Tmax (in/out, float) and d_cem43 (in/out, FP64)
 * accumulate max T and sum dt/60 R^(43-T) (R = 0.5 at T >= 43, else 0.25) after
 * every step (the dose increments of up to 32 consecutive steps are summed in
 * FP32 before each addition to the FP64 dose).  The kernels advance the rise
 * T - T_a in FP32 (finer than T near 37 C by about 2^10); d_T and d_Tmax are
 * converted on entry and back on exit, one FP32 rounding each.  Errors:
 * BVF_E_ARG (including dt above the explicit limit). */
int bvf_run_thermal(bvf_ctx *ctx, const bvf_thermal *th, const double *d_amp, float *d_T,
                    float *d_Tmax, double *d_cem43, void *stream);

/* Energy-loss factor (Sec. 2.4, Eq. 2): with I = A^2 / (2 rho cL) per voxel,
 * z_m is the plane of the largest water-run intensity (ties: lowest linear
 * index) and E_L = sum_xy I_a(z_m) / sum_xy I_w(z_m); T_S = sqrt(E_L)
 * (Sec. 3.2).  h_Iw_max receives the largest water-run intensity (W/m^2), the
 * reference for I_SPPA scaling (Sec. 2.4).  Index volumes and amplitude maps
 * are device arrays of nx*ny*nz; tables are host rows; any h_* output may be
 * NULL.  Synchronous: waits for `stream`. */
int bvf_transmission(int nx, int ny, int nz,
                     const uint8_t *d_idx_a, const bvf_material *h_mat_a, int n_a,
                     const double *d_amp_a,
                     const uint8_t *d_idx_w, const bvf_material *h_mat_w, int n_w,
                     const double *d_amp_w,
                     double *h_EL, double *h_TS, int *h_zm, double *h_Iw_max,
                     void *stream);

/* bvf_transmission without any device allocation (the paper has no
 * counterpart: this serves callers that cannot allocate device memory when
 * they need E_L, e.g. because their own pool already reserves the GPU's memory
 * or an allocation would stall a latency-bound loop).  Same arguments,
 * results and errors as bvf_transmission; each table may hold at most
 * BVF_MAX_MATERIALS rows (BVF_E_ARG beyond that).  Its temporaries live in one
 * fixed array of about 4 KiB inside the library, present on every GPU that
 * loads it until the process exits; each call looks up that array's address
 * on the current device.  All calls share the array: calls that overlap on
 * the GPU (e.g. unordered streams) race.  Synchronous: copies the tables from
 * host memory and waits for `stream` before returning. */
int bvf_transmission_noalloc(int nx, int ny, int nz,
                             const uint8_t *d_idx_a, const bvf_material *h_mat_a, int n_a,
                             const double *d_amp_a,
                             const uint8_t *d_idx_w, const bvf_material *h_mat_w, int n_w,
                             const double *d_amp_w,
                             double *h_EL, double *h_TS, int *h_zm, double *h_Iw_max,
                             void *stream);

/* Counters (host struct filled synchronously). */
int bvf_get_stats(const bvf_ctx *ctx, bvf_stats *out);

/* Enable (1) or disable (0) per-launch CUDA-event timing of the acoustic
 * kernels; enabling clears the accumulated times. */
int bvf_kernel_timing(bvf_ctx *ctx, int enable);

/* Wait for the recorded events and return the accumulated kernel times since
 * timing was enabled. */
int bvf_get_kernel_times(bvf_ctx *ctx, bvf_kernel_times *out);

/* Rayleigh-Sommerfeld field of a phased array given as elements (the paper's
 * devices are single bowls; multi-element layouts serve steering and
 * time-reversal refocusing):  p = (i k p0 / 2 pi) sum_e w_e dA_e exp(-i k r_e) / r_e
 * on the plane z = z_plane.  h_elem: ne rows of six doubles on the host,
 * (x, y, z, area, w_re, w_im) in metres, square metres and the complex weight
 * (1 + 0i for an unsteered element).  c0: coupling-medium speed.  Output as
 * bvf_rs_plane.  Every element must lie below the plane; ne >= 1.
 * Context-free; asynchronous on `stream` (the elements are copied first). */
int bvf_rs_elements(const double *h_elem, int ne, double p0, double c0, int nx, int ny,
                    double dx, double z_plane, double f0, float *d_out, void *stream);

/* Elements of a spherical cap for bvf_rs_elements: aperture, radius of
 * curvature, apex and axis from `bowl` (its other fields are unused); ring r
 * of n_rings rings of equal polar-angle width holds n_inner (r + 1) equal
 * elements, each carrying the area of its patch of the cap, weight 1 + 0i.
 * h_elem: NULL to count only, else room for the count (rows of six doubles as
 * in bvf_rs_elements); *n_out receives the count.  Host only, synchronous. */
int bvf_bowl_array(const bvf_bowl *bowl, int n_rings, int n_inner, double *h_elem, int *n_out);

/* Steering weights (geometric focusing of a phased array on a target, in a
 * medium of speed c0): w_e = exp(+i k r_e), k = 2 pi f0 / c0, r_e the distance
 * from element e to `target` (three doubles, metres), written into columns 4
 * and 5 of the ne rows of h_elem, so every element's wave reaches the target
 * in phase.  Host only, synchronous. */
int bvf_steer_weights(double *h_elem, int ne, const double *target, double f0, double c0);

/* Time-reversal (phase-conjugation) source plane through the context's medium
 * (aberration correction for transcranial focusing, Sec. 2.3 source plane): a
 * CW point source (one-cycle ramp) of unit amplitude at voxel (ti, tj, tk)
 * runs n_steps steps; the FP64 complex amplitude P it leaves on plane k_src
 * over the last two periods is captured, and conj(P) / max|P| is written to
 * d_plane (nx*ny complex values as interleaved float pairs, caller-owned
 * device memory), ready for bvf_set_source.  The context's state and capture
 * are reset before and after, and its source is cleared.  Needs n_steps > two
 * periods.  Synchronous: waits for `stream`. */
int bvf_time_reversal_plane(bvf_ctx *ctx, int ti, int tj, int tk, int k_src, int n_steps,
                            double c0, float *d_plane, void *stream);

/* ---- one placement end to end --------------------------------------------
 * The paper's transcranial and thermal steps for one transducer placement
 * (Sec. 2.3, 2.4): materials of the skull run; Rayleigh-Sommerfeld field of
 * the bowl on source plane k_src; the FDTD through the skull and the same FDTD
 * in water only (ramped CW source, peak map from step 1, FP64 amplitude over
 * the capture window); E_L and T_S on the plane of maximal water intensity
 * (Eq. 2); the skull field scaled to the requested brain intensity,
 * p_scale = sqrt(I_SPPA / (E_L I_w,max)); the BHTE with CEM43 from T_a. */
typedef struct {
    int n_steps;                 /* FDTD steps of each run */
    int dft_start, dft_steps;    /* amplitude window, whole periods (see bvf_capture) */
    double i_sppa;               /* requested brain I_SPPA (W/m^2); <= 0 selects 5e4 */
    bvf_thermal thermal;         /* regime; its p_scale is ignored (computed) */
    int serial;                  /* 0: the water run on a second stream of the skull
                                    context, concurrent with the skull run; 1: both
                                    on `stream`, one after the other */
} bvf_plan_params;

typedef struct {
    double EL, TS;               /* energy-loss factor and its square root */
    double Iw_max;               /* largest water-run intensity (W/m^2) */
    double p_scale;              /* factor applied to the skull amplitude */
    int z_m;                     /* plane of the largest water intensity */
} bvf_plan_result;

/* skull, water: two contexts on the same grid (the water context's materials
 * are set here to the one row h_water with an all-zero index).  The two FDTD
 * runs are independent: by default the water run goes to a second stream
 * (owned by the skull context) forked from and joined back into `stream`, so
 * their kernels share the GPU; results are bit for bit those of the serial
 * order.  d_index
 * (nx*ny*nz bytes) and h_table/n_mat: the skull run's material volume and
 * table.  Outputs, caller-owned device buffers of nx*ny*nz elements: d_peak
 * (float, max |p| of the skull run), d_amp (FP64 skull amplitude at the drive
 * level of the bowl's p0, before scaling), d_T, d_Tmax (float) and d_cem43
 * (FP64) of the thermal step; *out on the host.  Synchronous (returns after
 * the stream has finished).  Errors as the calls it makes. */
int bvf_plan(bvf_ctx *skull, bvf_ctx *water, const uint8_t *d_index, const bvf_material *h_table,
             int n_mat, const bvf_material *h_water, const bvf_bowl *bowl, int k_src,
             const bvf_plan_params *pp, float *d_peak, double *d_amp, float *d_T, float *d_Tmax,
             double *d_cem43, bvf_plan_result *out, void *stream);

/* bvf_plan with host buffers (no counterpart in the paper: the call a planning
 * service makes per placement).  h_index (nx*ny*nz bytes) is copied to the
 * skull context's device staging on `stream`, the plan runs as bvf_plan, and
 * the peak map, the final temperature (h_T, may be NULL), T_max and CEM43 are
 * copied back into the caller's host buffers before the call returns.  Host
 * buffers should be page-locked (cudaHostAlloc / cudaHostRegister) for the
 * copies to run at full speed.  The staging (29 bytes per voxel) is allocated
 * on the first call and owned by the skull context.  Errors as bvf_plan. */
int bvf_plan_host(bvf_ctx *skull, bvf_ctx *water, const uint8_t *h_index,
                  const bvf_material *h_table, int n_mat, const bvf_material *h_water,
                  const bvf_bowl *bowl, int k_src, const bvf_plan_params *pp, float *h_peak,
                  float *h_T, float *h_Tmax, double *h_cem43, bvf_plan_result *out, void *stream);

/* ---- batched planning sweeps -------------------------------------------
 * Several contexts (different grids, materials, sources, frequencies; the
 * paper repeats its acoustic step for each transducer placement, Sec. 2.3)
 * advanced in lockstep.  Each step is two persistent launches that share the
 * GPU among all domains: one velocity and one stress kernel over a work list
 * of (domain, 32 x 8 tile, z-chunk) items, plus a one-thread kernel advancing
 * the step counter the kernels read.  Results are those of bvf_run_acoustic
 * on each context, bit for bit.  The paper has no counterpart of this call;
 * it serves sweeps over placements and frequencies.
 *
 * bvf_batch_create: the contexts stay owned by the caller and must outlive
 * the batch; each needs its materials set, nx % 8 == 0 and at most 2 SLS
 * mechanisms, and all share the SLS count and storage type (BVF_E_ARG
 * otherwise).  Sources are taken from the contexts at each run. */
typedef struct bvf_batch bvf_batch;
int bvf_batch_create(bvf_ctx *const *ctxs, int n, bvf_batch **out);
void bvf_batch_destroy(bvf_batch *b);

/* Advance context d by n_steps[d] steps (lockstep; a domain whose count is
 * reached is skipped by later steps), with capture windows caps[d] (NULL: no
 * capture for any domain).  kchunk: z-planes per work item for every domain
 * (0: each context's default).  graph_steps > 0 captures that many steps in
 * a CUDA graph and replays it (launch overhead of one graph per graph_steps
 * steps); 0 launches the kernels directly.  Asynchronous on `stream`;
 * bvf_synchronize on each context reports its errors. */
int bvf_batch_run(bvf_batch *b, const int *n_steps, const bvf_capture *caps, int kchunk,
                  int graph_steps, void *stream);

/* The same sweep as separate per-context launches (bvf_run_acoustic) spread
 * over n_streams streams of the batch: contexts dealt round-robin, each
 * stream running its contexts one after another, so kernels of different
 * domains overlap (the stream-level alternative to the persistent batch
 * kernels).  Forks from and joins back into `stream`. */
int bvf_batch_run_streams(bvf_batch *b, const int *n_steps, const bvf_capture *caps,
                          int n_streams, void *stream);

/* The same sweep as one CUDA graph: the per-context launches of
 * bvf_run_acoustic, contexts dealt round-robin over n_branches parallel
 * branches (as bvf_batch_run_streams deals them over streams), recorded once
 * and replayed with a single graph launch on `stream`, so the host issues one
 * launch per sweep and the branches' kernels share the GPU.  The recording is
 * kept and replayed while the call's arguments, the contexts' tiles and
 * the step counts the contexts start from are those it was recorded for
 * (e.g. the same sweep after bvf_reset); anything else records anew, which
 * waits for `stream`.  Results are those of bvf_run_acoustic, bit for bit.
 * Contexts with a time budget, kernel timing or the test hook armed are
 * refused (BVF_E_ARG). */
int bvf_batch_run_graph(bvf_batch *b, const int *n_steps, const bvf_capture *caps, int n_branches,
                        void *stream);

/* Per-domain tile autotuner: for every context, times trial_steps steps (after
 * two warm-up steps) with each candidate tile (bvf_tile: rows of the stress
 * and velocity kernels' x-y tiles and z-planes per block; candidates with a
 * height other than 0 or 8 are skipped for contexts without two SLS
 * mechanisms), keeps the fastest in the context (as bvf_set_tile; used by
 * bvf_run_acoustic and the run modes above) and writes it to h_best[d] (may
 * be NULL).  Leaves every context reset (bvf_reset).  Errors: BVF_E_ARG (a
 * height other than 0, 4, 8, 16 or a negative z-chunk). */
int bvf_batch_tune_domains(bvf_batch *b, int trial_steps, const bvf_tile *candidates,
                           int n_candidates, bvf_tile *h_best, void *stream);

/* Tile autotuner of the graph mode: the same tile for every context, chosen
 * by timing, for each candidate, a replay of bvf_batch_run_graph (trial_steps
 * steps per context, no capture, n_branches branches) after one recording
 * replay; the domains then share the GPU, so the fastest tile under
 * concurrency differs from the one each domain prefers alone
 * (bvf_batch_tune_domains).  Keeps the fastest in every context, writes it to
 * *h_best and its time per step (ms) to *h_ms (may be NULL), and leaves every
 * context reset.  Errors: BVF_E_ARG. */
int bvf_batch_tune_graph(bvf_batch *b, int trial_steps, const bvf_tile *candidates,
                         int n_candidates, int n_branches, bvf_tile *h_best, double *h_ms,
                         void *stream);

/* Tile autotuner: times trial_steps steps of every domain for each candidate
 * z-chunk length, returns the fastest and its time per step (ms), and leaves
 * every context reset (bvf_reset: state, captures and step counts zeroed). */
int bvf_batch_tune(bvf_batch *b, int trial_steps, const int *candidates, int n_candidates,
                   int *best_kchunk, double *best_ms_per_step, void *stream);

/* Kernel launches enqueued by this batch so far (3 per step). */
int bvf_batch_launches(const bvf_batch *b, long long *out);

#ifdef __cplusplus
}
#endif

#endif /* BVF_H */
