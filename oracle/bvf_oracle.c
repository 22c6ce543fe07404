/*
 * bvf_oracle.c -- plain FP64 CPU oracle for the transcranial FDTD + BHTE hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The product
 * (libbvf, CUDA) never links, includes or calls anything here, and nothing here
 * includes a product header.
 *
 * Everything is written for clarity, in the order the method states its steps,
 * in double precision, with no blocking, fusion or reordering.  The only
 * parallelism is an OpenMP split of the outermost (z) loop of each sweep, which
 * leaves the arithmetic of every voxel unchanged.
 *
 * Method (arXiv 2301.12727, BabelBrain):
 *   - Sec. 2.3, Eq. 1: isotropic velocity-stress system; 4th-order-space /
 *     2nd-order-time staggered-grid FDTD (Levander; Virieux staggering; Bohlen's
 *     3D viscoelastic formulation).
 *   - Sec. 3.2 "Modeling", Eq. 3: Q = omega / (2 c alpha), with the correction
 *     Q = Q0 * q_c; relaxation constants and memory variables fitted to Q.
 *   - Sec. 2.3 (last paragraph): transducer split into elements of area
 *     lambda^2/16, Rayleigh-Sommerfeld onto the entry plane, forward-propagated
 *     as a stress source perpendicular to the acoustic axis.
 *   - Sec. 2.4: BHTE by FDTD, 37 C borders, duty cycle, 0.16 of the skull
 *     attenuation turned into heat, thermal dose; Eq. 2 energy-loss factor E_L.
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   grid points outside the array are zero (two ghost layers); the last
 *   half-grid point of each axis (position n - 1/2) is a ghost held at zero;
 *   buoyancy at a velocity point = 2 / (rho_a + rho_b); mu at a shear point =
 *   harmonic mean over its four cells (0 if any is 0); tau_S there = arithmetic
 *   mean; pairwise sums (a00 + a10) + (a01 + a11) keep mirror symmetry exact;
 *   SLS relaxation frequencies log-spaced over [f0/3, 3 f0]; single-frequency
 *   tau fit; relaxed moduli chosen so the phase speed at f0 equals c; CPML of
 *   Komatitsch-Martin form with kappa = 1, d = d0 xi^2, alpha = pi f0 (1 - xi);
 *   soft pressure-type stress source scaled by 2 c0 dt / dx and sampled at
 *   t = (n + 1/2) dt; DFT capture p cos / p sin at t = (n + 1) dt.
 *
 * Array layout: C order, x fastest, idx = (k*ny + j)*nx + i.
 * Staggering:  sxx,syy,szz at (i,j,k); vx at (i+1/2,j,k); vy at (i,j+1/2,k);
 *              vz at (i,j,k+1/2); sxy at (i+1/2,j+1/2,k); sxz at (i+1/2,j,k+1/2);
 *              syz at (i,j+1/2,k+1/2).  Memory variables sit with their stress.
 * State array: [NF][nz][ny][nx], NF = 9 + 6 L + 18:
 *   0 vx, 1 vy, 2 vz, 3 sxx, 4 syy, 5 szz, 6 sxy, 7 sxz, 8 syz,
 *   9 + 6 l + c : memory variable of mechanism l for stress component c
 *                 (c = 0 xx, 1 yy, 2 zz, 3 xy, 4 xz, 5 yz),
 *   9 + 6 L + q : CPML memory psi_q (q = 0..17, order given at PSI_* below).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define ORC_OK 0
#define ORC_E_ARG (-1)
#define ORC_E_CFL (-2)
#define ORC_E_MATERIAL (-3)

/* Levander 4th-order staggered coefficients (Sec. 2.3). */
static const double C1 = 9.0 / 8.0;
static const double C2 = -1.0 / 24.0;

typedef struct {
    int nx, ny, nz;
    double dx, dt;
    int n_pml;
    double pml_R;
    double f0, qc;
    int n_sls;
} orc_grid;

/* material row: rho, cL, cS, alphaL, alphaS, k_th, c_th, perf, heat_frac */
enum { M_RHO, M_CL, M_CS, M_AL, M_AS, M_K, M_CTH, M_PERF, M_HEAT, M_NCOL };

/* per-material derived coefficients */
enum { K_PI, K_MU, K_TAUP, K_TAUS, K_NCOL };

/* CPML memory slots: derivative (field, axis) used by one update */
enum {
    PSI_VX_X, PSI_VX_Y, PSI_VX_Z,   /* d/dx sxx, d/dy sxy, d/dz sxz  (vx) */
    PSI_VY_X, PSI_VY_Y, PSI_VY_Z,   /* d/dx sxy, d/dy syy, d/dz syz  (vy) */
    PSI_VZ_X, PSI_VZ_Y, PSI_VZ_Z,   /* d/dx sxz, d/dy syz, d/dz szz  (vz) */
    PSI_EXX, PSI_EYY, PSI_EZZ,      /* d/dx vx, d/dy vy, d/dz vz     (normal) */
    PSI_XY_Y, PSI_XY_X,             /* d/dy vx, d/dx vy              (sxy) */
    PSI_XZ_Z, PSI_XZ_X,             /* d/dz vx, d/dx vz              (sxz) */
    PSI_YZ_Z, PSI_YZ_Y,             /* d/dz vy, d/dy vz              (syz) */
    PSI_N
};

int orc_n_fields(int n_sls) { return 9 + 6 * n_sls + PSI_N; }

/* ------------------------------------------------------------------------ */
/* Sec. 3.2, Eq. 3 and the q_c correction: SLS relaxation times and fit.      */
/* ------------------------------------------------------------------------ */

/* Relaxation times tau_sigma_l = 1 / (2 pi f_l), f_l log-spaced on [f0/3, 3 f0]
 * (f0 itself when L = 1).  The paper only says relaxation constants are
 * optimised to match Q; this placement brackets the drive frequency. */
void orc_relaxation_times(double f0, int L, double *tau_sigma)
{
    for (int l = 0; l < L; ++l) {
        double e = (L == 1) ? 0.0 : -1.0 + 2.0 * (double)l / (double)(L - 1);
        double fl = f0 * pow(3.0, e);
        tau_sigma[l] = 1.0 / (2.0 * M_PI * fl);
    }
}

/* One propagation mode (P or S) of one material.  Q = qc * w / (2 c alpha)
 * (Eq. 3 with Q = Q0 q_c).  The tau-method quality factor of L standard linear
 * solids is Q(w) = (1 + tau B) / (tau A), A = sum w ts/(1+w^2 ts^2),
 * B = sum w^2 ts^2/(1+w^2 ts^2); solving Q(w0) = Q gives tau = 1 / (Q A - B).
 * The relaxed modulus M_R makes the phase speed at f0 equal to c:
 * M_R = rho c^2 [Re (m^-1/2)]^2 with m = 1 + tau sum i w ts / (1 + i w ts). */
static int fit_mode(double rho, double c, double alpha, double f0, double qc,
                    int L, const double *ts, double *M_R, double *tau)
{
    if (c == 0.0) { *M_R = 0.0; *tau = 0.0; return ORC_OK; }
    if (alpha <= 0.0 || L == 0) { *M_R = rho * c * c; *tau = 0.0; return ORC_OK; }
    double w = 2.0 * M_PI * f0;
    double Q = qc * w / (2.0 * c * alpha);
    double A = 0.0, B = 0.0;
    for (int l = 0; l < L; ++l) {
        double x = w * ts[l];
        A += x / (1.0 + x * x);
        B += x * x / (1.0 + x * x);
    }
    double den = Q * A - B;
    if (!(den > 0.0)) return ORC_E_MATERIAL;   /* Q below what L SLS can reach */
    double t = 1.0 / den;
    double complex m = 1.0;
    for (int l = 0; l < L; ++l) {
        double x = w * ts[l];
        m += t * (I * x) / (1.0 + I * x);
    }
    double re = creal(1.0 / csqrt(m));
    *M_R = rho * c * c * re * re;
    *tau = t;
    return ORC_OK;
}

/* Per-material validation and coefficients (pi_R, mu_R, tau_P, tau_S).
 * Rejects rho <= 0, cL <= 0, cS < 0, negative attenuation, a Poisson ratio
 * outside [-1, 0.5] (Sec. 3.2 "Mapping approaches": realistic range), and bad
 * thermal constants. */
int orc_material_coefs(const double *mat, int n_mat, double f0, double qc, int L,
                       double *coef, double *tau_sigma)
{
    if (n_mat <= 0 || n_mat > 256 || L < 0 || L > 4 || !(f0 > 0.0) || !(qc > 0.0))
        return ORC_E_ARG;
    orc_relaxation_times(f0, L, tau_sigma);
    for (int m = 0; m < n_mat; ++m) {
        const double *r = mat + (size_t)m * M_NCOL;
        double rho = r[M_RHO], cL = r[M_CL], cS = r[M_CS];
        if (!(rho > 0.0) || !(cL > 0.0) || !(cS >= 0.0)) return ORC_E_MATERIAL;
        if (!(r[M_AL] >= 0.0) || !(r[M_AS] >= 0.0)) return ORC_E_MATERIAL;
        /* nu = (cL^2 - 2 cS^2) / (2 (cL^2 - cS^2)) >= -1  <=>  4 cS^2 <= 3 cL^2 */
        if (!(4.0 * cS * cS <= 3.0 * cL * cL)) return ORC_E_MATERIAL;
        if (!(r[M_K] > 0.0) || !(r[M_CTH] > 0.0) || !(r[M_PERF] >= 0.0) ||
            !(r[M_HEAT] >= 0.0 && r[M_HEAT] <= 1.0))
            return ORC_E_MATERIAL;
        double *k = coef + (size_t)m * K_NCOL;
        if (fit_mode(rho, cL, r[M_AL], f0, qc, L, tau_sigma, &k[K_PI], &k[K_TAUP]))
            return ORC_E_MATERIAL;
        if (fit_mode(rho, cS, r[M_AS], f0, qc, L, tau_sigma, &k[K_MU], &k[K_TAUS]))
            return ORC_E_MATERIAL;
    }
    return ORC_OK;
}

/* Highest unrelaxed (instantaneous) wave speed over the table: the SLS
 * medium's fastest signal speed, used for the stability limit. */
static double max_unrelaxed_speed(const double *mat, const double *coef, int n_mat, int L)
{
    double cmax = 0.0;
    for (int m = 0; m < n_mat; ++m) {
        const double *k = coef + (size_t)m * K_NCOL;
        double rho = mat[(size_t)m * M_NCOL + M_RHO];
        double cp = sqrt(k[K_PI] * (1.0 + L * k[K_TAUP]) / rho);
        double cs = sqrt(k[K_MU] * (1.0 + L * k[K_TAUS]) / rho);
        if (cp > cmax) cmax = cp;
        if (cs > cmax) cmax = cs;
    }
    return cmax;
}

/* Stability limit of the O(4) staggered leapfrog in 3D: the largest symbol of
 * the staggered difference is (c1 - c2) = 7/6 per axis, so c dt/dx must not
 * exceed 1 / (sqrt(3) (c1 - c2)) = 6 / (7 sqrt 3). */
double orc_courant_limit(void) { return 1.0 / (sqrt(3.0) * (C1 - C2)); }

/* ------------------------------------------------------------------------ */
/* CPML profile (the paper defers boundary matching to its reference).        */
/* ------------------------------------------------------------------------ */

/* pos2 = 2*i for integer points, 2*i+1 for half points.  Depth into the layer
 * xi in [0,1]: low side (2P - pos2)/(2P), high side (pos2 - 2(n-1-P))/(2P). */
static void cpml_coef(int n, int P, double dx, double dt, double f0, double R,
                      double cmax, int pos2, double *a, double *b)
{
    *a = 0.0; *b = 0.0;
    if (P <= 0) return;
    double lo = (2.0 * P - pos2) / (2.0 * P);
    double hi = (pos2 - 2.0 * (n - 1 - P)) / (2.0 * P);
    double xi = lo > hi ? lo : hi;
    if (!(xi > 0.0)) return;
    if (xi > 1.0) xi = 1.0;
    double Lp = P * dx;
    double d0 = -3.0 * cmax * log(R) / (2.0 * Lp);
    double d = d0 * xi * xi;
    double al = M_PI * f0 * (1.0 - xi);
    *b = exp(-(d + al) * dt);
    *a = (d + al > 0.0) ? d * (*b - 1.0) / (d + al) : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Staggered differences with zero ghosts (Sec. 2.3, Levander O(4)).          */
/* ------------------------------------------------------------------------ */

/* The sweeps work on padded copies of every field: two layers of zeros on
 * each side of each axis hold the ghost values, so a stencil never needs a
 * bounds test.  P(i,j,k) addresses interior point (i,j,k) of a padded array. */
typedef struct {
    int px, py;          /* padded x and y extents */
} dims;

#define GH 2
#define P(i, j, k) ((((size_t)(k) + GH) * d.py + ((size_t)(j) + GH)) * d.px + ((size_t)(i) + GH))
#define F(f, dd, i, j, k) ((f)[P(i, j, k)])

/* D+ : integer-point field -> derivative at the half point ahead (s + 1/2).
 * D- : half-point field    -> derivative at the integer point (s).          */
static inline double Dp(double fm1, double f0, double f1, double f2, double dx)
{ return (C1 * (f1 - f0) + C2 * (f2 - fm1)) / dx; }
static inline double Dm(double fm2, double fm1, double f0, double f1, double dx)
{ return (C1 * (f0 - fm1) + C2 * (f1 - fm2)) / dx; }

#define DPX(f, i, j, k) Dp(F(f, d, i - 1, j, k), F(f, d, i, j, k), F(f, d, i + 1, j, k), F(f, d, i + 2, j, k), dx)
#define DPY(f, i, j, k) Dp(F(f, d, i, j - 1, k), F(f, d, i, j, k), F(f, d, i, j + 1, k), F(f, d, i, j + 2, k), dx)
#define DPZ(f, i, j, k) Dp(F(f, d, i, j, k - 1), F(f, d, i, j, k), F(f, d, i, j, k + 1), F(f, d, i, j, k + 2), dx)
#define DMX(f, i, j, k) Dm(F(f, d, i - 2, j, k), F(f, d, i - 1, j, k), F(f, d, i, j, k), F(f, d, i + 1, j, k), dx)
#define DMY(f, i, j, k) Dm(F(f, d, i, j - 2, k), F(f, d, i, j - 1, k), F(f, d, i, j, k), F(f, d, i, j + 1, k), dx)
#define DMZ(f, i, j, k) Dm(F(f, d, i, j, k - 2), F(f, d, i, j, k - 1), F(f, d, i, j, k), F(f, d, i, j, k + 1), dx)

/* CPML: psi <- b psi + a df ; the derivative used is df + psi (kappa = 1). */
static inline double pml(double *psi, size_t at, double a, double b, double df)
{
    if (a == 0.0 && b == 0.0) return df;
    psi[at] = b * psi[at] + a * df;
    return df + psi[at];
}

/* Source signature (Sec. 2.3: incident field injected as a stress source).
 * envelope 1: rectangular burst of n_cycles; 2: one-cycle raised-cosine ramp
 * then continuous wave; 0: no source. */
static double envelope_value(int envelope, int n_cycles, double f0, double t)
{
    if (envelope == 1) return (t >= 0.0 && t < n_cycles / f0) ? 1.0 : 0.0;
    if (envelope == 2) {
        if (t < 0.0) return 0.0;
        if (t < 1.0 / f0) return 0.5 * (1.0 - cos(M_PI * f0 * t));
        return 1.0;
    }
    return 0.0;
}

/* ------------------------------------------------------------------------ */
/* Acoustic time stepping: Eq. 1 with SLS memory variables, CPML, source,     */
/* peak and DFT capture.                                                      */
/* ------------------------------------------------------------------------ */

int orc_acoustic_run(const orc_grid *g, const uint8_t *index, const double *mat, int n_mat,
                     const double *src_plane, int k_src, double c0, int envelope, int n_cycles,
                     int n0, int n_steps, int peak_from, int dft_start, int dft_steps,
                     int check_cfl, double *state, double *peak, double *dftC, double *dftS)
{
    if (!g || !index || !mat || !state) return ORC_E_ARG;
    const int nx = g->nx, ny = g->ny, nz = g->nz, L = g->n_sls;
    if (nx < 1 || ny < 1 || nz < 1 || !(g->dx > 0.0) || !(g->dt > 0.0)) return ORC_E_ARG;
    const double dx = g->dx, dt = g->dt;
    const size_t N = (size_t)nx * ny * nz;

    double coef[256 * K_NCOL];
    double ts[4];
    int rc = orc_material_coefs(mat, n_mat, g->f0, g->qc, L, coef, ts);
    if (rc) return rc;
    for (size_t q = 0; q < N; ++q)
        if (index[q] >= n_mat) return ORC_E_MATERIAL;
    if (check_cfl) {
        double S = max_unrelaxed_speed(mat, coef, n_mat, L) * dt / dx;
        if (S > orc_courant_limit()) return ORC_E_CFL;
    }

    /* CPML coefficients per axis at integer (h=0) and half (h=1) points. */
    double cmax = 0.0;
    for (int m = 0; m < n_mat; ++m)
        if (mat[(size_t)m * M_NCOL + M_CL] > cmax) cmax = mat[(size_t)m * M_NCOL + M_CL];
    int nmax = nx > ny ? (nx > nz ? nx : nz) : (ny > nz ? ny : nz);
    double *pa = calloc((size_t)6 * nmax, sizeof(double));  /* [axis][h][s] */
    double *pb = calloc((size_t)6 * nmax, sizeof(double));
    /* padded working copy of every state array */
    const int NF = 9 + 6 * L + PSI_N;
    dims d = {nx + 2 * GH, ny + 2 * GH};
    const size_t NP = (size_t)(nx + 2 * GH) * (ny + 2 * GH) * (nz + 2 * GH);
    double *work = calloc((size_t)NF * NP, sizeof(double));
    if (!pa || !pb || !work) { free(pa); free(pb); free(work); return ORC_E_ARG; }
    int nax[3] = {nx, ny, nz};
    for (int ax = 0; ax < 3; ++ax)
        for (int h = 0; h < 2; ++h)
            for (int s = 0; s < nax[ax]; ++s) {
                size_t o = ((size_t)ax * 2 + h) * nmax + s;
                cpml_coef(nax[ax], g->n_pml, dx, dt, g->f0, g->pml_R, cmax, 2 * s + h, &pa[o], &pb[o]);
            }
#define PA(ax, h, s) pa[((size_t)(ax) * 2 + (h)) * nmax + (s)]
#define PB(ax, h, s) pb[((size_t)(ax) * 2 + (h)) * nmax + (s)]
    for (int f = 0; f < NF; ++f)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i)
                    work[(size_t)f * NP + P(i, j, k)] = state[(size_t)f * N + ((size_t)k * ny + j) * nx + i];

    double *vx = work + 0 * NP, *vy = work + 1 * NP, *vz = work + 2 * NP;
    double *sxx = work + 3 * NP, *syy = work + 4 * NP, *szz = work + 5 * NP;
    double *sxy = work + 6 * NP, *sxz = work + 7 * NP, *syz = work + 8 * NP;
    double *rmem = work + 9 * NP;                     /* [l][c][NP] */
    double *psi = work + (size_t)(9 + 6 * L) * NP;    /* [q][NP] */
#define PSI(q) (psi + (size_t)(q) * NP)
#define MAT(q, col) mat[(size_t)index[q] * M_NCOL + (col)]
#define COEF(q, col) coef[(size_t)index[q] * K_NCOL + (col)]

    /* Crank-Nicolson memory-variable coefficients per mechanism. */
    double ca[4], cb[4];
    for (int l = 0; l < L; ++l) {
        double h = dt / (2.0 * ts[l]);
        ca[l] = (1.0 - h) / (1.0 + h);
        cb[l] = (dt / ts[l]) / (1.0 + h);
    }
    const double w = 2.0 * M_PI * g->f0;
    const size_t sx = 1, sy = (size_t)nx, sz = (size_t)nx * ny;   /* index-volume strides */

    for (int n = n0; n < n0 + n_steps; ++n) {
        /* ---- velocity: v^{n+1/2} = v^{n-1/2} + dt b (div sigma^n) (Eq. 1, rows 1-3) */
#pragma omp parallel for schedule(static)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t q = ((size_t)k * ny + j) * nx + i;   /* index volume */
                    size_t p = P(i, j, k);                       /* padded fields */
                    if (i < nx - 1) {
                        double b = 2.0 / (MAT(q, M_RHO) + MAT(q + sx, M_RHO));
                        double d1 = pml(PSI(PSI_VX_X), p, PA(0, 1, i), PB(0, 1, i), DPX(sxx, i, j, k));
                        double d2 = pml(PSI(PSI_VX_Y), p, PA(1, 0, j), PB(1, 0, j), DMY(sxy, i, j, k));
                        double d3 = pml(PSI(PSI_VX_Z), p, PA(2, 0, k), PB(2, 0, k), DMZ(sxz, i, j, k));
                        vx[p] += dt * b * (d1 + d2 + d3);
                    }
                    if (j < ny - 1) {
                        double b = 2.0 / (MAT(q, M_RHO) + MAT(q + sy, M_RHO));
                        double d1 = pml(PSI(PSI_VY_X), p, PA(0, 0, i), PB(0, 0, i), DMX(sxy, i, j, k));
                        double d2 = pml(PSI(PSI_VY_Y), p, PA(1, 1, j), PB(1, 1, j), DPY(syy, i, j, k));
                        double d3 = pml(PSI(PSI_VY_Z), p, PA(2, 0, k), PB(2, 0, k), DMZ(syz, i, j, k));
                        vy[p] += dt * b * (d1 + d2 + d3);
                    }
                    if (k < nz - 1) {
                        double b = 2.0 / (MAT(q, M_RHO) + MAT(q + sz, M_RHO));
                        double d1 = pml(PSI(PSI_VZ_X), p, PA(0, 0, i), PB(0, 0, i), DMX(sxz, i, j, k));
                        double d2 = pml(PSI(PSI_VZ_Y), p, PA(1, 0, j), PB(1, 0, j), DMY(syz, i, j, k));
                        double d3 = pml(PSI(PSI_VZ_Z), p, PA(2, 1, k), PB(2, 1, k), DPZ(szz, i, j, k));
                        vz[p] += dt * b * (d1 + d2 + d3);
                    }
                }

        /* ---- stress + memory variables (Eq. 1 rows 4-9, Bohlen tau-method SLS) */
#pragma omp parallel for schedule(static)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t q = ((size_t)k * ny + j) * nx + i;
                    size_t p = P(i, j, k);
                    double piR = COEF(q, K_PI), muR = COEF(q, K_MU);
                    double tP = COEF(q, K_TAUP), tS = COEF(q, K_TAUS);

                    /* normal stresses at (i,j,k) */
                    double e[3];
                    e[0] = pml(PSI(PSI_EXX), p, PA(0, 0, i), PB(0, 0, i), DMX(vx, i, j, k));
                    e[1] = pml(PSI(PSI_EYY), p, PA(1, 0, j), PB(1, 0, j), DMY(vy, i, j, k));
                    e[2] = pml(PSI(PSI_EZZ), p, PA(2, 0, k), PB(2, 0, k), DMZ(vz, i, j, k));
                    double th = e[0] + e[1] + e[2];
                    double *sig[3] = {sxx, syy, szz};
                    for (int c = 0; c < 3; ++c) {
                        double Psi = piR * (1.0 + L * tP) * th - 2.0 * muR * (1.0 + L * tS) * (th - e[c]);
                        double The = piR * tP * th - 2.0 * muR * tS * (th - e[c]);
                        double sum = 0.0;
                        for (int l = 0; l < L; ++l) {
                            double *r = rmem + ((size_t)l * 6 + c) * NP;
                            double rn = ca[l] * r[p] - cb[l] * The;
                            sum += rn + r[p];
                            r[p] = rn;
                        }
                        sig[c][p] += dt * (Psi + 0.5 * sum);
                    }

                    /* shear stresses; each needs its four surrounding cells,
                     * offset o1 along its first axis and o2 along its second */
                    for (int c = 3; c < 6; ++c) {
                        size_t o1, o2;
                        double ev;
                        double *s;
                        if (c == 3) {          /* sxy at (i+1/2, j+1/2, k) */
                            if (i >= nx - 1 || j >= ny - 1) continue;
                            o1 = sx; o2 = sy; s = sxy;
                            ev = pml(PSI(PSI_XY_Y), p, PA(1, 1, j), PB(1, 1, j), DPY(vx, i, j, k)) +
                                 pml(PSI(PSI_XY_X), p, PA(0, 1, i), PB(0, 1, i), DPX(vy, i, j, k));
                        } else if (c == 4) {   /* sxz at (i+1/2, j, k+1/2) */
                            if (i >= nx - 1 || k >= nz - 1) continue;
                            o1 = sx; o2 = sz; s = sxz;
                            ev = pml(PSI(PSI_XZ_Z), p, PA(2, 1, k), PB(2, 1, k), DPZ(vx, i, j, k)) +
                                 pml(PSI(PSI_XZ_X), p, PA(0, 1, i), PB(0, 1, i), DPX(vz, i, j, k));
                        } else {               /* syz at (i, j+1/2, k+1/2) */
                            if (j >= ny - 1 || k >= nz - 1) continue;
                            o1 = sy; o2 = sz; s = syz;
                            ev = pml(PSI(PSI_YZ_Z), p, PA(2, 1, k), PB(2, 1, k), DPZ(vy, i, j, k)) +
                                 pml(PSI(PSI_YZ_Y), p, PA(1, 1, j), PB(1, 1, j), DPY(vz, i, j, k));
                        }
                        double u00 = COEF(q, K_MU), u10 = COEF(q + o1, K_MU);
                        double u01 = COEF(q + o2, K_MU), u11 = COEF(q + o1 + o2, K_MU);
                        double muh = 0.0;
                        if (u00 > 0.0 && u10 > 0.0 && u01 > 0.0 && u11 > 0.0)
                            muh = 4.0 / ((1.0 / u00 + 1.0 / u10) + (1.0 / u01 + 1.0 / u11));
                        double tsh = 0.25 * ((COEF(q, K_TAUS) + COEF(q + o1, K_TAUS)) +
                                             (COEF(q + o2, K_TAUS) + COEF(q + o1 + o2, K_TAUS)));
                        double Psi = muh * (1.0 + L * tsh) * ev;
                        double The = muh * tsh * ev;
                        double sum = 0.0;
                        for (int l = 0; l < L; ++l) {
                            double *r = rmem + ((size_t)l * 6 + c) * NP;
                            double rn = ca[l] * r[p] - cb[l] * The;
                            sum += rn + r[p];
                            r[p] = rn;
                        }
                        s[p] += dt * (Psi + 0.5 * sum);
                    }
                }

        /* ---- source: soft pressure-type stress source on plane k_src (Sec. 2.3) */
        if (src_plane && envelope && k_src >= 0 && k_src < nz) {
            double t = (n + 0.5) * dt;
            double env = envelope_value(envelope, n_cycles, g->f0, t);
            double scale = 2.0 * c0 * dt / dx;
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    double re = src_plane[2 * ((size_t)j * nx + i)];
                    double im = src_plane[2 * ((size_t)j * nx + i) + 1];
                    double A = sqrt(re * re + im * im);
                    double phi = atan2(im, re);
                    double sv = env * A * sin(w * t + phi);
                    size_t p = P(i, j, k_src);
                    sxx[p] -= scale * sv;
                    syy[p] -= scale * sv;
                    szz[p] -= scale * sv;
                }
        }

        /* ---- capture at t = (n+1) dt: p = -(sxx + syy + szz)/3 */
        int step = n + 1;
        int do_peak = peak && step >= peak_from;
        int do_dft = dftC && dftS && dft_steps > 0 && step >= dft_start && step < dft_start + dft_steps;
        if (do_peak || do_dft) {
            double cw = cos(w * step * dt), sw = sin(w * step * dt);
            for (int k = 0; k < nz; ++k)
                for (int j = 0; j < ny; ++j)
                    for (int i = 0; i < nx; ++i) {
                        size_t q = ((size_t)k * ny + j) * nx + i;
                        size_t p = P(i, j, k);
                        double pr = -(sxx[p] + syy[p] + szz[p]) / 3.0;
                        if (do_peak && fabs(pr) > peak[q]) peak[q] = fabs(pr);
                        if (do_dft) { dftC[q] += pr * cw; dftS[q] += pr * sw; }
                    }
        }
    }
    for (int f = 0; f < NF; ++f)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i)
                    state[(size_t)f * N + ((size_t)k * ny + j) * nx + i] = work[(size_t)f * NP + P(i, j, k)];
    free(pa);
    free(pb);
    free(work);
    return ORC_OK;
#undef PA
#undef PB
#undef PSI
#undef MAT
#undef COEF
}

/* Amplitude and phase from the DFT sums over N samples spanning whole
 * periods: p(t) = A cos(w t + phi)  =>  C = A N/2 cos phi, S = -A N/2 sin phi. */
void orc_amp_phase(const double *C, const double *S, size_t n, int n_samples,
                   double *amp, double *phase)
{
    for (size_t q = 0; q < n; ++q) {
        amp[q] = 2.0 * sqrt(C[q] * C[q] + S[q] * S[q]) / n_samples;
        phase[q] = atan2(-S[q], C[q]);
    }
}

/* ------------------------------------------------------------------------ */
/* Rayleigh-Sommerfeld incident field (Sec. 2.3, last paragraph).             */
/* ------------------------------------------------------------------------ */

/* Spherical bowl of aperture diameter `aperture` and radius of curvature `roc`,
 * apex at `apex` (m), acoustic axis `dir` (unit).  The cap is cut into rings of
 * equal polar-angle width and each ring into equal azimuthal elements, both of
 * length about ds = ds_over_lambda * lambda (area ds^2 = lambda^2/16 at 1/4).
 * Returns the number of elements, writing (x,y,z,area) rows when out != NULL. */
long orc_bowl_elements(double aperture, double roc, const double *apex, const double *dir,
                       double lambda, double ds_over_lambda, double *out)
{
    double a = 0.5 * aperture, R = roc;
    if (!(a > 0.0) || !(R >= a)) return -1;
    double ds = ds_over_lambda * lambda;
    double thmax = asin(a / R);
    int nr = (int)ceil(R * thmax / ds);
    if (nr < 1) nr = 1;
    /* rotation taking +z to dir (Rodrigues, about z x dir) */
    double ux = dir[0], uy = dir[1], uz = dir[2];
    double nrm = sqrt(ux * ux + uy * uy + uz * uz);
    ux /= nrm; uy /= nrm; uz /= nrm;
    double kx = -uy, ky = ux;                 /* z x u = (-uy, ux, 0) */
    double sn = sqrt(kx * kx + ky * ky), cs = uz;
    if (sn > 0.0) { kx /= sn; ky /= sn; }
    long count = 0;
    for (int r = 0; r < nr; ++r) {
        double t0 = thmax * r / nr, t1 = thmax * (r + 1) / nr, tc = 0.5 * (t0 + t1);
        double ring_area = 2.0 * M_PI * R * R * (cos(t0) - cos(t1));
        int naz = (int)lround(2.0 * M_PI * R * sin(tc) / ds);
        if (naz < 1) naz = 1;
        for (int e = 0; e < naz; ++e) {
            double ph = 2.0 * M_PI * (e + 0.5) / naz;
            double px = R * sin(tc) * cos(ph), py = R * sin(tc) * sin(ph), pz = R * (1.0 - cos(tc));
            /* rotate p about unit axis (kx,ky,0) by angle with cos=cs, sin=sn */
            double kdotp = kx * px + ky * py;
            double cx = ky * pz, cy = -kx * pz, cz = kx * py - ky * px;   /* k x p */
            double rx = px * cs + cx * sn + kx * kdotp * (1.0 - cs);
            double ry = py * cs + cy * sn + ky * kdotp * (1.0 - cs);
            double rz = pz * cs + cz * sn;
            if (out) {
                out[4 * count + 0] = apex[0] + rx;
                out[4 * count + 1] = apex[1] + ry;
                out[4 * count + 2] = apex[2] + rz;
                out[4 * count + 3] = ring_area / naz;
            }
            ++count;
        }
    }
    return count;
}

/* p(x) = (i k p0 / 2 pi) sum_e dA_e exp(-i k r_e) / r_e  on the plane z = z_plane,
 * grid point (i,j) at (i dx, j dx); p0 = rho0 c0 u0 is the surface pressure. */
int orc_rs_plane(double aperture, double roc, const double *apex, const double *dir,
                 double ds_over_lambda, int nx, int ny, double dx, double z_plane,
                 double f0, double c0, double p0, double *out)
{
    double lambda = c0 / f0, k = 2.0 * M_PI / lambda;
    long ne = orc_bowl_elements(aperture, roc, apex, dir, lambda, ds_over_lambda, NULL);
    if (ne <= 0) return ORC_E_ARG;
    double *el = malloc(sizeof(double) * 4 * ne);
    if (!el) return ORC_E_ARG;
    orc_bowl_elements(aperture, roc, apex, dir, lambda, ds_over_lambda, el);
    double complex pref = I * k * p0 / (2.0 * M_PI);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double x = i * dx, y = j * dx;
            double complex acc = 0.0;
            for (long e = 0; e < ne; ++e) {
                double ddx = x - el[4 * e], ddy = y - el[4 * e + 1], ddz = z_plane - el[4 * e + 2];
                double r = sqrt(ddx * ddx + ddy * ddy + ddz * ddz);
                acc += el[4 * e + 3] * cexp(-I * k * r) / r;
            }
            double complex p = pref * acc;
            out[2 * ((size_t)j * nx + i)] = creal(p);
            out[2 * ((size_t)j * nx + i) + 1] = cimag(p);
        }
    free(el);
    return ORC_OK;
}

/* Elements with complex weights (phased arrays): rows (x, y, z, area, w_re,
 * w_im); p(x) = (i k p0 / 2 pi) sum_e w_e dA_e exp(-i k r_e) / r_e on the plane
 * z = z_plane, grid point (i,j) at (i dx, j dx). */
int orc_rs_elements(const double *elem, long ne, double p0, double c0, int nx, int ny,
                    double dx, double z_plane, double f0, double *out)
{
    if (ne < 1) return ORC_E_ARG;
    double k = 2.0 * M_PI * f0 / c0;
    double complex pref = I * k * p0 / (2.0 * M_PI);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double x = i * dx, y = j * dx;
            double complex acc = 0.0;
            for (long e = 0; e < ne; ++e) {
                const double *r = elem + 6 * e;
                double ddx = x - r[0], ddy = y - r[1], ddz = z_plane - r[2];
                double d = sqrt(ddx * ddx + ddy * ddy + ddz * ddz);
                acc += (r[4] + I * r[5]) * r[3] * cexp(-I * k * d) / d;
            }
            double complex p = pref * acc;
            out[2 * ((size_t)j * nx + i)] = creal(p);
            out[2 * ((size_t)j * nx + i) + 1] = cimag(p);
        }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* BHTE (Pennes) with CEM43 dose (Sec. 2.4).                                  */
/* ------------------------------------------------------------------------ */

/* rho c_th dT/dt = div(k grad T) - w_b rhob_cb (T - T_a) + DC * Q, explicit
 * forward Euler, 7-point stencil with face conductivity = harmonic mean.
 * Q = heat_frac * alphaL * (p_scale * amp)^2 / (rho cL) during the first n_on
 * steps, 0 during the n_off that follow.  Border voxels stay at T_a.
 * T_max and CEM43 = sum dt/60 R^(43 - T), R = 0.5 for T >= 43 else 0.25,
 * are taken after every step. */
int orc_bhte_run(int nx, int ny, int nz, double dx, const uint8_t *index, const double *mat,
                 int n_mat, const double *amp, double p_scale, double dt, int n_on, int n_off,
                 double duty, double T_a, double rhob_cb, double *T, double *Tmax, double *cem)
{
    const size_t N = (size_t)nx * ny * nz;
    for (size_t q = 0; q < N; ++q)
        if (index[q] >= n_mat) return ORC_E_MATERIAL;
    double *Tn = malloc(sizeof(double) * N);
    double *Q = malloc(sizeof(double) * N);
    if (!Tn || !Q) { free(Tn); free(Q); return ORC_E_ARG; }
    for (size_t q = 0; q < N; ++q) {
        const double *m = mat + (size_t)index[q] * M_NCOL;
        double A = amp ? p_scale * amp[q] : 0.0;
        Q[q] = m[M_HEAT] * m[M_AL] * A * A / (m[M_RHO] * m[M_CL]);
    }
    double idx2 = 1.0 / (dx * dx);
    for (int n = 0; n < n_on + n_off; ++n) {
        double dc = (n < n_on) ? duty : 0.0;
#pragma omp parallel for schedule(static)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t q = ((size_t)k * ny + j) * nx + i;
                    if (i == 0 || j == 0 || k == 0 || i == nx - 1 || j == ny - 1 || k == nz - 1) {
                        Tn[q] = T_a;
                        continue;
                    }
                    const double *m = mat + (size_t)index[q] * M_NCOL;
                    double kc = m[M_K];
                    size_t nb[6] = {q - 1, q + 1, q - (size_t)nx, q + (size_t)nx,
                                    q - (size_t)nx * ny, q + (size_t)nx * ny};
                    double lap = 0.0;
                    for (int f = 0; f < 6; ++f) {
                        double kn = mat[(size_t)index[nb[f]] * M_NCOL + M_K];
                        double kf = 2.0 * kc * kn / (kc + kn);
                        lap += kf * (T[nb[f]] - T[q]);
                    }
                    double rhs = lap * idx2 - m[M_PERF] * rhob_cb * (T[q] - T_a) + dc * Q[q];
                    Tn[q] = T[q] + dt * rhs / (m[M_RHO] * m[M_CTH]);
                }
        memcpy(T, Tn, sizeof(double) * N);
        /* independent per voxel: the same arithmetic in any thread order */
#pragma omp parallel for schedule(static)
        for (size_t q = 0; q < N; ++q) {
            if (T[q] > Tmax[q]) Tmax[q] = T[q];
            double R = (T[q] >= 43.0) ? 0.5 : 0.25;
            cem[q] += dt / 60.0 * pow(R, 43.0 - T[q]);
        }
    }
    free(Tn);
    free(Q);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Energy-loss factor E_L (Sec. 2.4, Eq. 2) and T_S = sqrt(E_L) (Sec. 3.2).   */
/* ------------------------------------------------------------------------ */

/* I_PA = A^2 / (2 rho c) per voxel.  z_m is the plane holding the largest
 * water-run intensity (ties: the lowest linear index).  E_L is the ratio of
 * the plane sums of the two intensity maps at z_m. */
int orc_transmission(int nx, int ny, int nz,
                     const uint8_t *idx_a, const double *mat_a, const double *amp_a,
                     const uint8_t *idx_w, const double *mat_w, const double *amp_w,
                     double *EL, int *zm)
{
    const size_t N = (size_t)nx * ny * nz;
    double best = -1.0;
    size_t qbest = 0;
    for (size_t q = 0; q < N; ++q) {
        const double *m = mat_w + (size_t)idx_w[q] * M_NCOL;
        double inten = amp_w[q] * amp_w[q] / (2.0 * m[M_RHO] * m[M_CL]);
        if (inten > best) { best = inten; qbest = q; }
    }
    int z = (int)(qbest / ((size_t)nx * ny));
    double sa = 0.0, sw = 0.0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t q = ((size_t)z * ny + j) * nx + i;
            const double *ma = mat_a + (size_t)idx_a[q] * M_NCOL;
            const double *mw = mat_w + (size_t)idx_w[q] * M_NCOL;
            sa += amp_a[q] * amp_a[q] / (2.0 * ma[M_RHO] * ma[M_CL]);
            sw += amp_w[q] * amp_w[q] / (2.0 * mw[M_RHO] * mw[M_CL]);
        }
    if (!(sw > 0.0)) return ORC_E_ARG;
    *EL = sa / sw;
    *zm = z;
    return ORC_OK;
}
