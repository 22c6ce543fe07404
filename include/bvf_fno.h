/* bvf_fno.h - C ABI of the Fourier-neural-operator surrogate of the acoustic
 * solve (inference on the GPU).
 *
 * The paper's Discussion names machine-learned models as the route to
 * interactive planning; this surrogate maps the feature volume of one
 * placement (material maps and the source plane) to a field of the same grid
 * with the Fourier neural operator of Li et al. (ICLR 2021, Sec. 4): a
 * pointwise lift, L Fourier layers v <- GELU(W v + b + IFFT(R . FFT(v))) (no
 * GELU after the last) and a two-layer pointwise projection.  The FDTD of
 * bvf.h stays the reference the surrogate is judged against.
 *
 * Conventions (all arrays channel-major [c][z][y][x], x fastest, FP32):
 *   - The FFT runs over (z, y, x) with the real-input half spectrum along x.
 *     Kept modes: kx = 0 .. m-1; ky and kz take the 2m signed frequencies
 *     0 .. m-1 and -m .. -1, slot j in [0, 2m) holding j for j < m and j - 2m
 *     otherwise.  The inverse is the real inverse transform of that half
 *     spectrum: kx = 0 terms count their real part once, kx >= 1 twice, all
 *     over N = nx ny nz.  Grids need m <= nx/2, 2m <= ny and 2m <= nz.
 *   - Flat weight blob (FP32, host memory, copied at create), in order:
 *       lift      Wp[width][c_in], bp[width]
 *       layer l   R_l[2m][2m][m][width_in][width_out][2] (re, im),
 *                 W_l[width_out][width_in], b_l[width]
 *       project   Q1[hidden][width], q1[hidden], Q2[c_out][hidden], q2[c_out]
 *   - GELU(x) = x Phi(x) with the exact normal CDF.
 *
 * Status codes and the material row are those of bvf.h.  Contexts are not
 * thread-safe; calls are asynchronous on `stream` (a cudaStream_t, NULL =
 * legacy default stream) unless stated otherwise.
 */
#ifndef BVF_FNO_H
#define BVF_FNO_H

#include "bvf.h"

#ifdef __cplusplus
extern "C" {
#endif

#define BVF_FNO_MAX_WIDTH 64
#define BVF_FNO_MAX_MODES 16
#define BVF_FNO_MAX_HIDDEN 256
#define BVF_FNO_MAX_CIN 16
#define BVF_FNO_MAX_COUT 8
#define BVF_FNO_MAX_LAYERS 16
#define BVF_FNO_FEATURES 8     /* channels written by bvf_fno_features */

typedef struct {
    int c_in;        /* input channels, 1 .. BVF_FNO_MAX_CIN            */
    int width;       /* channels of the Fourier layers: 16, 32, 48 or 64 */
    int modes;       /* m, 1 .. BVF_FNO_MAX_MODES                        */
    int n_layers;    /* Fourier layers, 1 .. BVF_FNO_MAX_LAYERS          */
    int hidden;      /* projection width, 1 .. BVF_FNO_MAX_HIDDEN         */
    int c_out;       /* output channels, 1 .. BVF_FNO_MAX_COUT            */
} bvf_fno_dims;

typedef struct bvf_fno bvf_fno;

/* Number of floats in the weight blob of `d` (layout above); 0 if the
 * dimensions are out of range or d is NULL. */
size_t bvf_fno_weight_count(const bvf_fno_dims *d);

/* Create a surrogate on the current device with the weights h_weights (n
 * floats, host memory, copied).  Errors: BVF_E_ARG (bad dims, n different from
 * bvf_fno_weight_count, NULL pointers), BVF_E_NOMEM.  *out is NULL on failure.
 * Synchronous. */
int bvf_fno_create(bvf_fno **out, const bvf_fno_dims *d, const float *h_weights, size_t n);

/* Free the surrogate and its workspace (synchronises the device). */
int bvf_fno_destroy(bvf_fno *f);

/* One inference: d_in [c_in][nz][ny][nx] -> d_out [c_out][nz][ny][nx], both
 * caller-owned device memory that must not overlap.  The context keeps a
 * workspace sized for the largest grid seen (two activation volumes of
 * width*nx*ny*nz floats plus the truncated spectra); a call on a grid other
 * than the previous call's synchronises the device first (the workspace may
 * grow and the twiddle tables are rebuilt).  Errors: BVF_E_ARG
 * (NULL pointers, grid too small for the modes, nx*ny*nz >= 2^31),
 * BVF_E_NOMEM, BVF_E_CUDA. */
int bvf_fno_forward(bvf_fno *f, int nx, int ny, int nz, const float *d_in, float *d_out,
                    void *stream);

/* Wait for `stream` and report: BVF_E_CUDA if a CUDA error occurred or if a
 * kernel's bounded wait for its tensor-core results ran out since the last
 * call (the flag is then cleared), BVF_E_ARG for a NULL surrogate. */
int bvf_fno_synchronize(bvf_fno *f, void *stream);

/* Feature volume of one placement for a surrogate with c_in =
 * BVF_FNO_FEATURES: d_out [8][nz][ny][nx] gets, per voxel of material row r
 * (d_index, uint8 on the device; h_table, n_mat rows in host memory) against
 * the coupling medium h_water:
 *   0: cL/cL_w - 1   1: rho/rho_w - 1   2: alphaL cL_w / f0 (Np per wavelength)
 *   3, 4: Re, Im of the source plane d_src (ny*nx interleaved complex floats,
 *         Pa, device) divided by p_norm, on plane k_src only (0 elsewhere)
 *   5, 6, 7: cell-centre coordinates (i+1/2)/nx, (j+1/2)/ny, (k+1/2)/nz.
 * Errors: BVF_E_ARG (NULL pointers, bad sizes, k_src outside [0, nz), p_norm
 * or f0 not positive, n_mat outside 1 .. BVF_MAX_MATERIALS), BVF_E_MATERIAL
 * (a water row with rho or cL not positive). */
int bvf_fno_features(const uint8_t *d_index, const bvf_material *h_table, int n_mat,
                     const bvf_material *h_water, int nx, int ny, int nz, double f0, int k_src,
                     const float *d_src, double p_norm, float *d_out, void *stream);

/* Device time of the last bvf_fno_forward per stage (ms), measured with CUDA
 * events when timing is enabled (bvf_fno_timing); all zero otherwise.
 * Stages: 0 lift, 1 forward DFT along x, 2 along y, 3 along z, 4 mode mixing,
 * 5 inverse along z, 6 inverse along y, 7 inverse along x + pointwise + GELU,
 * 8 projection.  Where a (z, y) row of every channel fits in shared memory,
 * the forward x transform runs inside the lift and the stage-7 pass (stage 1
 * then reads about zero).  Synchronises `stream` of the last forward. */
#define BVF_FNO_STAGES 9
int bvf_fno_timing(bvf_fno *f, int enable);
int bvf_fno_stage_times(bvf_fno *f, double *ms_out);

/* ---- BF16 tensor-core product ---------------------------------------------
 * C = alpha A B + beta C (+ bias) (-> GELU) on the fifth-generation tensor
 * cores: A, B and C are FP32 arrays in device memory, the operands are
 * rounded to BF16 and the products accumulate in FP32.  The surrogate's BF16
 * inference and its training are built from this product (no counterpart in
 * the paper).  Element (m, k) of A is A[b sab + m sam + k sak] for batch b,
 * (k, n) of B is B[b sbb + k sbk + n sbn], (m, n) of C is C[b scb + m scm +
 * n scn]; any strides (elements), so transposed and batched views need no
 * copies.  bias_mode 1 adds bias[n], 2 adds bias[m]; act 1 applies GELU and,
 * when C_pre is not NULL, stores the value before GELU there (same strides as
 * C); act 2 multiplies the result by GELU'(C_pre) (the backward of act 1, with
 * C_pre holding the forward pre-activation).  ksplit > 1 splits K over that many blocks that add alpha A B into C
 * atomically (then beta must be 1, with no bias and no activation).
 * d_flag: a device int that receives bit 2 if a bounded wait for the tensor
 * cores ran out (the blocks concerned leave their tile of C unwritten).
 * Asynchronous on `stream`.  Errors: BVF_E_ARG, BVF_E_CUDA. */
typedef struct bvf_gemm {
    const float *A;
    long long sam, sak, sab;
    const float *B;
    long long sbk, sbn, sbb;
    float *C;
    long long scm, scn, scb;
    float *C_pre;
    const float *bias;
    int bias_mode;
    int M, N, K, batch, ksplit;
    float alpha, beta;
    int act;           /* 0 none, 1 GELU, 2 times GELU'(C_pre) */
} bvf_gemm;
int bvf_gemm_bf16(const bvf_gemm *g, int *d_flag, void *stream);

/* ---- BF16 inference and training ----------------------------------------
 * The same network with every contraction on the BF16 tensor-core product
 * (bvf_gemm_bf16): the lift, W v + b and the projection as channel products;
 * each Fourier layer's truncated transform as three products (x: real ->
 * kept modes, y and z: complex, as real 2 x 2 blocks) with axis permutes in
 * between, the inverse likewise with the real-inverse weights c(kx)/N (c = 1
 * for kx = 0, 2 otherwise); the mode mix in FP32 (no counterpart in the
 * paper: planning-time inference and training of the surrogate).  A context
 * is sized for one grid and up to max_batch samples and keeps FP32 master
 * weights, their gradient, Adam moments and every activation the backward pass
 * needs.  Inputs [batch][c_in][nz][ny][nx], outputs [batch][c_out][...],
 * FP32 device memory.  bvf_fno_bf16_forward is inference: it writes d_out
 * directly, stores no pre-activation, makes no runtime call but its launches
 * after the first call of each product shape, and so may be recorded in a
 * CUDA graph; it must not overlap a gradient or Adam call of the same context.
 *
 * Loss of a batch (bvf_fno_bf16_gradient / _adam): the mean over samples of
 * the relative L2 error ||out_0 - target|| / ||target|| of output channel 0
 * (d_target [batch][nz][ny][nx]), plus, if c_out >= 2, el_weight times the
 * mean squared difference between the spatial mean of output channel 1 and
 * d_el[b] (the sample's transmission efficiency E_L; NULL when el_weight is
 * 0).  d_grad (n floats, the blob layout, may be NULL) receives the gradient;
 * *h_loss (may be NULL) the loss, which makes the call wait for `stream`.
 * bvf_fno_bf16_adam takes one Adam step (beta1 0.9, beta2 0.999, eps 1e-8,
 * learning rate lr) on the context's weights; bvf_fno_bf16_weights copies them
 * out (synchronous).  bvf_fno_bf16_synchronize reports BVF_E_CUDA if a bounded
 * tensor-core wait ran out.  Errors: BVF_E_ARG, BVF_E_NOMEM, BVF_E_CUDA. */
typedef struct bvf_fno_bf16 bvf_fno_bf16;
int bvf_fno_bf16_create(bvf_fno_bf16 **out, const bvf_fno_dims *d, const float *h_weights, size_t n,
                        int nx, int ny, int nz, int max_batch);
int bvf_fno_bf16_destroy(bvf_fno_bf16 *t);
int bvf_fno_bf16_forward(bvf_fno_bf16 *t, int batch, const float *d_in, float *d_out, void *stream);
int bvf_fno_bf16_gradient(bvf_fno_bf16 *t, int batch, const float *d_in, const float *d_target,
                          const float *d_el, double el_weight, float *d_grad, double *h_loss,
                          void *stream);
int bvf_fno_bf16_adam(bvf_fno_bf16 *t, int batch, const float *d_in, const float *d_target,
                      const float *d_el, double el_weight, double lr, double *h_loss, void *stream);
int bvf_fno_bf16_weights(bvf_fno_bf16 *t, float *h_weights);
int bvf_fno_bf16_synchronize(bvf_fno_bf16 *t, void *stream);

/* Mean of n floats of device memory (FP64 sum): the transmission efficiency
 * E_L read from the spatial mean of a surrogate output channel.  Waits for
 * `stream`.  Errors: BVF_E_ARG, BVF_E_CUDA. */
int bvf_fno_mean(const float *d_x, size_t n, double *h_mean, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BVF_FNO_H */
