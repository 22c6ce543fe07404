// bvf_transmission_noalloc: the energy-loss reduction of bvf_transmission
// without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need this
// result: an application whose memory is entirely reserved up front by its own
// pool (a framework's caching allocator), where a raw allocation may fail or
// fragment that pool, or a tight planning loop where an allocation call could
// stall the device.  This entry point runs the same kernels as
// bvf_transmission but keeps their temporaries in a fixed array compiled into
// the library, so it calls no allocator at all.
//
// The array lives in global memory of every GPU that loads the library, for as
// long as the process runs (about 4 KiB).  All calls share it and it keeps the
// contents of the last call; the parts that must start from a known value are
// re-initialised by each call.  Two calls whose work overlaps on the GPU (for
// example on two streams without ordering between them) use the same array and
// race; order such calls on one stream or synchronise between them.
//
// Every call looks up the array's device address on the current device
// (cudaGetSymbolAddress, with that device current).  The address is not
// cached: a cached one would dangle once the device's context is torn down and
// the library's module loaded again (cudaDeviceReset), and the look-up is cheap
// once the module is loaded.  The call waits for its stream before returning.
#include <cmath>
#include <cstddef>
#include <cstring>

#include "bvf_internal.cuh"

namespace {

using namespace bvf;

// Layout of the scratch array: per-material 1/(2 rho c) for both tables, the
// bit pattern of the largest water intensity, the index where it occurs, and
// the two plane sums plus the plane number.
struct TransmissionScratch {
    double z[2][BVF_MAX_MATERIALS];
    unsigned long long best;
    unsigned long long qbest;
    double sums[3];
};

constexpr size_t kScratchBytes = sizeof(TransmissionScratch);   // 4136 bytes

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// failures are reported through bvf_last_error(NULL), like every context-free call
int noalloc_fail(int code, const char *msg)
{
    set_context_free_error(msg);
    return code;
}

// Device address of the scratch array on the current device, looked up at
// each call (the host-side name g_scratch is not a device address and must
// never be handed to a kernel).
cudaError_t scratch_on_current_device(TransmissionScratch **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<TransmissionScratch *>(p);
    return cudaSuccess;
}

}  // namespace

extern "C" int bvf_transmission_noalloc(int nx, int ny, int nz, const uint8_t *d_idx_a,
                                        const bvf_material *h_mat_a, int n_a,
                                        const double *d_amp_a, const uint8_t *d_idx_w,
                                        const bvf_material *h_mat_w, int n_w,
                                        const double *d_amp_w, double *h_EL, double *h_TS,
                                        int *h_zm, double *h_Iw_max, void *stream)
{
    if (nx < 1 || ny < 1 || nz < 1 || !d_idx_a || !h_mat_a || !d_amp_a || !d_idx_w || !h_mat_w ||
        !d_amp_w)
        return noalloc_fail(BVF_E_ARG, "bvf_transmission_noalloc: bad argument");
    if (n_a < 1 || n_w < 1 || n_a > BVF_MAX_MATERIALS || n_w > BVF_MAX_MATERIALS)
        return noalloc_fail(BVF_E_ARG,
                            "bvf_transmission_noalloc: each material table must have 1 to 256 "
                            "rows (the fixed scratch array holds 256 per table)");
    TransmissionScratch *d = nullptr;
    cudaError_t e = scratch_on_current_device(&d);
    if (e != cudaSuccess)
        return noalloc_fail(BVF_E_CUDA, "bvf_transmission_noalloc: scratch array not reachable");

    // Host-side copy of the values that must start known: the 1/(2 rho c)
    // tables, the running maximum (0) and the running arg-min index (~0).
    static thread_local TransmissionScratch h;
    std::memset(&h, 0, sizeof h);
    for (int m = 0; m < n_a; ++m) h.z[0][m] = 1.0 / (2.0 * h_mat_a[m].rho * h_mat_a[m].cL);
    for (int m = 0; m < n_w; ++m) h.z[1][m] = 1.0 / (2.0 * h_mat_w[m].rho * h_mat_w[m].cL);
    h.best = 0ull;
    h.qbest = ~0ull;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)nx * ny * nz;
    double res[3] = {0.0, 0.0, 0.0};
    unsigned long long best_bits = 0;
    e = cudaMemcpyAsync(d, &h, offsetof(TransmissionScratch, sums), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_intensity_argmax(d_idx_w, d->z[1], d_amp_w, n, &d->best, s);
    if (e == cudaSuccess)
        e = launch_intensity_argmin_index(d_idx_w, d->z[1], d_amp_w, n, &d->best, &d->qbest, s);
    if (e == cudaSuccess)
        e = launch_plane_sums(d_idx_a, d->z[0], d_amp_a, d_idx_w, d->z[1], d_amp_w, nx, ny, nz,
                              &d->qbest, d->sums, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(res, d->sums, sizeof res, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&best_bits, &d->best, sizeof best_bits, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return noalloc_fail(BVF_E_CUDA, cudaGetErrorString(e));
    if (!(res[1] > 0.0)) return noalloc_fail(BVF_E_ARG, "bvf_transmission_noalloc: zero water intensity");
    const double el = res[0] / res[1];
    if (h_EL) *h_EL = el;
    if (h_TS) *h_TS = std::sqrt(el);
    if (h_zm) *h_zm = (int)res[2];
    if (h_Iw_max) std::memcpy(h_Iw_max, &best_bits, sizeof(double));
    return BVF_OK;
}
