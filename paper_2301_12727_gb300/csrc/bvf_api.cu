// Host side of libbvf: the C ABI declared in include/bvf.h.
//
// Coefficient derivation (FP64, once per material table) follows Sec. 3.2
// (Eq. 3: Q = w / (2 c alpha), Q = Q0 q_c; relaxation constants fitted to Q)
// and the standard-linear-solid tau method; the CPML profile follows the
// convolutional PML with kappa = 1 (the paper defers boundary matching to its
// reference).  All per-voxel work runs in the kernels of bvf_acoustic.cu and
// bvf_aux.cu.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "bvf_internal.cuh"
#include "bvf_tma.cuh"

using namespace bvf;

namespace {

constexpr double kPi = 3.14159265358979323846;
thread_local std::string g_last_error;

struct MatDerived {
    double piR, muR, tauP, tauS;
};

}  // namespace

void bvf::set_context_free_error(const char *msg) { g_last_error = msg; }

struct bvf_ctx {
    bvf_grid g{};
    bvf_physics ph{};
    int L = 0;
    size_t N = 0, fstride = 0;
    int h16 = 0;                      // state stored as scaled FP16
    size_t es = 4;                    // bytes per state element
    double s_sig = 1.0, s_v = 1.0, s_r = 1.0;   // storage scales of sigma, v, r
    int P = 0, W = 0, nmax = 0;
    // device state
    void *fields = nullptr;           // (9 + 6L) arrays of fstride elements
    float *psi = nullptr;             // 3 slabs x 6 memories
    size_t slab_x = 0, slab_y = 0, slab_z = 0;
    float *peak = nullptr;
    double *dftC = nullptr, *dftS = nullptr;
    int dft_count = 0;
    uint8_t *index = nullptr;
    MatCoef *lut = nullptr;
    float *buoy = nullptr;            // material-pair buoyancy table
    float2 *pml = nullptr;
    float2 *src = nullptr;
    int *flag = nullptr;
    unsigned *scratch_u = nullptr;
    float *T2 = nullptr, *Q = nullptr, *cemf = nullptr;
    ThermCoef *tlut = nullptr;
    float *kface = nullptr;      // [n_mat][n_mat] face conductivities of the BHTE
    // the material index with rows padded to a multiple of 16 bytes, read by
    // the tensor maps when nx % 16 != 0 (a TMA row stride is whole 16-byte units)
    uint8_t *index_p = nullptr;
    size_t index_pitch = 0;
    // device staging of bvf_plan_host (allocated on its first call)
    uint8_t *h_index_d = nullptr;
    float *h_peak_d = nullptr, *h_T_d = nullptr, *h_Tmax_d = nullptr;
    double *h_amp_d = nullptr, *h_cem_d = nullptr;
    // host mirror
    std::vector<bvf_material> table;
    std::vector<MatDerived> derived;
    std::vector<double> tau_sigma;
    bool have_materials = false;
    int k_src = -1, envelope = BVF_ENV_NONE, n_cycles = 0;
    double c0 = 1500.0;
    bool have_source = false;
    long long steps = 0, launches = 0, thermal_steps = 0;
    double courant = 0.0;
    int kchunk = 0;                   // z-planes per block (0 = default)
    bvf_tile tile{0, 0, 0};           // tile of the TMA kernels (bvf_set_tile; 0 = default)
    bool tma = false;                 // velocity kernel fed by TMA
    bool tma_stress = false;          // stress kernel fed by TMA
    StressTmaMaps smaps{};            // boxes of 8-row tiles
    VelocityTmaMaps vmaps{};
    StressTmaMaps smaps_x[2]{};       // boxes of 4- and 16-row tiles
    VelocityTmaMaps vmaps_x[2]{};
    std::string err;
    // per-launch event timing of the acoustic kernels
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<cudaEvent_t> ev_vel, ev_str;   // start/stop pairs, flattened
    size_t ev_used = 0;
    double vel_ms = 0.0, str_ms = 0.0;
    long long vel_n = 0, str_n = 0;
    // wall-clock budget of one bvf_run_acoustic / bvf_run_thermal call (s, 0 = none)
    double budget_s = 0.0;
    cudaEvent_t budget_ev[2] = {nullptr, nullptr};
    // test hook of the bounded TMA waits, applied to the next acoustic step
    int hold = 0, hold_plane = -1;
    unsigned hold_limit = 0;
    // second stream and fork/join events of bvf_plan's concurrent water run
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
};

struct bvf_batch {
    std::vector<bvf_ctx *> ctx;       // not owned
    int L = 0, h16 = 0, n_mat_max = 1;
    int grid_vel = 0, grid_str = 0;   // persistent grid sizes
    StressTmaMaps *d_sm = nullptr;    // [ctx.size()]
    VelocityTmaMaps *d_vm = nullptr;
    StepParam *d_steps = nullptr;
    size_t steps_cap = 0;
    int *d_step = nullptr;            // step counter read by the kernels
    cudaStream_t cap = nullptr;       // stream the graph is captured on
    cudaGraphExec_t exec = nullptr;
    BatchParams bp{};
    std::vector<StepParam> h_steps;
    long long launches = 0;
    // side streams of bvf_batch_run_streams, with their join events
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> side_ev;
    cudaEvent_t fork = nullptr;
    // bvf_batch_run_graph: the recorded graph, what it was recorded for (start
    // steps, step counts, capture windows, z-chunks, branches) and the counter
    // advances of one replay
    cudaGraphExec_t gexec = nullptr;
    std::vector<long long> gsig;
    std::vector<long long> gdsteps, gddft;
};

namespace {

int fail(bvf_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    g_last_error = msg;
    return code;
}

int cuda_fail(bvf_ctx *c, cudaError_t e, const char *where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(c, e == cudaErrorMemoryAllocation ? BVF_E_NOMEM : BVF_E_CUDA, m);
}

// context-free variant of CK (batch calls report through bvf_last_error(NULL))
#define CK_FREE(call, where)                                       \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(nullptr, e_, where); \
    } while (0)

#define CK(call, where)                                      \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
    } while (0)

// Relaxation times 1 / (2 pi f_l), f_l log-spaced on [f0/3, 3 f0] (f0 if L = 1).
std::vector<double> relaxation_times(double f0, int L)
{
    std::vector<double> ts(L);
    for (int l = 0; l < L; ++l) {
        const double e = (L == 1) ? 0.0 : -1.0 + 2.0 * l / double(L - 1);
        ts[l] = 1.0 / (2.0 * kPi * f0 * std::pow(3.0, e));
    }
    return ts;
}

// Single-frequency fit of the SLS strength tau to Q = qc w / (2 c alpha):
// Q(w) = (1 + tau B) / (tau A) with A = sum w ts / (1 + (w ts)^2),
// B = sum (w ts)^2 / (1 + (w ts)^2); relaxed modulus so that the phase speed
// at f0 is c:  M_R = rho c^2 (Re m^{-1/2})^2, m = 1 + tau sum i w ts / (1 + i w ts).
bool fit_mode(double rho, double c, double alpha, double f0, double qc,
              const std::vector<double> &ts, double &M_R, double &tau)
{
    if (c == 0.0) { M_R = 0.0; tau = 0.0; return true; }
    if (alpha <= 0.0 || ts.empty()) { M_R = rho * c * c; tau = 0.0; return true; }
    const double w = 2.0 * kPi * f0;
    const double Q = qc * w / (2.0 * c * alpha);
    double A = 0.0, B = 0.0;
    for (double t : ts) {
        const double x = w * t;
        A += x / (1.0 + x * x);
        B += x * x / (1.0 + x * x);
    }
    const double den = Q * A - B;
    if (!(den > 0.0)) return false;
    tau = 1.0 / den;
    std::complex<double> m(1.0, 0.0);
    for (double t : ts) {
        const std::complex<double> ix(0.0, w * t);
        m += tau * ix / (1.0 + ix);
    }
    const double re = (1.0 / std::sqrt(m)).real();
    M_R = rho * c * c * re * re;
    return true;
}

// CPML (a, b) at doubled position pos2 = 2s (+1 for half points).
void cpml_ab(int n, int P, double dx, double dt, double f0, double R, double cmax, int pos2,
             double &a, double &b)
{
    a = 0.0;
    b = 0.0;
    if (P <= 0) return;
    const double lo = (2.0 * P - pos2) / (2.0 * P);
    const double hi = (pos2 - 2.0 * (n - 1 - P)) / (2.0 * P);
    double xi = std::max(lo, hi);
    if (!(xi > 0.0)) return;
    xi = std::min(xi, 1.0);
    const double d0 = -3.0 * cmax * std::log(R) / (2.0 * P * dx);
    const double d = d0 * xi * xi;
    const double al = kPi * f0 * (1.0 - xi);
    b = std::exp(-(d + al) * dt);
    a = (d + al > 0.0) ? d * (b - 1.0) / (d + al) : 0.0;
}

double envelope(int env, int n_cycles, double f0, double t)
{
    if (env == BVF_ENV_BURST) return (t >= 0.0 && t < n_cycles / f0) ? 1.0 : 0.0;
    if (env == BVF_ENV_RAMP_CW) {
        if (t < 0.0) return 0.0;
        if (t < 1.0 / f0) return 0.5 * (1.0 - std::cos(kPi * f0 * t));
        return 1.0;
    }
    return 0.0;
}

// First element of state array `which`; its elements are field_stride apart.
// v and sigma: plain arrays; memory variable (l, c): element mem_index(l, c, q).
void *field_ptr(bvf_ctx *c, int which)
{
    if (which < BVF_FIELD_MEM0)
        return static_cast<char *>(c->fields) + (size_t)which * c->fstride * c->es;
    const int l = (which - BVF_FIELD_MEM0) / 6, cc = (which - BVF_FIELD_MEM0) % 6;
    return static_cast<char *>(c->fields) +
           ((size_t)BVF_FIELD_MEM0 * c->fstride + mem_index(l, cc, 0, c->fstride, c->L)) * c->es;
}
size_t field_stride(const bvf_ctx *c, int which)
{
    return which < BVF_FIELD_MEM0 ? 1 : (size_t)c->L;
}

// storage scale of state array `which` (physical value = stored value * scale)
double field_scale(const bvf_ctx *c, int which)
{
    if (which < BVF_FIELD_SXX) return c->s_v;
    if (which < BVF_FIELD_MEM0) return c->s_sig;
    return c->s_r;
}

cudaError_t next_event(bvf_ctx *c, cudaEvent_t *out)
{
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        c->ev_pool.push_back(e);
    }
    *out = c->ev_pool[c->ev_used++];
    return cudaSuccess;
}

// Sum the recorded event pairs into the accumulators and recycle the events.
cudaError_t drain_events(bvf_ctx *c)
{
    for (int kind = 0; kind < 2; ++kind) {
        std::vector<cudaEvent_t> &v = kind ? c->ev_str : c->ev_vel;
        for (size_t i = 0; i + 1 < v.size(); i += 2) {
            cudaError_t r = cudaEventSynchronize(v[i + 1]);
            if (r != cudaSuccess) return r;
            float ms = 0.0f;
            r = cudaEventElapsedTime(&ms, v[i], v[i + 1]);
            if (r != cudaSuccess) return r;
            (kind ? c->str_ms : c->vel_ms) += ms;
            (kind ? c->str_n : c->vel_n) += 1;
        }
        v.clear();
    }
    c->ev_used = 0;
    return cudaSuccess;
}

// cuTensorMapEncodeTiled from the driver (no link-time dependency on libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }
    return fn;
}

// 3-D map of an nx*ny*nz array (x fastest) with a bx x by x 1 box; points
// outside the array read as zero.
bool encode_map(CUtensorMap *m, void *base, int nx, int ny, int nz, CUtensorMapDataType type,
                size_t es, unsigned bx, unsigned by)
{
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    const size_t row = (size_t)nx * es;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)row, (cuuint64_t)row * ny};
    const cuuint32_t box[3] = {bx, by, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, type, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor maps of the TMA-fed kernels.  They need state rows that are whole
// multiples of 16 bytes in both storages and an even nx for the voxel pairs
// (nx % 8 == 0; the index is read from its padded copy when nx % 16 != 0) and
// at most 2 SLS mechanisms; other grids use the direct kernels.
void setup_maps(bvf_ctx *c)
{
    c->tma = false;
    c->tma_stress = false;
    const int nx = c->g.nx, ny = c->g.ny, nz = c->g.nz;
    if (nx % 8 != 0 || c->L > 2 || std::getenv("BVF_NO_TMA")) return;
    const auto ST = c->h16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const auto U8 = CU_TENSOR_MAP_DATA_TYPE_UINT8;
    const size_t es = c->es;
    const unsigned bw = 32 + 2 * (unsigned)(16 / es);   // halo'd box width: 16 bytes each side
    auto fld = [&](int f) { return field_ptr(c, f); };
    // the padded index copy is mapped over its whole padded rows: the pad
    // bytes are zero, the value the out-of-range fill gives past nx
    const int idx_nx = c->index_p ? (int)c->index_pitch : nx;
    // the boxes of tiles th rows high: velocities th + 4 rows (stress
    // kernel), each stress array the halo its stencil reads (velocity
    // kernel), the index th + 1 rows
    auto encode_for = [&](unsigned th, StressTmaMaps &sm, VelocityTmaMaps &vm) {
        bool ok = true;
        for (int v = 0; v < 3; ++v)
            ok = ok && encode_map(&sm.v[v], fld(BVF_FIELD_VX + v), nx, ny, nz, ST, es, bw, th + 4);
        const unsigned w6[6] = {bw, 32, 32, bw, bw, 32},
                       h6[6] = {th, th + 4, th, th + 4, th, th + 4};
        for (int g6 = 0; g6 < 6; ++g6)
            ok = ok && encode_map(&vm.sg[g6], fld(BVF_FIELD_SXX + g6), nx, ny, nz, ST, es, w6[g6],
                                  h6[g6]);
        ok = ok && encode_map(&sm.idx, c->index_p ? c->index_p : c->index, idx_nx, ny, nz, U8, 1,
                              48, th + 1);
        vm.idx = sm.idx;
        return ok;
    };
    bool ok = encode_for(8, c->smaps, c->vmaps);
    if (c->L == 2)
        ok = ok && encode_for(4, c->smaps_x[0], c->vmaps_x[0]) &&
             encode_for(16, c->smaps_x[1], c->vmaps_x[1]);
    c->tma = ok;
    // BVF_STRESS_TMA=0 keeps the stress kernel on the direct path
    const char *st = std::getenv("BVF_STRESS_TMA");
    c->tma_stress = ok && !(st && st[0] == '0');
}

bool tile_valid(const bvf_tile &t)
{
    auto rows_ok = [](int r) { return r == 0 || r == 4 || r == 8 || r == 16; };
    return rows_ok(t.stress_rows) && rows_ok(t.velocity_rows) && t.kchunk >= 0;
}

// The rows each TMA kernel uses: the context's choice, else 8 for the stress
// and 16 for the velocity kernel (the faster heights on the bench workload);
// 8 for both without two SLS mechanisms.
bvf_tile effective_tile(const bvf_ctx *c)
{
    bvf_tile t{8, 8, c->kchunk};
    if (c->L != 2) return t;
    t.stress_rows = c->tile.stress_rows ? c->tile.stress_rows : 8;
    t.velocity_rows = c->tile.velocity_rows ? c->tile.velocity_rows : 16;
    return t;
}

AcParams make_params(bvf_ctx *c)
{
    AcParams p{};
    p.nx = c->g.nx;
    p.ny = c->g.ny;
    p.nz = c->g.nz;
    p.P = c->P;
    p.W = c->W;
    p.L = c->L;
    p.n_mat = (int)c->table.size();
    p.h16 = c->h16;
    // storage scales folded into the constants (all 1 for float storage, so
    // the float path computes exactly dt, 0.5 and cb)
    p.dt = (float)(c->g.dt * c->s_v / c->s_sig);
    p.dtv = (float)(c->g.dt * c->s_sig / c->s_v);
    p.rh = (float)(0.5 * c->s_r / c->s_v);
    p.inv_dx = (float)(1.0 / c->g.dx);
    p.Lf = (float)c->L;
    for (int l = 0; l < c->L; ++l) {
        const double h = c->g.dt / (2.0 * c->tau_sigma[l]);
        p.ca[l] = (float)((1.0 - h) / (1.0 + h));
        p.ncb[l] = -(float)((c->g.dt / c->tau_sigma[l]) / (1.0 + h) * (c->s_v / c->s_r));
    }
    p.idx = c->index;
    p.lut = c->lut;
    p.buoy = c->buoy;
    p.vx = field_ptr(c, BVF_FIELD_VX);
    p.vy = field_ptr(c, BVF_FIELD_VY);
    p.vz = field_ptr(c, BVF_FIELD_VZ);
    p.sxx = field_ptr(c, BVF_FIELD_SXX);
    p.syy = field_ptr(c, BVF_FIELD_SYY);
    p.szz = field_ptr(c, BVF_FIELD_SZZ);
    p.sxy = field_ptr(c, BVF_FIELD_SXY);
    p.sxz = field_ptr(c, BVF_FIELD_SXZ);
    p.syz = field_ptr(c, BVF_FIELD_SYZ);
    p.mem = field_ptr(c, BVF_FIELD_MEM0);
    p.fstride = c->fstride;
    p.psx = c->psi;
    p.psy = c->psi + kNumCpmlSlots * c->slab_x;
    p.psz = c->psi + kNumCpmlSlots * (c->slab_x + c->slab_y);
    p.pml = c->pml;
    p.nmax = c->nmax;
    p.src = c->src;
    p.k_src = c->k_src;
    p.peak = c->peak;
    p.dftC = c->dftC;
    p.dftS = c->dftS;
    p.flag = c->flag;
    p.kchunk = c->kchunk;
    const bvf_tile t = effective_tile(c);
    p.tile_y = t.stress_rows;
    p.tile_yv = t.velocity_rows;
    p.wait_limit = tma::kWaitLimit;
    p.hold = 0;
    p.hold_plane = -1;
    p.src_scale = (float)(2.0 * c->c0 * c->g.dt / c->g.dx / c->s_sig);
    return p;
}

// Source and capture parameters of the update n -> n+1 (source sampled at
// (n + 1/2) dt, capture of p at (n + 1) dt).
StepParam step_param(const bvf_ctx *c, const bvf_capture &cp, long long n)
{
    const double w = 2.0 * kPi * c->ph.f0, dt = c->g.dt;
    const double t = (n + 0.5) * dt;
    const double env = c->have_source ? envelope(c->envelope, c->n_cycles, c->ph.f0, t) : 0.0;
    const long long step = n + 1;
    const bool peak = cp.peak_from >= 0 && step >= cp.peak_from;
    const bool dft = cp.dft_steps > 0 && step >= cp.dft_start &&
                     step < (long long)cp.dft_start + cp.dft_steps;
    StepParam q{};
    q.flags = ((c->have_source && env != 0.0) ? 1 : 0) | (peak ? 2 : 0) | (dft ? 4 : 0);
    q.src_ws = (float)(env * std::sin(w * t));
    q.src_wc = (float)(env * std::cos(w * t));
    q.cw = std::cos(w * step * dt);
    q.sw = std::sin(w * step * dt);
    return q;
}

// FP64 DFT sums of a context, allocated and zeroed on first use
int ensure_dft(bvf_ctx *c, cudaStream_t s)
{
    if (c->dftC) return BVF_OK;
    CK(cudaMalloc(&c->dftC, c->N * sizeof(double)), "dft buffers");
    CK(cudaMalloc(&c->dftS, c->N * sizeof(double)), "dft buffers");
    CK(cudaMemsetAsync(c->dftC, 0, c->N * sizeof(double), s), "dft buffers");
    CK(cudaMemsetAsync(c->dftS, 0, c->N * sizeof(double), s), "dft buffers");
    return BVF_OK;
}

// Wall-clock budget of a run call.  Every kBudgetChunk steps the call records
// an event, waits for the event of the chunk before (so at most two chunks
// are queued ahead of the host) and compares the time since the call began
// with the budget.  Without a budget nothing is recorded or waited for.
constexpr int kBudgetChunk = 32;
struct Budget {
    bvf_ctx *c;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    int slot = 0;
    bool armed[2] = {false, false};
    // before step `it` of the call: BVF_OK to go on, BVF_E_TIMEOUT (after the
    // queued work has finished) once the budget is spent
    int check(int it, cudaStream_t s, const char *what)
    {
        if (!(c->budget_s > 0.0) || it == 0 || it % kBudgetChunk) return BVF_OK;
        for (int b = 0; b < 2; ++b)
            if (!c->budget_ev[b]) CK(cudaEventCreateWithFlags(&c->budget_ev[b], cudaEventDisableTiming),
                                      "time budget");
        CK(cudaEventRecord(c->budget_ev[slot], s), "time budget");
        armed[slot] = true;
        slot ^= 1;
        if (armed[slot]) CK(cudaEventSynchronize(c->budget_ev[slot]), "time budget");
        const double el =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el < c->budget_s) return BVF_OK;
        CK(cudaStreamSynchronize(s), "time budget");
        char buf[200];
        std::snprintf(buf, sizeof buf,
                      "%s: wall-clock budget of %.3g s spent after %d steps of this call "
                      "(%.3g s); the context holds the state after them",
                      what, c->budget_s, it, el);
        return fail(c, BVF_E_TIMEOUT, buf);
    }
};

// Snapshot layout of bvf_state_save: a 256-byte header, then the state
// arrays, CPML memories, peak map, the two FP64 DFT sums and the device flag,
// each section starting on a 256-byte boundary.
constexpr uint64_t kStateMagic = 0x3176617473667662ull;   // "bvfstav1"
struct StateHeader {
    uint64_t magic;
    int32_t version, nx, ny, nz, L, h16, has_dft, pad;
    int64_t steps, dft_count;
    double dx, dt, f0;
    uint64_t bytes;
    char reserved[256 - 8 - 9 * 4 - 2 * 8 - 3 * 8 - 8];
};
static_assert(sizeof(StateHeader) == 256, "state header is 256 bytes");

struct StateSections {
    size_t fields, psi, peak, dft, flag, total;
    size_t off_fields, off_psi, off_peak, off_C, off_S, off_flag;
};
StateSections state_sections(const bvf_ctx *c)
{
    auto up = [](size_t n) { return (n + 255) & ~(size_t)255; };
    StateSections t{};
    t.fields = (9 + 6 * (size_t)c->L) * c->fstride * c->es;
    t.psi = kNumCpmlSlots * (c->slab_x + c->slab_y + c->slab_z) * sizeof(float);
    t.peak = c->N * sizeof(float);
    t.dft = c->N * sizeof(double);
    t.flag = sizeof(int);
    t.off_fields = 256;
    t.off_psi = t.off_fields + up(t.fields);
    t.off_peak = t.off_psi + up(t.psi);
    t.off_C = t.off_peak + up(t.peak);
    t.off_S = t.off_C + up(t.dft);
    t.off_flag = t.off_S + up(t.dft);
    t.total = t.off_flag + 256;
    return t;
}

}  // namespace

extern "C" {

int bvf_version(void) { return BVF_VERSION; }

double bvf_courant_limit(void) { return 6.0 / (7.0 * std::sqrt(3.0)); }

const char *bvf_strerror(int code)
{
    switch (code) {
    case BVF_OK: return "ok";
    case BVF_E_ARG: return "invalid argument or call order";
    case BVF_E_CFL: return "time step above the stability limit";
    case BVF_E_MATERIAL: return "invalid material or material index";
    case BVF_E_NOMEM: return "device allocation failed";
    case BVF_E_CUDA: return "CUDA error";
    case BVF_E_UNSTABLE: return "non-finite pressure detected";
    case BVF_E_TIMEOUT: return "wall-clock budget of the call spent";
    default: return "unknown status";
    }
}

const char *bvf_last_error(const bvf_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_last_error.c_str();
}

void bvf_destroy(bvf_ctx *c)
{
    if (!c) return;
    void *bufs[] = {c->fields, c->psi, c->peak, c->dftC, c->dftS, c->index, c->lut, c->buoy,
                    c->pml, c->src, c->flag, c->scratch_u, c->T2, c->Q, c->cemf, c->tlut,
                    c->kface, c->index_p, c->h_index_d, c->h_peak_d, c->h_T_d, c->h_Tmax_d,
                    c->h_amp_d, c->h_cem_d};
    for (void *b : bufs)
        if (b) cudaFree(b);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : c->budget_ev)
        if (e) cudaEventDestroy(e);
    if (c->fork_ev) cudaEventDestroy(c->fork_ev);
    if (c->join_ev) cudaEventDestroy(c->join_ev);
    if (c->side) cudaStreamDestroy(c->side);
    delete c;
}

int bvf_create(const bvf_grid *grid, const bvf_physics *phys, bvf_ctx **out)
{
    bvf_ctx *c = nullptr;
    if (!out) return fail(nullptr, BVF_E_ARG, "bvf_create: out is NULL");
    *out = nullptr;
    if (!grid || !phys) return fail(nullptr, BVF_E_ARG, "bvf_create: NULL grid or physics");
    const bvf_grid &g = *grid;
    if (g.nx < 1 || g.ny < 1 || g.nz < 1 || !(g.dx > 0.0) || !(g.dt > 0.0) || g.n_pml < 0)
        return fail(nullptr, BVF_E_ARG, "bvf_create: bad grid sizes or spacing");
    if (g.n_pml > 0 && (g.nx < 2 * g.n_pml + 2 || g.ny < 2 * g.n_pml + 2 ||
                        g.nz < 2 * g.n_pml + 2 || !(g.pml_R > 0.0 && g.pml_R < 1.0)))
        return fail(nullptr, BVF_E_ARG, "bvf_create: grid too small for the CPML or bad pml_R");
    if (phys->n_sls < 0 || phys->n_sls > BVF_MAX_SLS || !(phys->f0 > 0.0) || !(phys->qc > 0.0))
        return fail(nullptr, BVF_E_ARG, "bvf_create: bad physics (f0, qc or n_sls)");
    if ((double)g.nx * g.ny * g.nz >= 2147483648.0)
        return fail(nullptr, BVF_E_ARG, "bvf_create: grid of 2^31 voxels or more");
    if ((phys->storage != BVF_STORAGE_F32 && phys->storage != BVF_STORAGE_F16) ||
        !(phys->p_ref >= 0.0) || std::isinf(phys->p_ref))
        return fail(nullptr, BVF_E_ARG, "bvf_create: bad storage or p_ref");

    c = new (std::nothrow) bvf_ctx;
    if (!c) return fail(nullptr, BVF_E_NOMEM, "bvf_create: host allocation failed");
    c->g = g;
    c->ph = *phys;
    c->L = phys->n_sls;
    c->N = (size_t)g.nx * g.ny * g.nz;
    c->fstride = (c->N + 63) & ~(size_t)63;
    c->h16 = phys->storage == BVF_STORAGE_F16;
    c->es = c->h16 ? 2 : 4;
    if (c->h16) {
        // sigma / p_ref, v rho_w c_w / p_ref; memory variables r (a stress
        // rate) times 8 dt / p_ref, i.e. r' = r / S_v and S_r = S_v Z_w / (8 dt)
        const double zw = 1.5e6;
        c->s_sig = phys->p_ref > 0.0 ? phys->p_ref : 1e5;
        c->s_v = c->s_sig / zw;
        c->s_r = c->s_v * zw / (8.0 * g.dt);
    }
    c->P = g.n_pml;
    c->W = g.n_pml > 0 ? 2 * g.n_pml + 1 : 0;
    c->nmax = std::max(g.nx, std::max(g.ny, g.nz));
    c->slab_x = (size_t)g.nz * g.ny * c->W;
    c->slab_y = (size_t)g.nz * c->W * g.nx;
    c->slab_z = (size_t)c->W * g.ny * g.nx;
    c->tau_sigma = relaxation_times(phys->f0, c->L);
    if (const char *kc = std::getenv("BVF_KCHUNK")) c->kchunk = std::max(0, std::atoi(kc));

    auto cleanup = [&](int code) { bvf_destroy(c); return code; };
    cudaError_t e;
    const size_t nf = 9 + 6 * (size_t)c->L;
    if ((e = cudaMalloc(&c->fields, nf * c->fstride * c->es)) != cudaSuccess)
        return cleanup(cuda_fail(nullptr, e, "bvf_create: fields"));
    const size_t npsi = kNumCpmlSlots * (c->slab_x + c->slab_y + c->slab_z);
    if (npsi && (e = cudaMalloc(&c->psi, npsi * sizeof(float))) != cudaSuccess)
        return cleanup(cuda_fail(nullptr, e, "bvf_create: cpml"));
    if ((e = cudaMalloc(&c->peak, c->N * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&c->index, c->N)) != cudaSuccess ||
        (e = cudaMalloc(&c->lut, BVF_MAX_MATERIALS * sizeof(MatCoef))) != cudaSuccess ||
        (e = cudaMalloc(&c->buoy, (size_t)BVF_MAX_MATERIALS * BVF_MAX_MATERIALS * sizeof(float))) !=
            cudaSuccess ||
        (e = cudaMalloc(&c->pml, 6 * (size_t)c->nmax * sizeof(float2))) != cudaSuccess ||
        (e = cudaMalloc(&c->src, (size_t)g.nx * g.ny * sizeof(float2))) != cudaSuccess ||
        (e = cudaMalloc(&c->flag, sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&c->scratch_u, sizeof(unsigned))) != cudaSuccess)
        return cleanup(cuda_fail(nullptr, e, "bvf_create: buffers"));
    if ((e = cudaMemset(c->fields, 0, nf * c->fstride * c->es)) != cudaSuccess ||
        (npsi && (e = cudaMemset(c->psi, 0, npsi * sizeof(float))) != cudaSuccess) ||
        (e = cudaMemset(c->peak, 0, c->N * sizeof(float))) != cudaSuccess ||
        (e = cudaMemset(c->index, 0, c->N)) != cudaSuccess ||
        (e = cudaMemset(c->pml, 0, 6 * (size_t)c->nmax * sizeof(float2))) != cudaSuccess ||
        (e = cudaMemset(c->flag, 0, sizeof(int))) != cudaSuccess ||
        (e = cudaDeviceSynchronize()) != cudaSuccess)
        return cleanup(cuda_fail(nullptr, e, "bvf_create: zero fill"));
    if (g.nx % 8 == 0 && g.nx % 16 != 0) {
        c->index_pitch = (size_t)(g.nx + 15) / 16 * 16;
        const size_t bytes = c->index_pitch * g.ny * g.nz;
        if ((e = cudaMalloc(&c->index_p, bytes)) != cudaSuccess ||
            (e = cudaMemset(c->index_p, 0, bytes)) != cudaSuccess ||
            (e = cudaDeviceSynchronize()) != cudaSuccess)
            return cleanup(cuda_fail(nullptr, e, "bvf_create: padded index"));
    }
    setup_maps(c);
    *out = c;
    return BVF_OK;
}

int bvf_set_materials(bvf_ctx *c, const uint8_t *d_index, const bvf_material *h_table, int n_mat)
{
    if (!c) return fail(nullptr, BVF_E_ARG, "bvf_set_materials: NULL context");
    if (!d_index || !h_table || n_mat < 1 || n_mat > BVF_MAX_MATERIALS)
        return fail(c, BVF_E_ARG, "bvf_set_materials: NULL pointer or n_mat out of [1, 256]");
    std::vector<MatDerived> der(n_mat);
    double cmax_unrelaxed = 0.0, cmax = 0.0;
    for (int m = 0; m < n_mat; ++m) {
        const bvf_material &r = h_table[m];
        char buf[160];
        if (!(r.rho > 0.0) || !(r.cL > 0.0) || !(r.cS >= 0.0) || !(r.alphaL >= 0.0) ||
            !(r.alphaS >= 0.0)) {
            std::snprintf(buf, sizeof buf, "material %d: need rho > 0, cL > 0, cS >= 0, alpha >= 0", m);
            return fail(c, BVF_E_MATERIAL, buf);
        }
        if (!(4.0 * r.cS * r.cS <= 3.0 * r.cL * r.cL)) {
            std::snprintf(buf, sizeof buf, "material %d: Poisson ratio below -1 (cS > 0.866 cL)", m);
            return fail(c, BVF_E_MATERIAL, buf);
        }
        if (!(r.k_th > 0.0) || !(r.c_th > 0.0) || !(r.perf >= 0.0) ||
            !(r.heat_frac >= 0.0 && r.heat_frac <= 1.0)) {
            std::snprintf(buf, sizeof buf, "material %d: bad thermal constants", m);
            return fail(c, BVF_E_MATERIAL, buf);
        }
        MatDerived &d = der[m];
        if (!fit_mode(r.rho, r.cL, r.alphaL, c->ph.f0, c->ph.qc, c->tau_sigma, d.piR, d.tauP) ||
            !fit_mode(r.rho, r.cS, r.alphaS, c->ph.f0, c->ph.qc, c->tau_sigma, d.muR, d.tauS)) {
            std::snprintf(buf, sizeof buf,
                          "material %d: Q = qc w/(2 c alpha) below what %d SLS mechanisms reach", m,
                          c->L);
            return fail(c, BVF_E_MATERIAL, buf);
        }
        cmax = std::max(cmax, r.cL);
        cmax_unrelaxed = std::max(cmax_unrelaxed, std::sqrt(d.piR * (1.0 + c->L * d.tauP) / r.rho));
        cmax_unrelaxed = std::max(cmax_unrelaxed, std::sqrt(d.muR * (1.0 + c->L * d.tauS) / r.rho));
    }
    const double S = cmax_unrelaxed * c->g.dt / c->g.dx;
    if (S > bvf_courant_limit()) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "Courant number %.5f above the limit %.5f", S,
                      bvf_courant_limit());
        return fail(c, BVF_E_CFL, buf);
    }
    // device LUT
    std::vector<MatCoef> lut(n_mat);
    for (int m = 0; m < n_mat; ++m) {
        const MatDerived &d = der[m];
        MatCoef &k = lut[m];
        k.rho = (float)h_table[m].rho;
        k.piU = (float)(d.piR * (1.0 + c->L * d.tauP));
        k.piT = (float)(d.piR * d.tauP);
        k.mu2U = (float)(2.0 * d.muR * (1.0 + c->L * d.tauS));
        k.mu2T = (float)(2.0 * d.muR * d.tauS);
        k.inv_mu = d.muR > 0.0 ? (float)(1.0 / d.muR) : INFINITY;
        k.tauS = (float)d.tauS;
        k.pad = 0.0f;
    }
    // CPML profile at integer (h = 0) and half (h = 1) points of each axis
    std::vector<float2> pml(6 * (size_t)c->nmax, make_float2(0.0f, 0.0f));
    const int nax[3] = {c->g.nx, c->g.ny, c->g.nz};
    for (int ax = 0; ax < 3; ++ax)
        for (int h = 0; h < 2; ++h)
            for (int s = 0; s < nax[ax]; ++s) {
                double a, b;
                cpml_ab(nax[ax], c->P, c->g.dx, c->g.dt, c->ph.f0, c->g.pml_R, cmax, 2 * s + h, a, b);
                pml[((size_t)ax * 2 + h) * c->nmax + s] = make_float2((float)a, (float)b);
            }
    CK(cudaMemcpy(c->index, d_index, c->N, cudaMemcpyDeviceToDevice), "copy index");
    if (c->index_p)
        CK(cudaMemcpy2D(c->index_p, c->index_pitch, c->index, c->g.nx, c->g.nx,
                        (size_t)c->g.ny * c->g.nz, cudaMemcpyDeviceToDevice),
           "copy padded index");
    CK(cudaMemcpy(c->lut, lut.data(), n_mat * sizeof(MatCoef), cudaMemcpyHostToDevice), "copy lut");
    // buoyancy at a velocity point between cells of materials a and b: 2 / (rho_a + rho_b)
    std::vector<float> buoy((size_t)n_mat * n_mat);
    for (int a = 0; a < n_mat; ++a)
        for (int b = 0; b < n_mat; ++b)
            buoy[(size_t)a * n_mat + b] = (float)(2.0 / (h_table[a].rho + h_table[b].rho));
    CK(cudaMemcpy(c->buoy, buoy.data(), buoy.size() * sizeof(float), cudaMemcpyHostToDevice),
       "copy buoyancy");
    CK(cudaMemcpy(c->pml, pml.data(), pml.size() * sizeof(float2), cudaMemcpyHostToDevice), "copy pml");
    CK(cudaMemset(c->scratch_u, 0, sizeof(unsigned)), "memset");
    CK(launch_index_max(c->index, c->N, c->scratch_u, 0), "index scan");
    c->launches++;
    unsigned mx = 0;
    CK(cudaMemcpy(&mx, c->scratch_u, sizeof(unsigned), cudaMemcpyDeviceToHost), "index scan");
    if ((int)mx >= n_mat) {
        char buf[120];
        std::snprintf(buf, sizeof buf, "material index %u >= table size %d", mx, n_mat);
        c->have_materials = false;
        return fail(c, BVF_E_MATERIAL, buf);
    }
    c->table.assign(h_table, h_table + n_mat);
    c->derived = der;
    c->courant = S;
    c->have_materials = true;
    return BVF_OK;
}

int bvf_set_source(bvf_ctx *c, int k_plane, const float *d_plane, double c0, int env,
                   int n_cycles, void *stream)
{
    if (!c) return fail(nullptr, BVF_E_ARG, "bvf_set_source: NULL context");
    if (env == BVF_ENV_NONE) {
        c->have_source = false;
        c->envelope = BVF_ENV_NONE;
        return BVF_OK;
    }
    if (!d_plane || k_plane < 0 || k_plane >= c->g.nz || !(c0 > 0.0) ||
        (env != BVF_ENV_BURST && env != BVF_ENV_RAMP_CW) || (env == BVF_ENV_BURST && n_cycles < 1))
        return fail(c, BVF_E_ARG, "bvf_set_source: bad plane, speed, envelope or cycle count");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(c->src, d_plane, (size_t)c->g.nx * c->g.ny * sizeof(float2),
                       cudaMemcpyDeviceToDevice, s), "copy source plane");
    c->k_src = k_plane;
    c->c0 = c0;
    c->envelope = env;
    c->n_cycles = n_cycles;
    c->have_source = true;
    return BVF_OK;
}

int bvf_reset(bvf_ctx *c, void *stream)
{
    if (!c) return fail(nullptr, BVF_E_ARG, "bvf_reset: NULL context");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nf = 9 + 6 * (size_t)c->L;
    CK(cudaMemsetAsync(c->fields, 0, nf * c->fstride * c->es, s), "reset");
    const size_t npsi = kNumCpmlSlots * (c->slab_x + c->slab_y + c->slab_z);
    if (npsi) CK(cudaMemsetAsync(c->psi, 0, npsi * sizeof(float), s), "reset");
    CK(cudaMemsetAsync(c->peak, 0, c->N * sizeof(float), s), "reset");
    if (c->dftC) {
        CK(cudaMemsetAsync(c->dftC, 0, c->N * sizeof(double), s), "reset");
        CK(cudaMemsetAsync(c->dftS, 0, c->N * sizeof(double), s), "reset");
    }
    CK(cudaMemsetAsync(c->flag, 0, sizeof(int), s), "reset");
    c->dft_count = 0;
    c->steps = 0;
    return BVF_OK;
}

int bvf_run_acoustic(bvf_ctx *c, int n_steps, const bvf_capture *cap, void *stream)
{
    if (!c) return fail(nullptr, BVF_E_ARG, "bvf_run_acoustic: NULL context");
    if (!c->have_materials) return fail(c, BVF_E_ARG, "bvf_run_acoustic: call bvf_set_materials first");
    if (n_steps < 0) return fail(c, BVF_E_ARG, "bvf_run_acoustic: negative step count");
    cudaStream_t s = (cudaStream_t)stream;
    bvf_capture cp{-1, 0, 0};
    if (cap) cp = *cap;
    if (cp.dft_steps < 0) return fail(c, BVF_E_ARG, "bvf_run_acoustic: negative dft_steps");
    if (cp.dft_steps > 0) {
        const int rc = ensure_dft(c, s);
        if (rc != BVF_OK) return rc;
    }
    AcParams p = make_params(c);
    Budget budget{c};
    for (int it = 0; it < n_steps; ++it) {
        const int rb = budget.check(it, s, "bvf_run_acoustic");
        if (rb != BVF_OK) return rb;
        p.st = step_param(c, cp, c->steps);
        if (c->hold == 1 || c->hold == 2) {  // test hook: this one step only
            p.hold = c->hold;
            p.hold_plane = c->hold_plane;
            p.wait_limit = c->hold_limit ? c->hold_limit : tma::kWaitLimit;
            c->hold = 0;
        } else {
            p.hold = 0;
            p.wait_limit = tma::kWaitLimit;
        }
        // the tensor maps whose boxes match each kernel's tile height
        const int tv = p.tile_yv == 4 ? 0 : (p.tile_yv == 16 ? 1 : -1);
        const int ts = p.tile_y == 4 ? 0 : (p.tile_y == 16 ? 1 : -1);
        const VelocityTmaMaps &vm = tv < 0 ? c->vmaps : c->vmaps_x[tv];
        const StressTmaMaps &sm = ts < 0 ? c->smaps : c->smaps_x[ts];
        auto vel = [&]() { return c->tma ? launch_velocity_tma(p, vm, s) : launch_velocity(p, s); };
        auto str = [&]() { return c->tma_stress ? launch_stress_tma(p, sm, s) : launch_stress(p, s); };
        if (c->timing) {
            if (c->ev_used + 3 > 3072) CK(drain_events(c), "kernel timing");
            cudaEvent_t e0, e1, e2;
            CK(next_event(c, &e0), "kernel timing");
            CK(next_event(c, &e1), "kernel timing");
            CK(next_event(c, &e2), "kernel timing");
            CK(cudaEventRecord(e0, s), "kernel timing");
            CK(vel(), "velocity kernel");
            CK(cudaEventRecord(e1, s), "kernel timing");
            CK(str(), "stress kernel");
            CK(cudaEventRecord(e2, s), "kernel timing");
            c->ev_vel.push_back(e0);
            c->ev_vel.push_back(e1);
            c->ev_str.push_back(e1);
            c->ev_str.push_back(e2);
        } else {
            CK(vel(), "velocity kernel");
            CK(str(), "stress kernel");
        }
        c->launches += 2;
        c->dft_count += (p.st.flags & kStepDft) ? 1 : 0;
        c->steps++;
    }
    return BVF_OK;
}

int bvf_synchronize(bvf_ctx *c, void *stream)
{
    if (!c) return fail(nullptr, BVF_E_ARG, "bvf_synchronize: NULL context");
    CK(cudaStreamSynchronize((cudaStream_t)stream), "synchronize");
    int f = 0;
    CK(cudaMemcpy(&f, c->flag, sizeof(int), cudaMemcpyDeviceToHost), "read flag");
    if (f & 2) return fail(c, BVF_E_CUDA, "a TMA copy did not complete within its wait limit");
    if (f) return fail(c, BVF_E_UNSTABLE, "non-finite pressure detected");
    return BVF_OK;
}

int bvf_get_field(bvf_ctx *c, int which, float *d_out, void *stream)
{
    if (!c || !d_out || which < 0 || which >= 9 + 6 * c->L)
        return fail(c, BVF_E_ARG, "bvf_get_field: bad context, pointer or field id");
    if (!c->h16 && field_stride(c, which) == 1)
        CK(cudaMemcpyAsync(d_out, field_ptr(c, which), c->N * sizeof(float),
                           cudaMemcpyDeviceToDevice, (cudaStream_t)stream), "get field");
    else {
        CK(launch_field_out(field_ptr(c, which), c->h16, field_stride(c, which),
                            (float)field_scale(c, which), d_out, c->N, (cudaStream_t)stream),
           "get field");
        c->launches++;
    }
    return BVF_OK;
}

int bvf_set_field(bvf_ctx *c, int which, const float *d_in, void *stream)
{
    if (!c || !d_in || which < 0 || which >= 9 + 6 * c->L)
        return fail(c, BVF_E_ARG, "bvf_set_field: bad context, pointer or field id");
    if (!c->h16 && field_stride(c, which) == 1)
        CK(cudaMemcpyAsync(field_ptr(c, which), d_in, c->N * sizeof(float),
                           cudaMemcpyDeviceToDevice, (cudaStream_t)stream), "set field");
    else {
        CK(launch_field_in(d_in, c->h16, field_stride(c, which),
                           (float)(1.0 / field_scale(c, which)), field_ptr(c, which), c->N,
                           (cudaStream_t)stream), "set field");
        c->launches++;
    }
    return BVF_OK;
}

int bvf_get_pressure(bvf_ctx *c, float *d_out, void *stream)
{
    if (!c || !d_out) return fail(c, BVF_E_ARG, "bvf_get_pressure: NULL argument");
    CK(launch_pressure(field_ptr(c, BVF_FIELD_SXX), field_ptr(c, BVF_FIELD_SYY),
                       field_ptr(c, BVF_FIELD_SZZ), c->h16, (float)c->s_sig, d_out, c->N,
                       (cudaStream_t)stream),
       "pressure kernel");
    c->launches++;
    return BVF_OK;
}

int bvf_get_peak(bvf_ctx *c, float *d_out, void *stream)
{
    if (!c || !d_out) return fail(c, BVF_E_ARG, "bvf_get_peak: NULL argument");
    if (!c->h16)
        CK(cudaMemcpyAsync(d_out, c->peak, c->N * sizeof(float), cudaMemcpyDeviceToDevice,
                           (cudaStream_t)stream), "get peak");
    else {
        CK(launch_scale_copy(c->peak, (float)c->s_sig, d_out, c->N, (cudaStream_t)stream),
           "get peak");
        c->launches++;
    }
    return BVF_OK;
}

int bvf_get_amp_phase(bvf_ctx *c, double *d_amp, double *d_phase, void *stream)
{
    if (!c) return fail(nullptr, BVF_E_ARG, "bvf_get_amp_phase: NULL context");
    if (!c->dftC || c->dft_count <= 0)
        return fail(c, BVF_E_ARG, "bvf_get_amp_phase: no step was captured");
    CK(launch_amp_phase(c->dftC, c->dftS, c->N, c->dft_count, c->s_sig, d_amp, d_phase,
                        (cudaStream_t)stream), "amp/phase kernel");
    c->launches++;
    return BVF_OK;
}

int bvf_run_thermal(bvf_ctx *c, const bvf_thermal *th, const double *d_amp, float *d_T,
                    float *d_Tmax, double *d_cem43, void *stream)
{
    if (!c || !th || !d_T || !d_Tmax || !d_cem43)
        return fail(c, BVF_E_ARG, "bvf_run_thermal: NULL argument");
    if (!c->have_materials) return fail(c, BVF_E_ARG, "bvf_run_thermal: call bvf_set_materials first");
    if (th->n_on < 0 || th->n_off < 0 || !(th->dt > 0.0) || !(th->duty >= 0.0 && th->duty <= 1.0) ||
        !(th->rhob_cb >= 0.0))
        return fail(c, BVF_E_ARG, "bvf_run_thermal: bad regime");
    const int n_mat = (int)c->table.size();
    std::vector<ThermCoef> tl(n_mat);
    double dt_lim = 1e300;
    for (int m = 0; m < n_mat; ++m) {
        const bvf_material &r = c->table[m];
        tl[m].inv_rhoc = (float)(1.0 / (r.rho * r.c_th));
        tl[m].perfw = (float)(r.perf * th->rhob_cb);
        tl[m].qfac = (float)(r.heat_frac * r.alphaL / (r.rho * r.cL));
        dt_lim = std::min(dt_lim, c->g.dx * c->g.dx * r.rho * r.c_th / (6.0 * r.k_th));
    }
    if (th->dt > dt_lim)
        return fail(c, BVF_E_ARG, "bvf_run_thermal: dt above the explicit stability limit");
    cudaStream_t s = (cudaStream_t)stream;
    if (!c->T2) {
        CK(cudaMalloc(&c->T2, c->N * sizeof(float)), "thermal buffers");
        CK(cudaMalloc(&c->Q, c->N * sizeof(float)), "thermal buffers");
        CK(cudaMalloc(&c->cemf, c->N * sizeof(float)), "thermal buffers");
        CK(cudaMalloc(&c->tlut, BVF_MAX_MATERIALS * sizeof(ThermCoef)), "thermal buffers");
        CK(cudaMalloc(&c->kface, (size_t)BVF_MAX_MATERIALS * BVF_MAX_MATERIALS * sizeof(float)),
           "thermal buffers");
    }
    // harmonic-mean face conductivity of every material pair (Sec. 2.4 FTCS
    // stencil), in FP64 then rounded once
    std::vector<float> kf((size_t)n_mat * n_mat);
    for (int a = 0; a < n_mat; ++a)
        for (int b = 0; b < n_mat; ++b) {
            const double ka = c->table[a].k_th, kb = c->table[b].k_th;
            kf[(size_t)a * n_mat + b] = (ka + kb > 0.0) ? (float)(2.0 * ka * kb / (ka + kb)) : 0.0f;
        }
    // the diagonal rides with each material's coefficients: the kernels take
    // it for a voxel whose six neighbours share its material
    for (int m = 0; m < n_mat; ++m) tl[m].k = kf[(size_t)m * n_mat + m];
    CK(cudaMemsetAsync(c->cemf, 0, c->N * sizeof(float), s), "thermal buffers");
    CK(cudaMemcpyAsync(c->tlut, tl.data(), n_mat * sizeof(ThermCoef), cudaMemcpyHostToDevice, s),
       "thermal lut");
    CK(cudaMemcpyAsync(c->kface, kf.data(), kf.size() * sizeof(float), cudaMemcpyHostToDevice, s),
       "thermal face table");
    CK(launch_heat_source(c->index, c->tlut, n_mat, d_amp, th->p_scale, c->Q, c->N, s), "heat source");
    c->launches++;
    ThParams p{};
    p.nx = c->g.nx;
    p.ny = c->g.ny;
    p.nz = c->g.nz;
    p.dt = (float)th->dt;
    p.inv_dx2 = (float)(1.0 / (c->g.dx * c->g.dx));
    p.rise43 = (float)(43.0 - th->T_a);
    p.dt60 = (float)(th->dt / 60.0);
    p.idx = c->index;
    p.lut = c->tlut;
    p.kface = c->kface;
    p.n_mat = n_mat;
    p.Q = c->Q;
    p.Tmax = d_Tmax;
    p.cemf = c->cemf;
    p.cem = d_cem43;
    const int total = th->n_on + th->n_off;
    float *a = d_T, *b = c->T2;
    // TMA-fed steps where the index rows are whole multiples of 16 bytes and
    // both temperature buffers can be mapped (BVF_NO_TMA forces the direct
    // kernel); one map per temperature buffer, chosen per step
    ThermTmaMaps tmaps[2];
    bool th_tma = false;
    if (c->g.nx % 8 == 0 && !std::getenv("BVF_NO_TMA")) {
        const int nx = c->g.nx, ny = c->g.ny, nz = c->g.nz;
        const auto F32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
        th_tma = encode_map(&tmaps[0].T, d_T, nx, ny, nz, F32, 4, 40, 18) &&
                 encode_map(&tmaps[1].T, c->T2, nx, ny, nz, F32, 4, 40, 18) &&
                 encode_map(&tmaps[0].idx, c->index_p ? c->index_p : c->index,
                            c->index_p ? (int)c->index_pitch : nx, ny, nz,
                            CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, 64, 18) &&
                 encode_map(&tmaps[0].Q, c->Q, nx, ny, nz, F32, 4, 32, 16) &&
                 encode_map(&tmaps[0].Tmax, d_Tmax, nx, ny, nz, F32, 4, 32, 16) &&
                 encode_map(&tmaps[0].cemf, c->cemf, nx, ny, nz, F32, 4, 32, 16);
        tmaps[1].idx = tmaps[0].idx;
        tmaps[1].Q = tmaps[0].Q;
        tmaps[1].Tmax = tmaps[0].Tmax;
        tmaps[1].cemf = tmaps[0].cemf;
    }
    p.kz = thermal_kchunk(c->g.nx, c->g.ny, c->g.nz, th_tma, n_mat);
    // the kernels advance the rise T - T_a (see ThParams); T and T_max are
    // converted in the caller's buffers on entry and back on every exit
    const float Ta = (float)th->T_a;
    CK(launch_add_const(d_T, -Ta, c->N, s), "rise in");
    CK(launch_add_const(d_Tmax, -Ta, c->N, s), "rise in");
    c->launches += 2;
    auto to_celsius = [&](const float *cur) -> int {
        if (cur != d_T)
            CK(cudaMemcpyAsync(d_T, cur, c->N * sizeof(float), cudaMemcpyDeviceToDevice, s), "T out");
        CK(launch_add_const(d_T, Ta, c->N, s), "rise out");
        CK(launch_add_const(d_Tmax, Ta, c->N, s), "rise out");
        c->launches += 2;
        return BVF_OK;
    };
    Budget budget{c};
    for (int n = 0; n < total; ++n) {
        const int rb = budget.check(n, s, "bvf_run_thermal");
        if (rb != BVF_OK) {
            // the last completed step's temperature goes to d_T
            const int rc = to_celsius(a);
            c->thermal_steps += n;
            return rc != BVF_OK ? rc : rb;
        }
        p.dc = (n < th->n_on) ? (float)th->duty : 0.0f;
        p.flush = ((n + 1) % 32 == 0 || n + 1 == total) ? 1 : 0;
        p.wait_limit = tma::kWaitLimit;
        p.hold_plane = -1;
        if (n == 0 && c->hold == 3) {        // test hook: the first step only
            p.hold_plane = c->hold_plane;
            p.wait_limit = c->hold_limit ? c->hold_limit : tma::kWaitLimit;
            c->hold = 0;
        }
        p.T = a;
        p.Tn = b;
        CK(launch_thermal_step(p, th_tma ? &tmaps[a == d_T ? 0 : 1] : nullptr, c->flag, s),
           "thermal kernel");
        c->launches++;
        std::swap(a, b);
    }
    const int rc = to_celsius(a);
    if (rc != BVF_OK) return rc;
    c->thermal_steps += total;
    return BVF_OK;
}

int bvf_plan_host(bvf_ctx *skull, bvf_ctx *water, const uint8_t *h_index,
                  const bvf_material *h_table, int n_mat, const bvf_material *h_water,
                  const bvf_bowl *bowl, int k_src, const bvf_plan_params *pp, float *h_peak,
                  float *h_T, float *h_Tmax, double *h_cem43, bvf_plan_result *out, void *stream)
{
    if (!skull || !h_index || !h_peak || !h_Tmax || !h_cem43)
        return fail(skull, BVF_E_ARG, "bvf_plan_host: NULL argument");
    bvf_ctx *c = skull;
    const size_t N = c->N;
    if (!c->h_index_d) {
        CK(cudaMalloc(&c->h_index_d, N), "bvf_plan_host: staging");
        CK(cudaMalloc(&c->h_peak_d, N * sizeof(float)), "bvf_plan_host: staging");
        CK(cudaMalloc(&c->h_T_d, N * sizeof(float)), "bvf_plan_host: staging");
        CK(cudaMalloc(&c->h_Tmax_d, N * sizeof(float)), "bvf_plan_host: staging");
        CK(cudaMalloc(&c->h_amp_d, N * sizeof(double)), "bvf_plan_host: staging");
        CK(cudaMalloc(&c->h_cem_d, N * sizeof(double)), "bvf_plan_host: staging");
    }
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(c->h_index_d, h_index, N, cudaMemcpyHostToDevice, s), "bvf_plan_host: index in");
    const int rc = bvf_plan(skull, water, c->h_index_d, h_table, n_mat, h_water, bowl, k_src, pp,
                            c->h_peak_d, c->h_amp_d, c->h_T_d, c->h_Tmax_d, c->h_cem_d, out, stream);
    if (rc != BVF_OK) return rc;
    CK(cudaMemcpyAsync(h_peak, c->h_peak_d, N * sizeof(float), cudaMemcpyDeviceToHost, s),
       "bvf_plan_host: peak out");
    if (h_T)
        CK(cudaMemcpyAsync(h_T, c->h_T_d, N * sizeof(float), cudaMemcpyDeviceToHost, s),
           "bvf_plan_host: T out");
    CK(cudaMemcpyAsync(h_Tmax, c->h_Tmax_d, N * sizeof(float), cudaMemcpyDeviceToHost, s),
       "bvf_plan_host: T_max out");
    CK(cudaMemcpyAsync(h_cem43, c->h_cem_d, N * sizeof(double), cudaMemcpyDeviceToHost, s),
       "bvf_plan_host: CEM43 out");
    CK(cudaStreamSynchronize(s), "bvf_plan_host");
    return BVF_OK;
}

int bvf_rs_plane(const bvf_bowl *bw, int nx, int ny, double dx, double z_plane, double f0,
                 float *d_out, void *stream)
{
    if (!bw || !d_out || nx < 1 || ny < 1 || !(dx > 0.0) || !(f0 > 0.0) || !(bw->c0 > 0.0))
        return fail(nullptr, BVF_E_ARG, "bvf_rs_plane: bad argument");
    const double a = 0.5 * bw->aperture, R = bw->roc;
    if (!(a > 0.0) || !(R >= a)) return fail(nullptr, BVF_E_ARG, "bvf_rs_plane: need 0 < aperture/2 <= roc");
    const double lambda = bw->c0 / f0;
    const double ds = (bw->ds_over_lambda > 0.0 ? bw->ds_over_lambda : 0.25) * lambda;
    // Cap cut into rings of equal polar-angle width, each into equal azimuthal
    // elements of length about ds, then rotated from +z to dir about the apex.
    double ux = bw->dir[0], uy = bw->dir[1], uz = bw->dir[2];
    const double nrm = std::sqrt(ux * ux + uy * uy + uz * uz);
    if (!(nrm > 0.0)) return fail(nullptr, BVF_E_ARG, "bvf_rs_plane: zero direction");
    ux /= nrm; uy /= nrm; uz /= nrm;
    double kx = -uy, ky = ux;
    const double sn = std::sqrt(kx * kx + ky * ky), cs = uz;
    if (sn > 0.0) { kx /= sn; ky /= sn; }
    const double thmax = std::asin(a / R);
    const int nr = std::max(1, (int)std::ceil(R * thmax / ds));
    std::vector<float4> el;
    for (int r = 0; r < nr; ++r) {
        const double t0 = thmax * r / nr, t1 = thmax * (r + 1) / nr, tc = 0.5 * (t0 + t1);
        const double area = 2.0 * kPi * R * R * (std::cos(t0) - std::cos(t1));
        const int naz = std::max(1, (int)std::lround(2.0 * kPi * R * std::sin(tc) / ds));
        for (int e = 0; e < naz; ++e) {
            const double ph = 2.0 * kPi * (e + 0.5) / naz;
            const double px = R * std::sin(tc) * std::cos(ph), py = R * std::sin(tc) * std::sin(ph);
            const double pz = R * (1.0 - std::cos(tc));
            const double kp = kx * px + ky * py;
            const double cx = ky * pz, cy = -kx * pz, cz = kx * py - ky * px;
            const double rx = px * cs + cx * sn + kx * kp * (1.0 - cs);
            const double ry = py * cs + cy * sn + ky * kp * (1.0 - cs);
            const double rz = pz * cs + cz * sn;
            const double ex = bw->apex[0] + rx, ey = bw->apex[1] + ry, ez = bw->apex[2] + rz;
            if (!(ez < z_plane)) return fail(nullptr, BVF_E_ARG, "bvf_rs_plane: bowl crosses the source plane");
            el.push_back(make_float4((float)ex, (float)ey, (float)ez, (float)(area / naz)));
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    float4 *d_el = nullptr;
    cudaError_t e = cudaMallocAsync(&d_el, el.size() * sizeof(float4), s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "bvf_rs_plane: element buffer");
    e = cudaMemcpyAsync(d_el, el.data(), el.size() * sizeof(float4), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        const double k = 2.0 * kPi / lambda;
        e = launch_rs(d_el, (int)el.size(), nx, ny, (float)dx, (float)z_plane, (float)(k / kPi),
                      k * bw->p0 / (2.0 * kPi), reinterpret_cast<float2 *>(d_out), s);
    }
    cudaError_t e2 = cudaFreeAsync(d_el, s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "bvf_rs_plane");
    if (e2 != cudaSuccess) return cuda_fail(nullptr, e2, "bvf_rs_plane: free");
    return BVF_OK;
}

int bvf_rs_elements(const double *h_elem, int ne, double p0, double c0, int nx, int ny,
                    double dx, double z_plane, double f0, float *d_out, void *stream)
{
    if (!h_elem || ne < 1 || !d_out || nx < 1 || ny < 1 || !(dx > 0.0) || !(f0 > 0.0) ||
        !(c0 > 0.0))
        return fail(nullptr, BVF_E_ARG, "bvf_rs_elements: bad argument");
    std::vector<float4> el(ne);
    std::vector<float2> wt(ne);
    for (int e = 0; e < ne; ++e) {
        const double *r = h_elem + 6 * (size_t)e;
        if (!(r[2] < z_plane) || !(r[3] >= 0.0))
            return fail(nullptr, BVF_E_ARG,
                        "bvf_rs_elements: an element lies on or above the plane, or has negative area");
        el[e] = make_float4((float)r[0], (float)r[1], (float)r[2], (float)r[3]);
        wt[e] = make_float2((float)r[4], (float)r[5]);
    }
    cudaStream_t s = (cudaStream_t)stream;
    char *buf = nullptr;
    const size_t bytes = ne * (sizeof(float4) + sizeof(float2));
    cudaError_t e = cudaMallocAsync((void **)&buf, bytes, s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "bvf_rs_elements: element buffer");
    float4 *d_el = reinterpret_cast<float4 *>(buf);
    float2 *d_wt = reinterpret_cast<float2 *>(buf + ne * sizeof(float4));
    e = cudaMemcpyAsync(d_el, el.data(), ne * sizeof(float4), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_wt, wt.data(), ne * sizeof(float2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        const double k = 2.0 * kPi * f0 / c0;
        e = launch_rs_weighted(d_el, d_wt, ne, nx, ny, (float)dx, (float)z_plane, (float)(k / kPi),
                               k * p0 / (2.0 * kPi), reinterpret_cast<float2 *>(d_out), s);
    }
    cudaError_t e2 = cudaFreeAsync(buf, s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "bvf_rs_elements");
    if (e2 != cudaSuccess) return cuda_fail(nullptr, e2, "bvf_rs_elements: free");
    return BVF_OK;
}

int bvf_transmission(int nx, int ny, int nz, const uint8_t *d_idx_a, const bvf_material *h_mat_a,
                     int n_a, const double *d_amp_a, const uint8_t *d_idx_w,
                     const bvf_material *h_mat_w, int n_w, const double *d_amp_w, double *h_EL,
                     double *h_TS, int *h_zm, double *h_Iw_max, void *stream)
{
    bvf_ctx *c = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || !d_idx_a || !h_mat_a || !d_amp_a || !d_idx_w || !h_mat_w ||
        !d_amp_w || n_a < 1 || n_w < 1 || n_a > BVF_MAX_MATERIALS || n_w > BVF_MAX_MATERIALS)
        return fail(nullptr, BVF_E_ARG, "bvf_transmission: bad argument");
    std::vector<double> z(2 * BVF_MAX_MATERIALS, 0.0);
    for (int m = 0; m < n_a; ++m) z[m] = 1.0 / (2.0 * h_mat_a[m].rho * h_mat_a[m].cL);
    for (int m = 0; m < n_w; ++m) z[BVF_MAX_MATERIALS + m] = 1.0 / (2.0 * h_mat_w[m].rho * h_mat_w[m].cL);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)nx * ny * nz;
    // one scratch block: [z tables][best][idx][sums]
    const size_t bytes = 2 * BVF_MAX_MATERIALS * sizeof(double) + 2 * sizeof(unsigned long long) +
                         3 * sizeof(double);
    char *d = nullptr;
    CK(cudaMallocAsync((void **)&d, bytes, s), "transmission scratch");
    double *dz = reinterpret_cast<double *>(d);
    unsigned long long *best = reinterpret_cast<unsigned long long *>(dz + 2 * BVF_MAX_MATERIALS);
    unsigned long long *qb = best + 1;
    double *sums = reinterpret_cast<double *>(qb + 1);
    const unsigned long long init[2] = {0ull, ~0ull};
    double res[3] = {0, 0, 0};
    unsigned long long best_bits = 0;
    cudaError_t e = cudaMemcpyAsync(dz, z.data(), z.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(best, init, sizeof init, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_intensity_argmax(d_idx_w, dz + BVF_MAX_MATERIALS, d_amp_w, n, best, s);
    if (e == cudaSuccess)
        e = launch_intensity_argmin_index(d_idx_w, dz + BVF_MAX_MATERIALS, d_amp_w, n, best, qb, s);
    if (e == cudaSuccess)
        e = launch_plane_sums(d_idx_a, dz, d_amp_a, d_idx_w, dz + BVF_MAX_MATERIALS, d_amp_w, nx, ny,
                              nz, qb, sums, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(res, sums, sizeof res, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&best_bits, best, sizeof best_bits, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(d, s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "bvf_transmission");
    if (!(res[1] > 0.0)) return fail(nullptr, BVF_E_ARG, "bvf_transmission: zero water intensity");
    const double el = res[0] / res[1];
    if (h_EL) *h_EL = el;
    if (h_TS) *h_TS = std::sqrt(el);
    if (h_zm) *h_zm = (int)res[2];
    if (h_Iw_max) {
        double bw;
        std::memcpy(&bw, &best_bits, sizeof bw);
        *h_Iw_max = bw;
    }
    (void)c;
    return BVF_OK;
}

int bvf_kernel_timing(bvf_ctx *c, int enable)
{
    if (!c) return fail(nullptr, BVF_E_ARG, "bvf_kernel_timing: NULL context");
    CK(drain_events(c), "kernel timing");
    c->timing = enable != 0;
    c->vel_ms = c->str_ms = 0.0;
    c->vel_n = c->str_n = 0;
    return BVF_OK;
}

int bvf_get_kernel_times(bvf_ctx *c, bvf_kernel_times *out)
{
    if (!c || !out) return fail(c, BVF_E_ARG, "bvf_get_kernel_times: NULL argument");
    CK(drain_events(c), "kernel timing");
    out->velocity_launches = c->vel_n;
    out->stress_launches = c->str_n;
    out->velocity_ms = c->vel_ms;
    out->stress_ms = c->str_ms;
    return BVF_OK;
}

// ---- one placement end to end ---------------------------------------------

int bvf_plan(bvf_ctx *skull, bvf_ctx *water, const uint8_t *d_index, const bvf_material *h_table,
             int n_mat, const bvf_material *h_water, const bvf_bowl *bowl, int k_src,
             const bvf_plan_params *pp, float *d_peak, double *d_amp, float *d_T, float *d_Tmax,
             double *d_cem43, bvf_plan_result *out, void *stream)
{
    if (!skull || !water || !d_index || !h_table || !h_water || !bowl || !pp || !d_peak ||
        !d_amp || !d_T || !d_Tmax || !d_cem43 || !out)
        return fail(nullptr, BVF_E_ARG, "bvf_plan: NULL argument");
    if (skull->g.nx != water->g.nx || skull->g.ny != water->g.ny || skull->g.nz != water->g.nz ||
        skull->g.dx != water->g.dx || skull->g.dt != water->g.dt || skull->ph.f0 != water->ph.f0)
        return fail(nullptr, BVF_E_ARG, "bvf_plan: the two contexts differ in grid or frequency");
    if (pp->n_steps < 1 || pp->dft_steps < 1)
        return fail(nullptr, BVF_E_ARG, "bvf_plan: need n_steps >= 1 and a capture window");
    cudaStream_t s = (cudaStream_t)stream;
    const bvf_grid &g = skull->g;
    const size_t N = skull->N, plane = (size_t)g.nx * g.ny;
    int rc = bvf_set_materials(skull, d_index, h_table, n_mat);
    if (rc != BVF_OK) return rc;
    // temporaries: the water run's zero index and amplitude, the source plane
    uint8_t *zidx = nullptr;
    double *amp_w = nullptr;
    float *src = nullptr;
    auto release = [&]() {
        if (zidx) cudaFreeAsync(zidx, s);
        if (amp_w) cudaFreeAsync(amp_w, s);
        if (src) cudaFreeAsync(src, s);
    };
    cudaError_t e = cudaMallocAsync((void **)&zidx, N, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&amp_w, N * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&src, plane * 2 * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(zidx, 0, N, s);
    // bvf_set_materials copies the index with a blocking copy: finish the fill first
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        release();
        return cuda_fail(nullptr, e, "bvf_plan: temporaries");
    }
    bool forked = false;      // work on the skull context's second stream not yet joined
    auto done = [&](int code) {
        if (forked) {         // join before the temporaries are released on `stream`
            cudaEventRecord(skull->join_ev, skull->side);
            cudaStreamWaitEvent(s, skull->join_ev, 0);
        }
        release();
        return code;
    };
    if ((rc = bvf_set_materials(water, zidx, h_water, 1)) != BVF_OK) return done(rc);
    if ((rc = bvf_rs_plane(bowl, g.nx, g.ny, g.dx, k_src * g.dx, skull->ph.f0, src, stream)) != BVF_OK)
        return done(rc);
    const bvf_capture cap{0, pp->dft_start, pp->dft_steps};
    // the water run on the skull context's second stream, forked after the
    // source plane exists and joined before the reductions (serial: `stream`)
    void *ws = stream;
    if (!pp->serial) {
        if (!skull->side) {
            e = cudaStreamCreateWithFlags(&skull->side, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&skull->fork_ev, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&skull->join_ev, cudaEventDisableTiming);
            if (e != cudaSuccess) return done(cuda_fail(nullptr, e, "bvf_plan: second stream"));
        }
        e = cudaEventRecord(skull->fork_ev, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(skull->side, skull->fork_ev, 0);
        if (e != cudaSuccess) return done(cuda_fail(nullptr, e, "bvf_plan: fork"));
        ws = skull->side;
        forked = true;
    }
    bvf_ctx *runs[2] = {skull, water};
    for (bvf_ctx *c : runs) {
        void *cs = (c == water) ? ws : stream;
        if ((rc = bvf_reset(c, cs)) != BVF_OK) return done(rc);
        if ((rc = bvf_set_source(c, k_src, src, bowl->c0, BVF_ENV_RAMP_CW, 0, cs)) != BVF_OK)
            return done(rc);
        if ((rc = bvf_run_acoustic(c, pp->n_steps, &cap, cs)) != BVF_OK) return done(rc);
    }
    if ((rc = bvf_get_amp_phase(skull, d_amp, nullptr, stream)) != BVF_OK) return done(rc);
    if ((rc = bvf_get_amp_phase(water, amp_w, nullptr, ws)) != BVF_OK) return done(rc);
    if (forked) {
        forked = false;
        e = cudaEventRecord(skull->join_ev, skull->side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, skull->join_ev, 0);
        if (e != cudaSuccess) return done(cuda_fail(nullptr, e, "bvf_plan: join"));
    }
    if ((rc = bvf_get_peak(skull, d_peak, stream)) != BVF_OK) return done(rc);
    for (bvf_ctx *c : runs)
        if ((rc = bvf_synchronize(c, stream)) != BVF_OK) return done(rc);
    bvf_plan_result r{};
    rc = bvf_transmission(g.nx, g.ny, g.nz, d_index, h_table, n_mat, d_amp, zidx, h_water, 1,
                          amp_w, &r.EL, &r.TS, &r.z_m, &r.Iw_max, stream);
    if (rc != BVF_OK) return done(rc);
    const double i_sppa = pp->i_sppa > 0.0 ? pp->i_sppa : 5.0e4;
    r.p_scale = (r.EL > 0.0 && r.Iw_max > 0.0) ? std::sqrt(i_sppa / (r.EL * r.Iw_max)) : 0.0;
    bvf_thermal th = pp->thermal;
    th.p_scale = r.p_scale;
    e = launch_fill(d_T, (float)th.T_a, N, s);
    if (e == cudaSuccess) e = launch_fill(d_Tmax, (float)th.T_a, N, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cem43, 0, N * sizeof(double), s);
    if (e != cudaSuccess) return done(cuda_fail(nullptr, e, "bvf_plan: thermal start"));
    skull->launches += 2;
    if ((rc = bvf_run_thermal(skull, &th, d_amp, d_T, d_Tmax, d_cem43, stream)) != BVF_OK)
        return done(rc);
    release();
    CK_FREE(cudaStreamSynchronize(s), "bvf_plan");
    *out = r;
    return BVF_OK;
}

// ---- batched runs --------------------------------------------------------

int bvf_batch_create(bvf_ctx *const *ctxs, int n, bvf_batch **out)
{
    if (!out) return fail(nullptr, BVF_E_ARG, "bvf_batch_create: out is NULL");
    *out = nullptr;
    if (!ctxs || n < 1 || n > kMaxBatch)
        return fail(nullptr, BVF_E_ARG, "bvf_batch_create: need 1 to 64 contexts");
    for (int d = 0; d < n; ++d) {
        const bvf_ctx *c = ctxs[d];
        if (!c || !c->have_materials)
            return fail(nullptr, BVF_E_ARG, "bvf_batch_create: NULL context or materials not set");
        if (!c->tma || !c->tma_stress)
            return fail(nullptr, BVF_E_ARG,
                        "bvf_batch_create: every grid needs nx % 8 == 0 and at most 2 SLS");
        if (c->L != ctxs[0]->L || c->h16 != ctxs[0]->h16)
            return fail(nullptr, BVF_E_ARG,
                        "bvf_batch_create: contexts differ in SLS count or storage");
    }
    bvf_batch *b = new (std::nothrow) bvf_batch;
    if (!b) return fail(nullptr, BVF_E_NOMEM, "bvf_batch_create: host allocation failed");
    b->ctx.assign(ctxs, ctxs + n);
    b->L = ctxs[0]->L;
    b->h16 = ctxs[0]->h16;
    for (const bvf_ctx *c : b->ctx) b->n_mat_max = std::max(b->n_mat_max, (int)c->table.size());
    cudaError_t e = cudaMalloc(&b->d_step, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_sm, n * sizeof(StressTmaMaps));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_vm, n * sizeof(VelocityTmaMaps));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = batch_prepare(b->L, b->h16, b->n_mat_max, &b->grid_vel, &b->grid_str);
    if (e != cudaSuccess) {
        bvf_batch_destroy(b);
        return cuda_fail(nullptr, e, "bvf_batch_create");
    }
    *out = b;
    return BVF_OK;
}

void bvf_batch_destroy(bvf_batch *b)
{
    if (b && b->gexec) cudaGraphExecDestroy(b->gexec);
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (cudaStream_t t : b->side) cudaStreamDestroy(t);
    for (cudaEvent_t ev : b->side_ev) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    void *bufs[] = {b->d_sm, b->d_vm, b->d_steps, b->d_step};
    for (void *p : bufs)
        if (p) cudaFree(p);
    delete b;
}

int bvf_batch_run(bvf_batch *b, const int *n_steps, const bvf_capture *caps, int kchunk,
                  int graph_steps, void *stream)
{
    if (!b || !n_steps) return fail(nullptr, BVF_E_ARG, "bvf_batch_run: NULL argument");
    const int n = (int)b->ctx.size();
    cudaStream_t s = (cudaStream_t)stream;
    long long total_steps = 0;
    int n_max = 0;
    for (int d = 0; d < n; ++d) {
        if (n_steps[d] < 0) return fail(nullptr, BVF_E_ARG, "bvf_batch_run: negative step count");
        if (caps && caps[d].dft_steps < 0)
            return fail(nullptr, BVF_E_ARG, "bvf_batch_run: negative dft_steps");
        total_steps += n_steps[d];
        n_max = std::max(n_max, n_steps[d]);
    }
    if (kchunk < 0) return fail(nullptr, BVF_E_ARG, "bvf_batch_run: negative kchunk");
    // device buffers: tensor maps and per-step tables
    if (b->steps_cap < (size_t)std::max<long long>(total_steps, 1)) {
        if (b->d_steps) cudaFree(b->d_steps);
        b->d_steps = nullptr;
        b->steps_cap = 0;
        cudaError_t e = cudaMalloc(&b->d_steps, std::max<long long>(total_steps, 1) * sizeof(StepParam));
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "bvf_batch_run: step tables");
        b->steps_cap = std::max<long long>(total_steps, 1);
    }
    std::vector<StressTmaMaps> hsm(n);
    std::vector<VelocityTmaMaps> hvm(n);
    b->h_steps.resize(std::max<long long>(total_steps, 1));
    BatchParams &bp = b->bp;
    bp = BatchParams{};
    bp.sm = b->d_sm;
    bp.vm = b->d_vm;
    bp.steps = b->d_steps;
    bp.n_dom = n;
    int total = 0;
    long long off = 0;
    for (int d = 0; d < n; ++d) {
        bvf_ctx *c = b->ctx[d];
        bvf_capture cp{-1, 0, 0};
        if (caps) cp = caps[d];
        if (cp.dft_steps > 0) {
            const int rc = ensure_dft(c, s);
            if (rc != BVF_OK) return rc;
        }
        hsm[d] = c->smaps;
        hvm[d] = c->vmaps;
        bp.p[d] = make_params(c);
        const int kc0 = kchunk > 0 ? kchunk : (c->kchunk > 0 ? c->kchunk
                                                             : default_kchunk_tma(c->g.nx, c->g.ny, c->g.nz));
        bp.kchunk[d] = std::min(kc0, c->g.nz);
        bp.tiles_x[d] = (c->g.nx + 31) / 32;
        bp.tiles_y[d] = (c->g.ny + 7) / 8;
        const int chunks = (c->g.nz + bp.kchunk[d] - 1) / bp.kchunk[d];
        bp.block0[d] = total;
        total += bp.tiles_x[d] * bp.tiles_y[d] * chunks;
        bp.n_steps[d] = n_steps[d];
        bp.step_off[d] = (int)off;
        for (int k = 0; k < n_steps[d]; ++k) b->h_steps[off + k] = step_param(c, cp, c->steps + k);
        off += n_steps[d];
    }
    bp.total = total;
    CK_FREE(cudaMemcpyAsync(b->d_sm, hsm.data(), n * sizeof(StressTmaMaps), cudaMemcpyHostToDevice,
                            s), "bvf_batch_run: tensor maps");
    CK_FREE(cudaMemcpyAsync(b->d_vm, hvm.data(), n * sizeof(VelocityTmaMaps),
                            cudaMemcpyHostToDevice, s), "bvf_batch_run: tensor maps");
    if (total_steps)
        CK_FREE(cudaMemcpyAsync(b->d_steps, b->h_steps.data(), total_steps * sizeof(StepParam),
                                cudaMemcpyHostToDevice, s), "bvf_batch_run: step tables");
    CK_FREE(cudaMemsetAsync(b->d_step, 0, sizeof(int), s), "bvf_batch_run: step counter");
    if (graph_steps <= 0) {
        for (int k = 0; k < n_max; ++k)
            CK_FREE(launch_batch_step(bp, b->L, b->h16, b->n_mat_max, b->d_step, b->grid_vel,
                                      b->grid_str, s), "bvf_batch_run: kernels");
        b->launches += 3LL * n_max;
    } else if (n_max > 0) {
        // one graph of G steps (3 kernels each), replayed; steps past a domain's
        // end find it finished and skip it
        const int G = std::min(graph_steps, n_max);
        if (b->exec) {
            CK_FREE(cudaStreamSynchronize(s), "bvf_batch_run: previous graph");
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        CK_FREE(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal),
                "bvf_batch_run: capture");
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < G && e == cudaSuccess; ++k)
            e = launch_batch_step(bp, b->L, b->h16, b->n_mat_max, b->d_step, b->grid_vel,
                                  b->grid_str, b->cap);
        cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "bvf_batch_run: graph");
        const int reps = (n_max + G - 1) / G;
        for (int r = 0; r < reps; ++r)
            CK_FREE(cudaGraphLaunch(b->exec, s), "bvf_batch_run: graph launch");
        b->launches += 3LL * G * reps;
    }
    off = 0;
    for (int d = 0; d < n; ++d) {
        bvf_ctx *c = b->ctx[d];
        for (int k = 0; k < n_steps[d]; ++k) c->dft_count += (b->h_steps[off + k].flags >> 2) & 1;
        off += n_steps[d];
        c->steps += n_steps[d];
    }
    return BVF_OK;
}

int bvf_batch_run_streams(bvf_batch *b, const int *n_steps, const bvf_capture *caps,
                          int n_streams, void *stream)
{
    if (!b || !n_steps || n_streams < 1)
        return fail(nullptr, BVF_E_ARG, "bvf_batch_run_streams: bad argument");
    const int n = (int)b->ctx.size();
    for (int d = 0; d < n; ++d)
        if (n_steps[d] < 0) return fail(nullptr, BVF_E_ARG, "bvf_batch_run_streams: negative step count");
    cudaStream_t s = (cudaStream_t)stream;
    while ((int)b->side.size() < n_streams) {
        cudaStream_t t = nullptr;
        CK_FREE(cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking), "bvf_batch_run_streams");
        b->side.push_back(t);
        cudaEvent_t ev = nullptr;
        CK_FREE(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "bvf_batch_run_streams");
        b->side_ev.push_back(ev);
    }
    if (!b->fork) CK_FREE(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "bvf_batch_run_streams");
    // fork: every side stream waits for the caller's stream
    CK_FREE(cudaEventRecord(b->fork, s), "bvf_batch_run_streams");
    for (int k = 0; k < n_streams; ++k)
        CK_FREE(cudaStreamWaitEvent(b->side[k], b->fork, 0), "bvf_batch_run_streams");
    // domains dealt round-robin; each side stream runs its domains one after another
    for (int d = 0; d < n; ++d) {
        const int rc = bvf_run_acoustic(b->ctx[d], n_steps[d], caps ? &caps[d] : nullptr,
                                        b->side[d % n_streams]);
        if (rc != BVF_OK) return rc;
        b->launches += 2LL * n_steps[d];
    }
    // join: the caller's stream waits for every side stream
    for (int k = 0; k < n_streams; ++k) {
        CK_FREE(cudaEventRecord(b->side_ev[k], b->side[k]), "bvf_batch_run_streams");
        CK_FREE(cudaStreamWaitEvent(s, b->side_ev[k], 0), "bvf_batch_run_streams");
    }
    return BVF_OK;
}

// side streams and events of the batch, at least n of each
static int batch_side_streams(bvf_batch *b, int n)
{
    while ((int)b->side.size() < n) {
        cudaStream_t t = nullptr;
        CK_FREE(cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking), "batch streams");
        b->side.push_back(t);
        cudaEvent_t ev = nullptr;
        CK_FREE(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "batch streams");
        b->side_ev.push_back(ev);
    }
    if (!b->fork) CK_FREE(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "batch streams");
    return BVF_OK;
}

int bvf_batch_run_graph(bvf_batch *b, const int *n_steps, const bvf_capture *caps, int n_branches,
                        void *stream)
{
    if (!b || !n_steps || n_branches < 1)
        return fail(nullptr, BVF_E_ARG, "bvf_batch_run_graph: bad argument");
    const int n = (int)b->ctx.size();
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<long long> sig;
    sig.push_back(n_branches);
    for (int d = 0; d < n; ++d) {
        bvf_ctx *c = b->ctx[d];
        if (n_steps[d] < 0 || (caps && caps[d].dft_steps < 0))
            return fail(nullptr, BVF_E_ARG, "bvf_batch_run_graph: negative step count");
        if (c->budget_s > 0.0 || c->timing || c->hold)
            return fail(nullptr, BVF_E_ARG, "bvf_batch_run_graph: a context has a time budget, "
                                            "kernel timing or the test hook armed");
        const bvf_capture cp = caps ? caps[d] : bvf_capture{-1, 0, 0};
        sig.insert(sig.end(), {c->steps, n_steps[d], cp.peak_from, cp.dft_start, cp.dft_steps,
                               c->kchunk, c->tile.stress_rows, c->tile.velocity_rows});
    }
    if (!b->gexec || sig != b->gsig) {
        // record the per-domain launches once, domains dealt round-robin over
        // the branches, on the batch's own stream (the caller's may be the
        // legacy default stream, which cannot be recorded)
        int rc = batch_side_streams(b, n_branches);
        if (rc != BVF_OK) return rc;
        for (int d = 0; d < n; ++d)
            if (caps && caps[d].dft_steps > 0 && (rc = ensure_dft(b->ctx[d], s)) != BVF_OK) return rc;
        CK_FREE(cudaStreamSynchronize(s), "bvf_batch_run_graph");
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        std::vector<long long> st0(n), df0(n), ln0(n);
        for (int d = 0; d < n; ++d) {
            st0[d] = b->ctx[d]->steps;
            df0[d] = b->ctx[d]->dft_count;
            ln0[d] = b->ctx[d]->launches;
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) e = cudaEventRecord(b->fork, b->cap);
        for (int k = 0; k < n_branches && e == cudaSuccess; ++k)
            e = cudaStreamWaitEvent(b->side[k], b->fork, 0);
        for (int d = 0; d < n && e == cudaSuccess && rc == BVF_OK; ++d)
            rc = bvf_run_acoustic(b->ctx[d], n_steps[d], caps ? &caps[d] : nullptr,
                                  b->side[d % n_branches]);
        for (int k = 0; k < n_branches && e == cudaSuccess; ++k) {
            e = cudaEventRecord(b->side_ev[k], b->side[k]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->side_ev[k], 0);
        }
        const cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess && rc == BVF_OK) e = cudaGraphInstantiate(&b->gexec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        // nothing ran yet: the counters go back to where the recording began
        b->gdsteps.assign(n, 0);
        b->gddft.assign(n, 0);
        for (int d = 0; d < n; ++d) {
            bvf_ctx *c = b->ctx[d];
            b->gdsteps[d] = c->steps - st0[d];
            b->gddft[d] = c->dft_count - df0[d];
            c->steps = st0[d];
            c->dft_count = (int)df0[d];
            c->launches = ln0[d];
        }
        if (rc != BVF_OK) return rc;
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "bvf_batch_run_graph: recording");
        b->gsig = sig;
    }
    CK_FREE(cudaGraphLaunch(b->gexec, s), "bvf_batch_run_graph: launch");
    for (int d = 0; d < n; ++d) {
        bvf_ctx *c = b->ctx[d];
        c->steps += b->gdsteps[d];
        c->dft_count += (int)b->gddft[d];
        c->launches += 2 * b->gdsteps[d];
        b->launches += 2 * b->gdsteps[d];
    }
    return BVF_OK;
}

int bvf_batch_tune_domains(bvf_batch *b, int trial_steps, const bvf_tile *candidates,
                           int n_candidates, bvf_tile *h_best, void *stream)
{
    if (!b || !candidates || n_candidates < 1 || trial_steps < 1)
        return fail(nullptr, BVF_E_ARG, "bvf_batch_tune_domains: bad argument");
    for (int ci = 0; ci < n_candidates; ++ci)
        if (!tile_valid(candidates[ci]))
            return fail(nullptr, BVF_E_ARG, "bvf_batch_tune_domains: bad candidate");
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK_FREE(cudaEventCreate(&e0), "bvf_batch_tune_domains");
    CK_FREE(cudaEventCreate(&e1), "bvf_batch_tune_domains");
    int rc = BVF_OK;
    for (size_t d = 0; d < b->ctx.size() && rc == BVF_OK; ++d) {
        bvf_ctx *c = b->ctx[d];
        double best = 1e300;
        bvf_tile best_t = c->tile;
        for (int ci = 0; ci < n_candidates && rc == BVF_OK; ++ci) {
            const bvf_tile cand = candidates[ci];
            // heights other than 8 run with L = 2 only: other contexts skip them
            if (c->L != 2 && ((cand.stress_rows != 0 && cand.stress_rows != 8) ||
                              (cand.velocity_rows != 0 && cand.velocity_rows != 8)))
                continue;
            c->tile = cand;
            c->tile.kchunk = std::min(cand.kchunk, c->g.nz);
            c->kchunk = c->tile.kchunk;
            if ((rc = bvf_reset(c, stream)) != BVF_OK) break;
            if ((rc = bvf_run_acoustic(c, 2, nullptr, stream)) != BVF_OK) break;   // warm-up
            cudaEventRecord(e0, s);
            if ((rc = bvf_run_acoustic(c, trial_steps, nullptr, stream)) != BVF_OK) break;
            cudaEventRecord(e1, s);
            float ms = 0.0f;
            cudaError_t e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                rc = cuda_fail(nullptr, e, "bvf_batch_tune_domains");
                break;
            }
            if (ms < best) {
                best = ms;
                best_t = c->tile;
            }
        }
        c->tile = best_t;
        c->kchunk = best_t.kchunk;
        if (h_best) h_best[d] = best_t;
        if (rc == BVF_OK) rc = bvf_reset(c, stream);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

int bvf_batch_tune_graph(bvf_batch *b, int trial_steps, const bvf_tile *candidates,
                         int n_candidates, int n_branches, bvf_tile *h_best, double *h_ms,
                         void *stream)
{
    if (!b || !candidates || n_candidates < 1 || trial_steps < 1 || n_branches < 1 || !h_best)
        return fail(nullptr, BVF_E_ARG, "bvf_batch_tune_graph: bad argument");
    for (int ci = 0; ci < n_candidates; ++ci)
        if (!tile_valid(candidates[ci]))
            return fail(nullptr, BVF_E_ARG, "bvf_batch_tune_graph: bad candidate");
    const size_t n = b->ctx.size();
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK_FREE(cudaEventCreate(&e0), "bvf_batch_tune_graph");
    CK_FREE(cudaEventCreate(&e1), "bvf_batch_tune_graph");
    const std::vector<int> steps(n, trial_steps);
    double best = 1e300;
    bvf_tile best_t = candidates[0];
    int rc = BVF_OK;
    for (int ci = 0; ci < n_candidates && rc == BVF_OK; ++ci) {
        for (bvf_ctx *c : b->ctx) {
            c->tile = candidates[ci];
            c->kchunk = candidates[ci].kchunk;
        }
        // one replay records the graph (and warms up), the second is timed
        for (int rep = 0; rep < 2 && rc == BVF_OK; ++rep) {
            for (bvf_ctx *c : b->ctx)
                if ((rc = bvf_reset(c, stream)) != BVF_OK) break;
            if (rc != BVF_OK) break;
            if (rep == 1) cudaEventRecord(e0, s);
            rc = bvf_batch_run_graph(b, steps.data(), nullptr, n_branches, stream);
            if (rc == BVF_OK && rep == 1) cudaEventRecord(e1, s);
        }
        if (rc != BVF_OK) break;
        float ms = 0.0f;
        cudaError_t e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            rc = cuda_fail(nullptr, e, "bvf_batch_tune_graph");
            break;
        }
        if (ms < best) {
            best = ms;
            best_t = candidates[ci];
        }
    }
    for (bvf_ctx *c : b->ctx) {
        c->tile = best_t;
        c->kchunk = best_t.kchunk;
        if (rc == BVF_OK) rc = bvf_reset(c, stream);
    }
    *h_best = best_t;
    if (h_ms) *h_ms = best / trial_steps;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

int bvf_set_tile(bvf_ctx *c, const bvf_tile *t)
{
    if (!c || !t) return fail(c, BVF_E_ARG, "bvf_set_tile: NULL argument");
    if (!tile_valid(*t))
        return fail(c, BVF_E_ARG, "bvf_set_tile: rows must be 0, 4, 8 or 16 and kchunk >= 0");
    c->tile = *t;
    c->kchunk = t->kchunk;
    return BVF_OK;
}

int bvf_get_tile(const bvf_ctx *c, bvf_tile *out)
{
    if (!c || !out) return fail(nullptr, BVF_E_ARG, "bvf_get_tile: NULL argument");
    *out = effective_tile(c);
    out->kchunk = c->kchunk > 0 ? std::min(c->kchunk, c->g.nz)
                                : (c->tma ? default_kchunk_tma(c->g.nx, c->g.ny, c->g.nz,
                                                               out->stress_rows)
                                          : default_kchunk(c->g.nx, c->g.ny, c->g.nz));
    return BVF_OK;
}

int bvf_batch_tune(bvf_batch *b, int trial_steps, const int *candidates, int n_candidates,
                   int *best_kchunk, double *best_ms_per_step, void *stream)
{
    if (!b || !candidates || n_candidates < 1 || trial_steps < 1 || !best_kchunk)
        return fail(nullptr, BVF_E_ARG, "bvf_batch_tune: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    const int n = (int)b->ctx.size();
    std::vector<int> steps(n, trial_steps);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK_FREE(cudaEventCreate(&e0), "bvf_batch_tune");
    CK_FREE(cudaEventCreate(&e1), "bvf_batch_tune");
    double best = 1e300;
    int best_kc = candidates[0];
    int rc = BVF_OK;
    for (int ci = 0; ci < n_candidates && rc == BVF_OK; ++ci) {
        for (bvf_ctx *c : b->ctx)
            if ((rc = bvf_reset(c, stream)) != BVF_OK) break;
        if (rc != BVF_OK) break;
        // one untimed pass builds the graph's first replay path, the second is timed
        rc = bvf_batch_run(b, steps.data(), nullptr, candidates[ci], trial_steps, stream);
        if (rc != BVF_OK) break;
        cudaEventRecord(e0, s);
        rc = bvf_batch_run(b, steps.data(), nullptr, candidates[ci], trial_steps, stream);
        if (rc != BVF_OK) break;
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            rc = cuda_fail(nullptr, e, "bvf_batch_tune");
            break;
        }
        if (ms < best) {
            best = ms;
            best_kc = candidates[ci];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != BVF_OK) return rc;
    for (bvf_ctx *c : b->ctx)
        if ((rc = bvf_reset(c, stream)) != BVF_OK) return rc;
    *best_kchunk = best_kc;
    if (best_ms_per_step) *best_ms_per_step = best / trial_steps;
    return BVF_OK;
}

int bvf_batch_launches(const bvf_batch *b, long long *out)
{
    if (!b || !out) return fail(nullptr, BVF_E_ARG, "bvf_batch_launches: NULL argument");
    *out = b->launches;
    return BVF_OK;
}

int bvf_get_stats(const bvf_ctx *c, bvf_stats *out)
{
    if (!c || !out) return fail(nullptr, BVF_E_ARG, "bvf_get_stats: NULL argument");
    out->steps = c->steps;
    out->kernel_launches = c->launches;
    out->thermal_steps = c->thermal_steps;
    out->courant = c->courant;
    // velocity: read 6 sigma + 3 v, write 3 v (12 words); stress: read 3 v,
    // read + write 6 sigma and 6L memory variables (15 + 12 L words); the index
    // byte in each kernel and the FP32 peak map (read + write)
    out->bytes_per_voxel_step = (double)c->es * (12 + 15 + 12 * c->L) + 2.0 + 8.0;
    return BVF_OK;
}

// ---- call budget, time-out test hook, snapshots ---------------------------

int bvf_set_time_budget(bvf_ctx *c, double seconds)
{
    if (!c || !(seconds >= 0.0) || std::isinf(seconds))
        return fail(c, BVF_E_ARG, "bvf_set_time_budget: bad context or budget");
    c->budget_s = seconds;
    return BVF_OK;
}

int bvf_test_withhold_copy(bvf_ctx *c, int kernel, int plane, unsigned wait_limit)
{
    if (!c) return fail(nullptr, BVF_E_ARG, "bvf_test_withhold_copy: NULL context");
    if (kernel == 0) {
        c->hold = 0;
        return BVF_OK;
    }
    if ((kernel < 1 || kernel > 3) || plane < 0 || plane >= c->g.nz)
        return fail(c, BVF_E_ARG,
                    "bvf_test_withhold_copy: kernel must be 1, 2 or 3, plane inside the grid");
    if (kernel < 3 ? !(kernel == 1 ? c->tma : c->tma_stress)
                   : (c->g.nx % 8 != 0 || std::getenv("BVF_NO_TMA") != nullptr))
        return fail(c, BVF_E_ARG, "bvf_test_withhold_copy: this context does not use the TMA-fed kernel");
    c->hold = kernel;
    c->hold_plane = plane;
    c->hold_limit = wait_limit;
    return BVF_OK;
}

int bvf_state_bytes(const bvf_ctx *c, size_t *out)
{
    if (!c || !out) return fail(nullptr, BVF_E_ARG, "bvf_state_bytes: NULL argument");
    *out = state_sections(c).total;
    return BVF_OK;
}

int bvf_state_save(bvf_ctx *c, void *d_buf, size_t bytes, void *stream)
{
    if (!c || !d_buf) return fail(c, BVF_E_ARG, "bvf_state_save: NULL argument");
    const StateSections t = state_sections(c);
    if (bytes < t.total) return fail(c, BVF_E_ARG, "bvf_state_save: buffer smaller than bvf_state_bytes");
    cudaStream_t s = (cudaStream_t)stream;
    char *b = static_cast<char *>(d_buf);
    StateHeader h{};
    h.magic = kStateMagic;
    h.version = BVF_VERSION;
    h.nx = c->g.nx;
    h.ny = c->g.ny;
    h.nz = c->g.nz;
    h.L = c->L;
    h.h16 = c->h16;
    h.has_dft = c->dftC ? 1 : 0;
    h.steps = c->steps;
    h.dft_count = c->dft_count;
    h.dx = c->g.dx;
    h.dt = c->g.dt;
    h.f0 = c->ph.f0;
    h.bytes = t.total;
    // pageable source: the copy is staged before the call returns
    CK(cudaMemcpyAsync(b, &h, sizeof h, cudaMemcpyHostToDevice, s), "bvf_state_save");
    CK(cudaMemcpyAsync(b + t.off_fields, c->fields, t.fields, cudaMemcpyDeviceToDevice, s), "bvf_state_save");
    if (t.psi) CK(cudaMemcpyAsync(b + t.off_psi, c->psi, t.psi, cudaMemcpyDeviceToDevice, s), "bvf_state_save");
    CK(cudaMemcpyAsync(b + t.off_peak, c->peak, t.peak, cudaMemcpyDeviceToDevice, s), "bvf_state_save");
    if (c->dftC) {
        CK(cudaMemcpyAsync(b + t.off_C, c->dftC, t.dft, cudaMemcpyDeviceToDevice, s), "bvf_state_save");
        CK(cudaMemcpyAsync(b + t.off_S, c->dftS, t.dft, cudaMemcpyDeviceToDevice, s), "bvf_state_save");
    } else {
        CK(cudaMemsetAsync(b + t.off_C, 0, 2 * (t.off_S - t.off_C), s), "bvf_state_save");
    }
    CK(cudaMemcpyAsync(b + t.off_flag, c->flag, t.flag, cudaMemcpyDeviceToDevice, s), "bvf_state_save");
    return BVF_OK;
}

int bvf_state_load(bvf_ctx *c, const void *d_buf, size_t bytes, void *stream)
{
    if (!c || !d_buf) return fail(c, BVF_E_ARG, "bvf_state_load: NULL argument");
    const StateSections t = state_sections(c);
    if (bytes < t.total) return fail(c, BVF_E_ARG, "bvf_state_load: buffer smaller than bvf_state_bytes");
    cudaStream_t s = (cudaStream_t)stream;
    const char *b = static_cast<const char *>(d_buf);
    StateHeader h{};
    CK(cudaMemcpyAsync(&h, b, sizeof h, cudaMemcpyDeviceToHost, s), "bvf_state_load");
    CK(cudaStreamSynchronize(s), "bvf_state_load");
    if (h.magic != kStateMagic || h.version != BVF_VERSION || h.bytes != t.total)
        return fail(c, BVF_E_ARG, "bvf_state_load: not a snapshot of this library version and layout");
    if (h.nx != c->g.nx || h.ny != c->g.ny || h.nz != c->g.nz || h.L != c->L || h.h16 != c->h16 ||
        h.dx != c->g.dx || h.dt != c->g.dt || h.f0 != c->ph.f0)
        return fail(c, BVF_E_ARG, "bvf_state_load: snapshot of a different grid, time step, "
                                  "frequency, SLS count or storage");
    if (h.has_dft) {
        const int rc = ensure_dft(c, s);
        if (rc != BVF_OK) return rc;
    }
    CK(cudaMemcpyAsync(c->fields, b + t.off_fields, t.fields, cudaMemcpyDeviceToDevice, s), "bvf_state_load");
    if (t.psi) CK(cudaMemcpyAsync(c->psi, b + t.off_psi, t.psi, cudaMemcpyDeviceToDevice, s), "bvf_state_load");
    CK(cudaMemcpyAsync(c->peak, b + t.off_peak, t.peak, cudaMemcpyDeviceToDevice, s), "bvf_state_load");
    if (c->dftC) {
        CK(cudaMemcpyAsync(c->dftC, b + t.off_C, t.dft, cudaMemcpyDeviceToDevice, s), "bvf_state_load");
        CK(cudaMemcpyAsync(c->dftS, b + t.off_S, t.dft, cudaMemcpyDeviceToDevice, s), "bvf_state_load");
    }
    CK(cudaMemcpyAsync(c->flag, b + t.off_flag, t.flag, cudaMemcpyDeviceToDevice, s), "bvf_state_load");
    c->steps = h.steps;
    c->dft_count = (int)h.dft_count;
    return BVF_OK;
}

// ---- phased sources ---------------------------------------------------------

int bvf_bowl_array(const bvf_bowl *bw, int n_rings, int n_inner, double *h_elem, int *n_out)
{
    if (!bw || !n_out || n_rings < 1 || n_inner < 1)
        return fail(nullptr, BVF_E_ARG, "bvf_bowl_array: bad argument");
    const double a = 0.5 * bw->aperture, R = bw->roc;
    if (!(a > 0.0) || !(R >= a)) return fail(nullptr, BVF_E_ARG, "bvf_bowl_array: need 0 < aperture/2 <= roc");
    double ux = bw->dir[0], uy = bw->dir[1], uz = bw->dir[2];
    const double nrm = std::sqrt(ux * ux + uy * uy + uz * uz);
    if (!(nrm > 0.0)) return fail(nullptr, BVF_E_ARG, "bvf_bowl_array: zero direction");
    ux /= nrm; uy /= nrm; uz /= nrm;
    // rotation taking +z to the axis: about z x u by the angle between them
    double kx = -uy, ky = ux;
    const double sn = std::sqrt(kx * kx + ky * ky), cs = uz;
    if (sn > 0.0) { kx /= sn; ky /= sn; }
    const double thmax = std::asin(a / R);
    int n = 0;
    for (int r = 0; r < n_rings; ++r) {
        const double t0 = thmax * r / n_rings, t1 = thmax * (r + 1) / n_rings, tc = 0.5 * (t0 + t1);
        const int m = n_inner * (r + 1);
        const double area = 2.0 * kPi * R * R * (std::cos(t0) - std::cos(t1)) / m;
        for (int e = 0; e < m; ++e, ++n) {
            if (!h_elem) continue;
            const double ph = 2.0 * kPi * (e + 0.5) / m;
            const double px = R * std::sin(tc) * std::cos(ph), py = R * std::sin(tc) * std::sin(ph);
            const double pz = R * (1.0 - std::cos(tc));
            const double kp = kx * px + ky * py;
            const double cx = ky * pz, cy = -kx * pz, cz = kx * py - ky * px;
            double *row = h_elem + 6 * (size_t)n;
            row[0] = bw->apex[0] + px * cs + cx * sn + kx * kp * (1.0 - cs);
            row[1] = bw->apex[1] + py * cs + cy * sn + ky * kp * (1.0 - cs);
            row[2] = bw->apex[2] + pz * cs + cz * sn;
            row[3] = area;
            row[4] = 1.0;
            row[5] = 0.0;
        }
    }
    *n_out = n;
    return BVF_OK;
}

int bvf_steer_weights(double *h_elem, int ne, const double *target, double f0, double c0)
{
    if (!h_elem || !target || ne < 1 || !(f0 > 0.0) || !(c0 > 0.0))
        return fail(nullptr, BVF_E_ARG, "bvf_steer_weights: bad argument");
    const double k = 2.0 * kPi * f0 / c0;
    for (int e = 0; e < ne; ++e) {
        double *row = h_elem + 6 * (size_t)e;
        const double dx = row[0] - target[0], dy = row[1] - target[1], dz = row[2] - target[2];
        const double r = std::sqrt(dx * dx + dy * dy + dz * dz);
        row[4] = std::cos(k * r);
        row[5] = std::sin(k * r);
    }
    return BVF_OK;
}

int bvf_time_reversal_plane(bvf_ctx *c, int ti, int tj, int tk, int k_src, int n_steps, double c0,
                            float *d_plane, void *stream)
{
    if (!c || !d_plane) return fail(c, BVF_E_ARG, "bvf_time_reversal_plane: NULL argument");
    const int nx = c->g.nx, ny = c->g.ny, nz = c->g.nz;
    if (ti < 0 || ti >= nx || tj < 0 || tj >= ny || tk < 0 || tk >= nz || k_src < 0 || k_src >= nz)
        return fail(c, BVF_E_ARG, "bvf_time_reversal_plane: target or source plane outside the grid");
    const int M = (int)std::lround(1.0 / (c->ph.f0 * c->g.dt));
    if (M < 1 || n_steps < 2 * M + 1)
        return fail(c, BVF_E_ARG, "bvf_time_reversal_plane: need n_steps > two periods");
    if (!(c0 > 0.0)) return fail(c, BVF_E_ARG, "bvf_time_reversal_plane: bad c0");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t plane = (size_t)nx * ny;
    // temporaries: the point source plane and the 8-byte maximum
    char *tmp = nullptr;
    const size_t src_bytes = (plane * sizeof(float2) + 255) & ~(size_t)255;
    CK(cudaMallocAsync((void **)&tmp, src_bytes + 256, s), "bvf_time_reversal_plane: temporaries");
    float2 *src = reinterpret_cast<float2 *>(tmp);
    unsigned long long *d_max = reinterpret_cast<unsigned long long *>(tmp + src_bytes);
    auto done = [&](int code) {
        cudaFreeAsync(tmp, s);
        return code;
    };
    static const float one[2] = {1.0f, 0.0f};
    cudaError_t e = cudaMemsetAsync(src, 0, plane * sizeof(float2), s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(src + (size_t)tj * nx + ti, one, sizeof one, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return done(cuda_fail(c, e, "bvf_time_reversal_plane: source"));
    int rc = bvf_reset(c, stream);
    if (rc == BVF_OK) rc = bvf_set_source(c, tk, reinterpret_cast<float *>(src), c0, BVF_ENV_RAMP_CW, 0, stream);
    const bvf_capture cap{-1, n_steps - 2 * M + 1, 2 * M};
    if (rc == BVF_OK) rc = bvf_run_acoustic(c, n_steps, &cap, stream);
    if (rc != BVF_OK) return done(rc);
    e = launch_conj_plane(c->dftC + (size_t)k_src * plane, c->dftS + (size_t)k_src * plane, plane,
                          d_max, reinterpret_cast<float2 *>(d_plane), s);
    if (e != cudaSuccess) return done(cuda_fail(c, e, "bvf_time_reversal_plane: conjugate plane"));
    c->launches += 2;
    rc = bvf_synchronize(c, stream);
    if (rc != BVF_OK) return done(rc);
    if ((rc = bvf_reset(c, stream)) != BVF_OK) return done(rc);
    bvf_set_source(c, 0, nullptr, c0, BVF_ENV_NONE, 0, stream);
    return done(BVF_OK);
}

}  // extern "C"
