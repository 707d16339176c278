// lbve_api.cu -- runtime and C ABI (include/lbve.h) of the hybrid LB library.
//
// A handle owns every device buffer of one channel or of a batch of channels (stored one after the
// other in the node planes); allocation happens once in lbve_create / lbve_create_batch, after which
// lbve_step only enqueues kernels on the caller's stream.  The step counter and the per-channel
// parameters live in device memory, so a step is a fixed sequence of launches that needs no host
// state: lbve_step captures 16 steps into a CUDA graph once and replays it.
#include <cuda.h>   // driver API types (the context id check of lbve_fields_host_fixed)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "../../include/lbve.h"
#include "lbve_kernels.cuh"
#include "lbve_collide.cuh"
#include "lbve_tangent.cuh"
#include "lbve_adjoint.cuh"
#include "lbve_formf.cuh"

using namespace lbk;

namespace {

thread_local char g_cuda_err[256] = "";

int cuda_fail(cudaError_t e, const char* what) {
    std::snprintf(g_cuda_err, sizeof g_cuda_err, "%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LBVE_ENOMEM : LBVE_ECUDA;
}

#define LBVE_CUDA(call)                                     \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

constexpr int kGraphSteps = 16;   // steps per captured graph
constexpr int kRebase = 32;       // frame re-base interval of the 16-bit history
constexpr int kMaxChannels = 1 << 16;

}  // namespace

struct lbve {
    lbve_channel_desc d;                 // channel 0 (shared settings of a batch: lattice, grid, precisions)
    std::vector<lbve_channel_desc> descs;
    int nchan = 1;
    int D, Q, NS, N, L;
    long long Npad;
    int pop_dbl;               // 1: populations stored in double
    int hist_dbl;              // 1: history stored (and advanced) in double
    int hist_s16;              // 1: 16-bit block-scaled history (in a per-node frame for form P)
    int hist_formf = 0;        // 1: form F, the factor storage (per point F - 1 and kappa + kappa^T, written once)
    int part_ns = 0;           // components per chunk record of the sweep: NS (form P), NS + d*d (form F)
    int model = LBVE_MODEL_NLM;  // constitutive model (LBVE_MODEL_*)
    size_t pesz, hesz;         // element sizes of populations and history (partial sums)
    std::vector<Chan> chan_host;
    Chan* chan_dev = nullptr;  // [nchan] per-channel geometry and parameters
    int* chan_of = nullptr;    // [Npad] channel of every node (batches only)
    void* pops[2] = {nullptr, nullptr};
    int cur = 0;
    void* u_raw = nullptr;
    void* u = nullptr;
    void* rho = nullptr;
    void* sigma = nullptr;
    void* kappa = nullptr;
    void* tr_prev = nullptr;
    void* X = nullptr;
    void* K = nullptr;
    void* part = nullptr;      // sweep partial sums [S][NS][Npad] (history type)
    void* Qe = nullptr;        // 16-bit history: exponents of Q - 1 [L][Npad]
    void* Ke = nullptr;        //                 exponents of kappa [L][Npad]
    void* Rm = nullptr;        //                 frame R - 1 [DD][Npad] (float)
    void* gam_node = nullptr;  // White-Metzner form: accumulated strain Gamma(t) per node [Npad] (double)
    void* gam_pt = nullptr;    //                     Gamma(t') of every point [L][Npad] (double)
    int S = 1;                 // slot chunks of the sweep (autotuned at create)
    int sweep_grid = 0;        // persistent CTAs of the sweep
    int sweep_cta = 0;         // k_sweep task mode: 0 warp tasks, 1 CTA tasks (autotuned at create)
    int sweep_grid_full = 0;   // resident CTAs of the sweep on this device (SMs x CTAs per SM)
    int tuned_from_cache = 0;  // 1: the launch shape came from an earlier handle of the same shape
    int part_S = 0;            // slot chunks the partial-sum buffer holds
    int node_tpb = 256;        // threads per block of the per-node kernels (moments, commit + collide)
    long long* t_dev = nullptr;
    double* red = nullptr;     // reduction scratch (2 doubles)
    double* stage = nullptr;   // lbve_fields staging for host destinations
    size_t stage_n = 0;
    int64_t t_host = 0;
    size_t bytes = 0;
    int* flag = nullptr;       // non-finite flag of lbve_fields
    lbve_allocator al{};       // device-memory provider (lbve_create_ex); alloc == NULL: cudaMalloc / cudaFree
    // probe recorder (lbve_set_probes): records [cap][1 + probe_n (1 + D + NS)] appended after steps
    int probe_n = 0;
    int probe_every = 1;
    long long probe_cap = 0;
    long long* probe_nodes = nullptr;   // [probe_n] node indices
    double* probe_rec = nullptr;        // [probe_cap][record] records
    long long* probe_cnt = nullptr;     // records taken (may exceed probe_cap)
    // captured steps: kGraphSteps steps, both population parities (the graph is replayed from cur == 0)
    cudaGraphExec_t graph = nullptr;
    cudaStream_t graph_stream = nullptr;
    // tangent-linear mode (lbve_create_tangent): all state buffers hold duals
    int tangent = 0;
    // recording for the adjoint (lbve_create_adjoint): a state image every rec_K steps
    int rec_K = 0;
    std::vector<void*> ckpts;
    // kernel timing (lbve_profile): event pairs recorded around each launch of lbve_step
    int profiling = 0;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<int> ev_kind;  // kernel id of each recorded pair
};

namespace {

void dev_free(lbve* h, void* p, cudaStream_t s = 0);

void free_all(lbve* h) {
    void* ptrs[] = {h->pops[0], h->pops[1], h->u_raw, h->u, h->rho, h->sigma, h->kappa, h->tr_prev,
                    h->X, h->K, h->part, h->t_dev, h->red, h->stage, h->flag, h->chan_dev, h->chan_of,
                    h->Qe, h->Ke, h->Rm, h->gam_node, h->gam_pt, h->probe_nodes, h->probe_rec, h->probe_cnt};
    for (void* p : ptrs) dev_free(h, p);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    h->ev_pool.clear();
    for (void* c : h->ckpts) dev_free(h, c);
    h->ckpts.clear();
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->graph_stream) cudaStreamDestroy(h->graph_stream);
    h->graph = nullptr;
    h->graph_stream = nullptr;
}

// Kernel timing: mark(h, s, kind, true) before a launch and mark(h, s, kind, false) after it.
enum { KIND_MOMENTS = 0, KIND_HISTORY = 1, KIND_COLLIDE = 2, KIND_COUNT = 3 };

int prof_mark(lbve* h, cudaStream_t s, int kind, bool start) {
    if (!h->profiling) return LBVE_OK;
    if (h->ev_used == h->ev_pool.size()) {
        cudaEvent_t e;
        LBVE_CUDA(cudaEventCreate(&e));
        h->ev_pool.push_back(e);
    }
    LBVE_CUDA(cudaEventRecord(h->ev_pool[h->ev_used++], s));
    if (start) h->ev_kind.push_back(kind);
    return LBVE_OK;
}

// Device memory through the handle's provider (or cudaMalloc): every buffer the handle owns and the work
// buffers of its calls.  Buffers must start on 256-byte boundaries (the kernels' vector accesses).
int dev_alloc(lbve* h, void** p, size_t bytes, cudaStream_t s = 0) {
    *p = nullptr;
    if (h->al.alloc) {
        void* q = h->al.alloc(bytes, (void*)s, h->al.ctx);
        if (!q) return LBVE_ENOMEM;
        if (reinterpret_cast<uintptr_t>(q) & 255u) {
            h->al.free(q, (void*)s, h->al.ctx);
            std::snprintf(g_cuda_err, sizeof g_cuda_err, "allocator returned memory not aligned to 256 bytes");
            return LBVE_ENOMEM;
        }
        *p = q;
        return LBVE_OK;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, "cudaMalloc");
    }
    return LBVE_OK;
}

void dev_free(lbve* h, void* p, cudaStream_t s) {
    if (!p) return;
    if (h->al.alloc) h->al.free(p, (void*)s, h->al.ctx);
    else cudaFree(p);
}

int alloc(lbve* h, void** p, size_t bytes) {
    int rc = dev_alloc(h, p, bytes);
    if (rc == LBVE_OK) h->bytes += bytes;
    return rc;
}

Geom geom_of(const lbve* h) {
    Geom g;
    g.N = h->N;
    g.Npad = h->Npad;
    g.nchan = h->nchan;
    g.ch = h->chan_dev;
    g.chan_of = h->chan_of;
    return g;
}

// Per-channel device entry from a description (parameters of Sec. III / Eq. nlmax).
void fill_chan(const lbve_channel_desc& d, int off, Chan* c) {
    c->off = off;
    c->nx = d.nx;
    c->ny = d.ny;
    c->nz = d.nz;
    c->wall_z = d.lattice == LBVE_D3Q19 ? d.wall_z : 0;
    c->trace_full = d.trace_coupling == LBVE_TRACE_FULL;
    c->rho0 = d.rho0;
    c->tau_lb = d.tau_lb;
    c->omega = 1.0 / d.tau_lb;
    for (int a = 0; a < 3; ++a) c->f[a] = d.rho0 * d.g[a];
    c->G_inf = d.G_inf;
    c->inv_tau = 1.0 / d.tau;
    c->inv_gc = std::isinf(d.gamma_c) ? 0.0 : 1.0 / d.gamma_c;
    c->xbc = d.x_boundary == LBVE_X_PRESSURE;
    c->drho_gh = c->xbc ? 3.0 * d.dp * (d.nx + 1.0) / (2.0 * d.nx) : 0.0;   // (dp / c_s^2)(nx + 1)/(2 nx)
    c->rho0_f = (float)c->rho0;
    c->omega_f = (float)c->omega;
    for (int a = 0; a < 3; ++a) c->f_f[a] = (float)c->f[a];
    c->G_inf_f = (float)c->G_inf;
    c->drho_gh_f = (float)c->drho_gh;
}

int check_desc(const lbve_channel_desc* d) {
    if (!d) return LBVE_EINVAL;
    if (d->lattice != LBVE_D2Q9 && d->lattice != LBVE_D3Q19) return LBVE_EINVAL;
    if (d->nx < 1 || d->ny < 2 || d->nz < 1) return LBVE_EINVAL;
    if (d->lattice == LBVE_D2Q9 && d->nz != 1) return LBVE_EINVAL;
    if (d->lattice == LBVE_D3Q19 && d->wall_z && d->nz < 2) return LBVE_EINVAL;
    if ((long long)d->nx * d->ny * d->nz > (1ll << 30)) return LBVE_EINVAL;
    if (!(d->tau_lb > 0.5) || !(d->rho0 > 0) || !(d->G_inf >= 0) || !(d->tau > 0) || !(d->gamma_c > 0))
        return LBVE_EINVAL;
    if (!std::isfinite(d->tau_lb) || !std::isfinite(d->rho0) || !std::isfinite(d->G_inf) || !std::isfinite(d->tau))
        return LBVE_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(d->g[a])) return LBVE_EINVAL;
    // explicit stress coupling: shear-wave speed sqrt(G_inf/rho0) well below the lattice speed
    if (std::sqrt(d->G_inf / d->rho0) > 0.5) return LBVE_EINVAL;
    if (d->hist_C < 4 || d->hist_B < 1 || d->hist_B > LBVE_MAXB) return LBVE_EINVAL;
    if ((long long)d->hist_C * d->hist_B > 4096) return LBVE_EINVAL;
    if (d->trace_coupling != LBVE_TRACE_FULL && d->trace_coupling != LBVE_TRACE_NONE) return LBVE_EINVAL;
    if (d->pop_precision != LBVE_F32 && d->pop_precision != LBVE_F64) return LBVE_EINVAL;
    if (d->hist_storage != LBVE_F32 && d->hist_storage != LBVE_F64 && d->hist_storage != LBVE_BF16 &&
        d->hist_storage != LBVE_S16)
        return LBVE_EINVAL;
    if (d->model != LBVE_MODEL_NLM && d->model != LBVE_MODEL_INLM && d->model != LBVE_MODEL_WM) return LBVE_EINVAL;
    if (d->x_boundary != LBVE_X_PERIODIC && d->x_boundary != LBVE_X_PRESSURE) return LBVE_EINVAL;
    if (d->x_boundary == LBVE_X_PRESSURE && !std::isfinite(d->dp)) return LBVE_EINVAL;
    if (d->hist_form != LBVE_FORM_P && d->hist_form != LBVE_FORM_F) return LBVE_EINVAL;
    if (d->hist_storage == LBVE_BF16) return LBVE_ENOSUPPORT;
    if (d->model == LBVE_MODEL_WM && d->hist_storage == LBVE_S16) return LBVE_ENOSUPPORT;
    if (d->model == LBVE_MODEL_WM && d->hist_form == LBVE_FORM_F) return LBVE_ENOSUPPORT;
    return LBVE_OK;
}

// Settings every channel of a batch shares: the lattice, the history grid, the precisions, rho0.
bool same_batch_settings(const lbve_channel_desc& a, const lbve_channel_desc& b) {
    return a.lattice == b.lattice && a.hist_C == b.hist_C && a.hist_B == b.hist_B &&
           a.hist_storage == b.hist_storage && a.pop_precision == b.pop_precision && a.rho0 == b.rho0 &&
           a.model == b.model && a.hist_form == b.hist_form;
}

// Values per lane of the sweep (one 16-byte access): 4 floats or 2 doubles; 3D halves it (registers).
template <int D, typename R> constexpr int sweep_vn() { return (sizeof(R) == 4 ? 4 : 2) / (D == 3 ? 2 : 1); }

template <int D, typename R>
int launch_sweep(lbve* h, cudaStream_t s) {
    constexpr int VN = sweep_vn<D, R>();
    SweepArgs<R> a;
    a.X = (R*)h->X;
    a.K = (const R*)h->K;
    a.part = (R*)h->part;
    a.t_dev = h->t_dev;
    a.B = h->d.hist_B;
    a.C = h->d.hist_C;
    a.S = h->S;
    a.cta_tasks = h->sweep_cta;
    a.gam_node = (const double*)h->gam_node;
    a.gam_pt = (const double*)h->gam_pt;
    if (h->model == LBVE_MODEL_WM)
        k_sweep<D, R, VN, true><<<h->sweep_grid, 256, sweep_cta_smem_bytes(h->L), s>>>(a, geom_of(h));
    else
        k_sweep<D, R, VN, false><<<h->sweep_grid, 256, sweep_cta_smem_bytes(h->L), s>>>(a, geom_of(h));
    LBVE_CUDA(cudaGetLastError());
    return LBVE_OK;
}

CommitS16 commit_s16(lbve* h) {
    CommitS16 c;
    c.Qm = (unsigned short*)h->X;
    c.Qe = (unsigned char*)h->Qe;
    c.Km = (unsigned short*)h->K;
    c.Ke = (unsigned char*)h->Ke;
    c.Rm = (float*)h->Rm;
    c.part = (const float*)h->part;
    c.B = h->d.hist_B;
    c.C = h->d.hist_C;
    c.S = h->S;
    c.TB = kRebase;
    return c;
}

template <int D> constexpr int sweep_vn_s16() { return D == 2 ? 4 : 2; }

template <int D>
int launch_sweep_s16(lbve* h, cudaStream_t s) {
    constexpr int VN = sweep_vn_s16<D>();
    k_sweep_s16<D, VN><<<h->sweep_grid, 256, sweep_smem_bytes(h->L), s>>>(commit_s16(h), (const double*)h->kappa,
                                                                           h->t_dev, geom_of(h));
    LBVE_CUDA(cudaGetLastError());
    return LBVE_OK;
}

template <typename R>
CommitF<R> commit_f(lbve* h) {
    CommitF<R> c;
    c.Y = (R*)h->X;
    c.Dm = (R*)h->K;
    c.part = (R*)h->part;
    c.B = h->d.hist_B;
    c.C = h->d.hist_C;
    c.S = h->S;
    return c;
}

CommitF16 commit_f16(lbve* h) {
    CommitF16 c;
    c.blk = (unsigned char*)h->X;
    c.part = (float*)h->part;
    c.B = h->d.hist_B;
    c.C = h->d.hist_C;
    c.S = h->S;
    c.bal_nw = h->sweep_cta == 2 ? h->sweep_grid * 8 : 0;   // balanced ranges: one warp per 32 threads of the grid
    return c;
}

template <int D, typename R> constexpr int sweep_vn_f() { return (sizeof(R) == 4 ? 4 : 2) / (D == 3 ? 2 : 1); }

template <int D, typename R>
int launch_sweep_f(lbve* h, cudaStream_t s) {
    constexpr int VN = sweep_vn_f<D, R>();
    k_sweep_f<D, R, VN><<<h->sweep_grid, 256, sweep_f_smem_bytes(h->L), s>>>(commit_f<R>(h), h->t_dev, geom_of(h));
    LBVE_CUDA(cudaGetLastError());
    return LBVE_OK;
}

template <int D>
int launch_sweep_f16(lbve* h, cudaStream_t s) {
    constexpr int VN = sweep_vn_s16<D>();
    k_sweep_f16<D, VN><<<h->sweep_grid, 256, sweep_f_smem_bytes(h->L), s>>>(commit_f16(h), h->t_dev, geom_of(h));
    LBVE_CUDA(cudaGetLastError());
    return LBVE_OK;
}

// History kinds (template argument HK): form P in float (0), double (1), 16-bit block-scaled in a per-node
// frame (2); 3 none (the instantaneous model); form F (the factor storage) in float (4), double (5), 16-bit
// block-scaled (6).  Form P in float and double also carries the White-Metzner form (chosen at run time).
template <int D, int HK>
int launch_sweep_any(lbve* h, cudaStream_t s) {
    if (HK == 3) return LBVE_OK;
    if (HK == 6) return launch_sweep_f16<D>(h, s);
    if (HK == 5) return launch_sweep_f<D, double>(h, s);
    if (HK == 4) return launch_sweep_f<D, float>(h, s);
    if (HK == 2) return launch_sweep_s16<D>(h, s);
    if (HK == 1) return launch_sweep<D, double>(h, s);
    return launch_sweep<D, float>(h, s);
}

template <int D, int HK> struct SweepKernel;
template <int D> struct SweepKernel<D, 0> {
    static constexpr int VN = sweep_vn<D, float>();
    static const void* fn(bool wm) { return wm ? (const void*)k_sweep<D, float, VN, true> : (const void*)k_sweep<D, float, VN, false>; }
};
template <int D> struct SweepKernel<D, 1> {
    static constexpr int VN = sweep_vn<D, double>();
    static const void* fn(bool wm) { return wm ? (const void*)k_sweep<D, double, VN, true> : (const void*)k_sweep<D, double, VN, false>; }
};
template <int D> struct SweepKernel<D, 2> {
    static constexpr int VN = sweep_vn_s16<D>();
    static const void* fn(bool) { return (const void*)k_sweep_s16<D, VN>; }
};
template <int D> struct SweepKernel<D, 4> {
    static constexpr int VN = sweep_vn_f<D, float>();
    static const void* fn(bool) { return (const void*)k_sweep_f<D, float, VN>; }
};
template <int D> struct SweepKernel<D, 5> {
    static constexpr int VN = sweep_vn_f<D, double>();
    static const void* fn(bool) { return (const void*)k_sweep_f<D, double, VN>; }
};
template <int D> struct SweepKernel<D, 6> {
    static constexpr int VN = sweep_vn_s16<D>();
    static const void* fn(bool) { return (const void*)k_sweep_f16<D, VN>; }
};

// Autotuner of the sweep: candidate (task mode, slot-chunk count S) pairs -- warp tasks with about 2 to
// 32 tasks per resident warp, (k_sweep) CTA tasks with 1 to 8 tasks per resident CTA, and (16-bit form F)
// balanced ranges over all resident warps -- each timed on a few single launches on the freshly created,
// all-rest history (which the sweep leaves unchanged: exp(0) - 1 = 0), together with the commit's reduction
// of the S partial sums (k_part_read); the candidate with the fastest launch is kept.  The partial-sum buffer is sized for the largest candidate and then trimmed by reallocation.
// Launch shapes the autotuner has chosen in this process, keyed by everything the sweep's speed depends on
// (device and its SM count, lattice, history storage and model, history grid, padded node count), so that
// a second handle of the same shape -- a user re-creating a channel, a batch of equal size -- is not timed
// again.
struct TuneKey {
    int dev, sms, D, HK, wm, B, C;
    long long Npad;
    bool operator==(const TuneKey& o) const {
        return dev == o.dev && sms == o.sms && D == o.D && HK == o.HK && wm == o.wm && B == o.B && C == o.C &&
               Npad == o.Npad;
    }
};
struct TuneVal { int S, cta, grid, grid_full; };
std::mutex g_tune_mu;
std::vector<std::pair<TuneKey, TuneVal>> g_tune_cache;

template <int D, int HK>
int sweep_autotune(lbve* h) {
    constexpr int VN = SweepKernel<D, HK>::VN;
    const void* fn = SweepKernel<D, HK>::fn(h->model == LBVE_MODEL_WM);
    const bool has_cta = HK == 0 || HK == 1;   // the 16-bit and form-F sweeps run warp tasks only
    const size_t smem = HK >= 4 ? sweep_f_smem_bytes(h->L) : has_cta ? sweep_cta_smem_bytes(h->L) : sweep_smem_bytes(h->L);
    if (smem > 48 * 1024)
        LBVE_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0, per_sm = 0;
    LBVE_CUDA(cudaGetDevice(&dev));
    LBVE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const TuneKey key{dev, sms, D, HK, h->model == LBVE_MODEL_WM ? 1 : 0, h->d.hist_B, h->d.hist_C, h->Npad};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        for (const auto& kv : g_tune_cache)
            if (kv.first == key) {
                h->S = kv.second.S;
                h->sweep_cta = kv.second.cta;
                h->sweep_grid = kv.second.grid;
                h->sweep_grid_full = kv.second.grid_full;
                h->tuned_from_cache = 1;
                break;
            }
    }
    if (h->tuned_from_cache) {
        int rc = alloc(h, &h->part, h->hesz * (size_t)h->S * h->part_ns * h->Npad);
        if (rc) return rc;
        LBVE_CUDA(cudaMemset(h->part, 0, h->hesz * (size_t)h->S * h->part_ns * h->Npad));
        h->part_S = h->S;
        return LBVE_OK;
    }
    LBVE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, smem));
    if (per_sm < 1) per_sm = 1;
    const long long grid_full = (long long)sms * per_sm;
    const long long warps = grid_full * 8;
    const long long tiles = h->Npad / (32 * VN);
    const long long Smax = h->L >= 16 ? h->L / 8 : 1;
    struct Cand { int cta; long long S; };
    std::vector<Cand> cand;
    auto add = [&](int cta, long long S) {
        S = std::max(1ll, std::min(S, Smax));
        for (const Cand& c : cand)
            if (c.cta == cta && c.S == S) return;
        cand.push_back({cta, S});
    };
    // task counts just above and just below k waves of the resident warps (CTAs)
    for (long long k : {1, 2, 4, 8, 16, 32}) {
        add(0, (k * warps + tiles - 1) / tiles);
        add(0, k * warps / tiles);
    }
    // few nodes: the tasks above all hit Smax; fewer, longer chunks trade sweep parallelism for a
    // shorter reduction in the commit
    for (long long S = 8; S < Smax; S *= 2) add(0, S);
    if (has_cta)
        for (long long k : {1, 2, 4, 8}) {
            add(1, (k * grid_full + tiles - 1) / tiles);
            add(1, k * grid_full / tiles);
        }
    // 16-bit form F: balanced ranges over all resident warps (S = the most pieces a tile can be cut into)
    if (HK == 6 && f16_bal_max_pieces(tiles, (int)warps) <= Smax) add(2, f16_bal_max_pieces(tiles, (int)warps));
    long long Sbig = 1;
    for (const Cand& c : cand) Sbig = std::max(Sbig, c.S);
    int rc = alloc(h, &h->part, h->hesz * (size_t)Sbig * h->part_ns * h->Npad);
    if (rc) return rc;
    LBVE_CUDA(cudaMemset(h->part, 0, h->hesz * (size_t)Sbig * h->part_ns * h->Npad));
    auto grid_of = [&](const Cand& c) {
        if (c.cta == 2) return (int)grid_full;
        return (int)std::max(1ll, std::min(grid_full, c.cta ? tiles * c.S : (tiles * c.S + 7) / 8));
    };
    Cand best_c = cand[0];
    float best = 1e30f;
    if (cand.size() > 1) {
        cudaEvent_t e0, e1;
        LBVE_CUDA(cudaEventCreate(&e0));
        LBVE_CUDA(cudaEventCreate(&e1));
        // rounds over all candidates: one untimed (first launches), then two timed for a history of a gigabyte
        // or more (a launch then takes well over 100 us, long against the timer), three below; each launch
        // timed on its own and a candidate's fastest kept, so that neither a one-off stall of the memory
        // system nor the clocks settling while the tuner runs decides the shape.  The number of launches is
        // fixed by the size, so the launches at create do not depend on timings.
        const size_t hist_bytes = (size_t)h->L * h->Npad * (h->D * h->D + (h->hist_formf ? h->NS : h->D * h->D)) *
                                  (h->hist_s16 ? 2 : h->hesz);
        const int reps = hist_bytes >= ((size_t)1 << 30) ? 2 : 3;
        std::vector<float> fastest(cand.size(), 1e30f);
        const int pg = (h->N + h->node_tpb - 1) / h->node_tpb;
        for (int r = 0; r <= reps; ++r)
            for (size_t ci = 0; ci < cand.size(); ++ci) {
                const Cand& c = cand[ci];
                h->S = (int)c.S;
                h->sweep_cta = c.cta;
                h->sweep_grid = grid_of(c);
                LBVE_CUDA(cudaEventRecord(e0, 0));
                if ((rc = launch_sweep_any<D, HK>(h, 0))) return rc;
                if (h->hist_dbl)
                    k_part_read<double, double><<<pg, h->node_tpb>>>((const double*)h->part, (int)c.S, h->part_ns, h->Npad, h->N, h->red);
                else if (h->hist_s16 && !h->pop_dbl)   // the commit's float sums of the 16-bit forms
                    k_part_read<float, float><<<pg, h->node_tpb>>>((const float*)h->part, (int)c.S, h->part_ns, h->Npad, h->N, h->red);
                else
                    k_part_read<float, double><<<pg, h->node_tpb>>>((const float*)h->part, (int)c.S, h->part_ns, h->Npad, h->N, h->red);
                LBVE_CUDA(cudaGetLastError());
                LBVE_CUDA(cudaEventRecord(e1, 0));
                LBVE_CUDA(cudaEventSynchronize(e1));
                float one = 0.f;
                LBVE_CUDA(cudaEventElapsedTime(&one, e0, e1));
                if (r > 0) fastest[ci] = std::min(fastest[ci], one);
            }
        // balanced ranges must win by 3 %: on the 1024 x 512 channel they timed 1 % faster here, on the
        // all-rest history, and 2 % slower in the running steps than two chunks per tile (the duct and the
        // 64-channel batch, where they win by 5 % and more, take them either way)
        for (size_t ci = 0; ci < cand.size(); ++ci) {
            const float t_eff = cand[ci].cta == 2 ? fastest[ci] / 0.97f : fastest[ci];
            if (t_eff < best) { best = t_eff; best_c = cand[ci]; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    h->S = (int)best_c.S;
    h->sweep_cta = best_c.cta;
    h->sweep_grid = grid_of(best_c);
    h->sweep_grid_full = (int)grid_full;
    h->part_S = (int)Sbig;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache.push_back({key, TuneVal{h->S, h->sweep_cta, h->sweep_grid, h->sweep_grid_full}});
    }
    if (best_c.S < Sbig) {   // keep only what the chosen S needs
        dev_free(h, h->part);
        h->bytes -= h->hesz * (size_t)Sbig * h->part_ns * h->Npad;
        h->part = nullptr;
        h->part_S = 0;
        if ((rc = alloc(h, &h->part, h->hesz * (size_t)best_c.S * h->part_ns * h->Npad))) return rc;
        h->part_S = (int)best_c.S;
    }
    return LBVE_OK;
}

template <typename R>
CommitArgs<R> commit_args(lbve* h) {
    CommitArgs<R> c;
    c.X = (R*)h->X;
    c.K = (R*)h->K;
    c.part = (const R*)h->part;
    c.B = h->d.hist_B;
    c.C = h->d.hist_C;
    c.S = h->S;
    c.gam_node = (double*)h->gam_node;
    c.gam_pt = (double*)h->gam_pt;
    return c;
}

__global__ void k_advance_t(long long* t) { *t += 1; }
__global__ void k_set_ll(long long* p, long long v) { *p = v; }

// One hybrid step: moments -> history sweep -> commit + collide + stream.  pops[cur] -> pops[cur ^ 1].
// P: population storage type, HK: history kind (0 float, 1 double, 2 16-bit, 3 none: the instantaneous
// model, whose stress the collide kernel computes itself), T: collision arithmetic.
template <int Q, typename P, int HK, typename T>
int one_step(lbve* h, int cur, cudaStream_t s) {
    constexpr int D = Lattice<Q>::D;
    const Geom g = geom_of(h);
    const int tpb = h->node_tpb;
    const int grid = (h->N + tpb - 1) / tpb;
    const P* din = (const P*)h->pops[cur];
    P* dout = (P*)h->pops[cur ^ 1];
    int rc;
    if ((rc = prof_mark(h, s, KIND_MOMENTS, true))) return rc;
    using M = typename std::conditional<sizeof(P) == 4 && (HK == 2 || HK == 6), float, double>::type;
    k_moments<Q, P, M><<<grid, tpb, 0, s>>>(din, (double*)h->u_raw, g, h->t_dev);
    LBVE_CUDA(cudaGetLastError());
    if ((rc = prof_mark(h, s, KIND_MOMENTS, false))) return rc;
    if (HK != 3) {
        if ((rc = prof_mark(h, s, KIND_HISTORY, true))) return rc;
        if ((rc = launch_sweep_any<D, HK>(h, s))) return rc;
        if ((rc = prof_mark(h, s, KIND_HISTORY, false))) return rc;
    }
    CollArgs<P> c;
    c.dn_in = din;
    c.dn_out = dout;
    c.u_raw = (const double*)h->u_raw;
    c.sigma = (double*)h->sigma;
    c.kappa = (double*)h->kappa;
    c.tr_prev = (double*)h->tr_prev;
    c.rho = (double*)h->rho;
    c.u = (double*)h->u;
    c.t_dev = h->t_dev;
    if ((rc = prof_mark(h, s, KIND_COLLIDE, true))) return rc;
    if (HK == 3) k_collide_stream<Q, P, T, Instant<T>><<<grid, tpb, 0, s>>>(c, Instant<T>{1, 4}, g);
    else if (HK == 6) k_collide_stream<Q, P, T, CommitF16><<<grid, tpb, 0, s>>>(c, commit_f16(h), g);
    else if (HK == 5) k_collide_stream<Q, P, T, CommitF<double>><<<grid, tpb, 0, s>>>(c, commit_f<double>(h), g);
    else if (HK == 4) k_collide_stream<Q, P, T, CommitF<float>><<<grid, tpb, 0, s>>>(c, commit_f<float>(h), g);
    else if (HK == 2) k_collide_stream<Q, P, T, CommitS16><<<grid, tpb, 0, s>>>(c, commit_s16(h), g);
    else if (HK == 1) k_collide_stream<Q, P, T, CommitArgs<double>><<<grid, tpb, 0, s>>>(c, commit_args<double>(h), g);
    else k_collide_stream<Q, P, T, CommitArgs<float>><<<grid, tpb, 0, s>>>(c, commit_args<float>(h), g);
    LBVE_CUDA(cudaGetLastError());
    if ((rc = prof_mark(h, s, KIND_COLLIDE, false))) return rc;
    if (h->probe_n > 0) {
        k_probe<<<1, 256, 0, s>>>((const double*)h->rho, (const double*)h->u, (const double*)h->sigma, h->Npad, D,
                                  h->NS, h->probe_nodes, h->probe_n, h->d.rho0, h->t_dev, h->probe_every,
                                  h->probe_cap, h->probe_rec, h->probe_cnt);
        LBVE_CUDA(cudaGetLastError());
    }
    return LBVE_OK;
}

template <int Q, typename P, int HK, typename T>
int capture_graph(lbve* h) {
    if (!h->graph_stream) LBVE_CUDA(cudaStreamCreateWithFlags(&h->graph_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    LBVE_CUDA(cudaStreamBeginCapture(h->graph_stream, cudaStreamCaptureModeThreadLocal));
    int rc = LBVE_OK;
    for (int i = 0; i < kGraphSteps && rc == LBVE_OK; ++i) rc = one_step<Q, P, HK, T>(h, i & 1, h->graph_stream);
    cudaError_t e = cudaStreamEndCapture(h->graph_stream, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        h->graph = nullptr;
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    return LBVE_OK;
}

int record_checkpoint(lbve* h, cudaStream_t s);

// n steps as launch sequences: whole graphs of kGraphSteps steps (an even count, so populations end where
// they started; the graph is recorded for cur == 0, so a pending odd step is run first), the rest one by one.
// Profiling records per-launch events and therefore launches step by step.
template <int Q, typename P, int HK, typename T>
int advance(lbve* h, int64_t n, cudaStream_t s) {
    int rc;
    if (!h->profiling && n >= kGraphSteps) {
        if (h->cur == 1) {
            if ((rc = one_step<Q, P, HK, T>(h, 1, s))) return rc;
            h->cur = 0;
            h->t_host += 1;
            --n;
        }
        if (n >= kGraphSteps) {
            if (!h->graph && (rc = capture_graph<Q, P, HK, T>(h))) return rc;
            while (n >= kGraphSteps) {
                LBVE_CUDA(cudaGraphLaunch(h->graph, s));
                h->t_host += kGraphSteps;
                n -= kGraphSteps;
            }
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        if ((rc = one_step<Q, P, HK, T>(h, h->cur, s))) return rc;
        h->cur ^= 1;
        h->t_host += 1;
    }
    return LBVE_OK;
}

template <int Q, typename P, int HK, typename T>
int step_impl(lbve* h, int64_t n, cudaStream_t s) {
    if (!h->rec_K) return advance<Q, P, HK, T>(h, n, s);
    // recording for the adjoint: a state image at every multiple of rec_K steps, the steps in between as usual
    int rc;
    while (n > 0) {
        if (h->t_host % h->rec_K == 0 && (rc = record_checkpoint(h, s))) return rc;
        const int64_t seg = std::min<int64_t>(n, h->rec_K - h->t_host % h->rec_K);
        if ((rc = advance<Q, P, HK, T>(h, seg, s))) return rc;
        n -= seg;
    }
    return LBVE_OK;
}

// Population storage P (collision arithmetic the same type) x history kind.
template <int Q, typename P>
int step_dispatch(lbve* h, int hk, int64_t n, cudaStream_t s) {
    switch (hk) {
        case 0: return step_impl<Q, P, 0, P>(h, n, s);
        case 1: return step_impl<Q, P, 1, P>(h, n, s);
        case 2: return step_impl<Q, P, 2, P>(h, n, s);
        case 3: return step_impl<Q, P, 3, P>(h, n, s);
        case 4: return step_impl<Q, P, 4, P>(h, n, s);
        case 5: return step_impl<Q, P, 5, P>(h, n, s);
        default: return step_impl<Q, P, 6, P>(h, n, s);
    }
}

// Fluid at rest: n_q = w_q rho_init(n) (deviation w_q (rho_init - rho0)), density field rho_init - rho0.
template <typename P>
__global__ void k_init(P* dn, double* rho, long long Npad, int N, int Q, const double* rho_init, double rho0,
                       const double* w) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const double r = rho_init ? rho_init[n] : rho0;
    for (int q = 0; q < Q; ++q) dn[q * Npad + n] = (P)(w[q] * (r - rho0));
    rho[n] = r - rho0;
}

template <typename P>
int init_state(lbve* h, const double* rho_init_host) {
    double w[19];
    for (int q = 0; q < h->Q; ++q) w[q] = h->Q == 9 ? Lattice<9>::w(q) : Lattice<19>::w(q);
    double* tmp = nullptr;   // [Q] weights then [N] initial densities
    const size_t n_tmp = h->Q + (rho_init_host ? (size_t)h->N : 0);
    int rc = dev_alloc(h, (void**)&tmp, sizeof(double) * n_tmp);
    if (rc) return rc;
    cudaError_t e = cudaMemcpy(tmp, w, sizeof(double) * h->Q, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && rho_init_host)
        e = cudaMemcpy(tmp + h->Q, rho_init_host, sizeof(double) * h->N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_init<P><<<(h->N + 255) / 256, 256>>>((P*)h->pops[0], (double*)h->rho, h->Npad, h->N, h->Q,
                                               rho_init_host ? tmp + h->Q : nullptr, h->d.rho0, tmp);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    dev_free(h, tmp);
    if (e != cudaSuccess) return cuda_fail(e, "initial state");
    return LBVE_OK;
}

// The field gathers of lbve_fields into device memory `dst`, raising the device flag `flag` on a non-finite
// value (the handle's own flag, or the one kept in the fixed staging array of lbve_fields_host_fixed).
int fields_impl(lbve* h, uint32_t mask, double* dst, int* flag, cudaStream_t s) {
    using real = double;   // node fields are kept in double
    const long long Np = h->Npad;
    const int N = h->N;
    size_t off = 0;
    auto gather = [&](const void* src, int ncomp, double offset) -> int {
        const long long tot = (long long)ncomp * N;
        if (tot > 0) {
            k_gather<real><<<(int)((tot + 255) / 256), 256, 0, s>>>((const real*)src, Np, ncomp, N, offset,
                                                                      dst + off, flag);
            LBVE_CUDA(cudaGetLastError());
        }
        off += (size_t)tot;
        return LBVE_OK;
    };
    int rc;
    if (mask & LBVE_FIELD_RHO) if ((rc = gather(h->rho, 1, h->d.rho0))) return rc;   // stored as rho - rho0
    if (mask & LBVE_FIELD_U) if ((rc = gather(h->u, h->D, 0.0))) return rc;
    if (mask & LBVE_FIELD_SIGMA) if ((rc = gather(h->sigma, h->NS, 0.0))) return rc;
    if (mask & LBVE_FIELD_KAPPA) if ((rc = gather(h->kappa, h->D * h->D, 0.0))) return rc;
    if (mask & LBVE_FIELD_N1) {
        if (N > 0) {
            k_n1<real><<<(N + 255) / 256, 256, 0, s>>>((const real*)h->sigma, Np, N, dst + off, flag);
            LBVE_CUDA(cudaGetLastError());
        }
        off += N;
    }
    return LBVE_OK;
}

// Fields of the node range [n0, n0 + cnt) into dst (device) as values of type O, one block per field in
// increasing bit order, each block component-major; N1 = sigma_xx - sigma_yy.  Node fields are double.
template <typename O>
__global__ void k_gather_range(const double* __restrict__ src, long long Npad, int ncomp, long long n0, int cnt,
                               double offset, int n1, O* __restrict__ dst, int* nonfinite) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)ncomp * cnt) return;
    const int c = (int)(i / cnt);
    const long long n = n0 + (i - (long long)c * cnt);
    const double v = n1 ? src[n] - src[Npad + n] : src[c * Npad + n] + offset;
    dst[i] = (O)v;
    if (!isfinite(v)) atomicOr(nonfinite, 1);
}

template <typename O>
int fields_range_impl(lbve* h, uint32_t mask, long long n0, int cnt, O* dst, int* flag, cudaStream_t s) {
    struct Part { uint32_t bit; const void* src; int ncomp; double offset; int n1; };
    const Part parts[] = {{LBVE_FIELD_RHO, h->rho, 1, h->d.rho0, 0},      // stored as rho - rho0
                          {LBVE_FIELD_U, h->u, h->D, 0.0, 0},
                          {LBVE_FIELD_SIGMA, h->sigma, h->NS, 0.0, 0},
                          {LBVE_FIELD_KAPPA, h->kappa, h->D * h->D, 0.0, 0},
                          {LBVE_FIELD_N1, h->sigma, 1, 0.0, 1}};
    size_t off = 0;
    for (const Part& pt : parts) {
        if (!(mask & pt.bit)) continue;
        const long long tot = (long long)pt.ncomp * cnt;
        if (tot > 0) {
            k_gather_range<O><<<(int)((tot + 255) / 256), 256, 0, s>>>((const double*)pt.src, h->Npad, pt.ncomp, n0,
                                                                       cnt, pt.offset, pt.n1, dst + off, flag);
            LBVE_CUDA(cudaGetLastError());
        }
        off += (size_t)tot;
    }
    return LBVE_OK;
}

size_t fields_count(const lbve* h, uint32_t mask) {
    size_t c = 0;
    if (mask & LBVE_FIELD_RHO) c += 1;
    if (mask & LBVE_FIELD_U) c += h->D;
    if (mask & LBVE_FIELD_SIGMA) c += h->NS;
    if (mask & LBVE_FIELD_KAPPA) c += (size_t)h->D * h->D;
    if (mask & LBVE_FIELD_N1) c += 1;
    return c * (size_t)h->N;
}

template <typename P>
int mass_impl(lbve* h, double* sum_n, double* sum_drho, cudaStream_t s) {
    LBVE_CUDA(cudaMemsetAsync(h->red, 0, 2 * sizeof(double), s));
    const int grid = 4 * 152;
    k_sum<P><<<grid, 256, 0, s>>>((const P*)h->pops[h->cur], h->Npad, h->Q, h->N, 1.0, h->red);
    LBVE_CUDA(cudaGetLastError());
    // delta rho(t-1) = -tr sigma(t-1) / (d cs^2) = -3 tr / d
    k_sum<double><<<grid, 256, 0, s>>>((const double*)h->tr_prev, h->Npad, 1, h->N, -3.0 / h->D, h->red + 1);
    LBVE_CUDA(cudaGetLastError());
    double r[2];
    LBVE_CUDA(cudaMemcpyAsync(r, h->red, sizeof r, cudaMemcpyDeviceToHost, s));
    LBVE_CUDA(cudaStreamSynchronize(s));
    *sum_n = r[0] + h->d.rho0 * (double)h->N;   // populations are stored as n - w rho0
    *sum_drho = r[1];
    return LBVE_OK;
}

int create_impl(const lbve_channel_desc* descs, int32_t n, const double* rho_init, lbve_t** out,
                const lbve_allocator* allocator = nullptr) {
    if (!out) return LBVE_EINVAL;
    *out = nullptr;
    if (!descs || n < 1 || n > kMaxChannels) return LBVE_EINVAL;
    long long Ntot = 0;
    for (int c = 0; c < n; ++c) {
        int rc = check_desc(&descs[c]);
        if (rc) return rc;
        if (!same_batch_settings(descs[0], descs[c])) return LBVE_EINVAL;
        Ntot += (long long)descs[c].nx * descs[c].ny * descs[c].nz;
    }
    if (Ntot > (1ll << 30)) return LBVE_EINVAL;
    if (rho_init) {
        for (long long i = 0; i < Ntot; ++i)
            if (!std::isfinite(rho_init[i]) || !(rho_init[i] > 0)) return LBVE_EINVAL;
    }
    if (allocator && allocator->alloc && !allocator->free) return LBVE_EINVAL;
    lbve* h = new (std::nothrow) lbve();
    if (!h) return LBVE_ENOMEM;
    if (allocator && allocator->alloc) h->al = *allocator;
    const lbve_channel_desc* desc = &descs[0];
    h->d = *desc;
    h->descs.assign(descs, descs + n);
    h->nchan = n;
    h->D = desc->lattice == LBVE_D2Q9 ? 2 : 3;
    h->Q = desc->lattice;
    h->NS = h->D == 2 ? 3 : 6;
    h->N = (int)Ntot;
    {   // Block size of the per-node kernels.  Few nodes: blocks of fewer threads spread them over more SMs
        // (their FP64 work completes a warp instruction in active lanes / 2 cycles).  More nodes: the
        // largest block (<= 256) whose last wave of blocks over the SMs is at least 90 % full, so that no
        // SM holds twice the work of another.  A failed query keeps 256 (the allocations below report a
        // broken device).
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0) {
            int tpb = 1;
            while (tpb < 32 && (h->N + tpb - 1) / tpb > sms) tpb *= 2;
            if (tpb == 32 && (h->N + 31) / 32 > sms)
                for (int b = 256; b >= 32; b /= 2) {
                    const double waves = (double)((h->N + b - 1) / b) / sms;
                    if (b == 32 || std::ceil(waves) <= 1.1 * waves) { tpb = b; break; }
                }
            h->node_tpb = tpb;
        }
    }
    h->model = desc->model;
    h->L = desc->model == LBVE_MODEL_INLM ? 0 : desc->hist_C * desc->hist_B;   // the instantaneous model keeps no history
    h->Npad = ((long long)h->N + 127) / 128 * 128;
    h->pop_dbl = desc->pop_precision == LBVE_F64;
    h->hist_dbl = desc->hist_storage == LBVE_F64;
    h->hist_s16 = desc->hist_storage == LBVE_S16;
    h->hist_formf = desc->hist_form == LBVE_FORM_F && h->L > 0;
    h->part_ns = h->NS + (h->hist_formf ? h->D * h->D : 0);
    h->pesz = h->pop_dbl ? 8 : 4;
    h->hesz = h->hist_dbl ? 8 : 4;
    const size_t hist_elem = h->hist_s16 ? 2 : h->hesz;   // bytes of one stored history component
    // planes per point: form P keeps X = E - 1 and kappa (d*d each); form F keeps F - 1 (d*d) and
    // kappa + kappa^T (NS)
    const int kplanes = h->hist_formf ? h->NS : h->D * h->D;
    // history bytes: X (d*d planes) and K (kplanes); the 16-bit form F keeps both, with their exponents, in
    // one array of 2048-byte blocks, 16 (2D) or 32 (3D) bytes per point
    const bool f16 = h->hist_s16 && h->hist_formf;
    const size_t x_bytes = f16 ? (size_t)h->L * h->Npad * (h->D == 2 ? 16 : 32)
                               : hist_elem * (size_t)h->L * h->D * h->D * h->Npad;
    const size_t k_bytes = f16 ? 0 : hist_elem * (size_t)h->L * kplanes * h->Npad;
    h->chan_host.resize(n);
    {
        int off = 0;
        for (int c = 0; c < n; ++c) {
            fill_chan(descs[c], off, &h->chan_host[c]);
            off += descs[c].nx * descs[c].ny * descs[c].nz;
        }
    }
    const long long Np = h->Npad;
    const int DD = h->D * h->D;
    const size_t fe = sizeof(double);
    int rc;
    auto fail = [&](int code) {
        free_all(h);
        delete h;
        return code;
    };
    if ((rc = alloc(h, &h->pops[0], h->pesz * h->Q * Np)) || (rc = alloc(h, &h->pops[1], h->pesz * h->Q * Np)) ||
        (rc = alloc(h, &h->u_raw, fe * h->D * Np)) || (rc = alloc(h, &h->u, fe * h->D * Np)) ||
        (rc = alloc(h, &h->rho, fe * Np)) || (rc = alloc(h, &h->sigma, fe * h->NS * Np)) ||
        (rc = alloc(h, &h->kappa, fe * DD * Np)) || (rc = alloc(h, &h->tr_prev, fe * Np)) ||
        (h->L > 0 && (rc = alloc(h, &h->X, x_bytes))) ||
        (h->L > 0 && k_bytes > 0 && (rc = alloc(h, &h->K, k_bytes))) ||
        (rc = alloc(h, (void**)&h->t_dev, sizeof(long long))) || (rc = alloc(h, (void**)&h->red, 2 * sizeof(double))) ||
        (rc = alloc(h, (void**)&h->flag, sizeof(int))) ||
        (rc = alloc(h, (void**)&h->chan_dev, sizeof(Chan) * n)))
        return fail(rc);
    {
        cudaError_t e = cudaMemcpy(h->chan_dev, h->chan_host.data(), sizeof(Chan) * n, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemcpy"));
    }
    if (n > 1) {   // channel of every node (padding belongs to the last channel)
        if ((rc = alloc(h, (void**)&h->chan_of, sizeof(int) * Np))) return fail(rc);
        std::vector<int> co((size_t)Np, n - 1);
        for (int c = 0; c < n; ++c) {
            const int nn = descs[c].nx * descs[c].ny * descs[c].nz;
            std::fill(co.begin() + h->chan_host[c].off, co.begin() + h->chan_host[c].off + nn, c);
        }
        cudaError_t e = cudaMemcpy(h->chan_of, co.data(), sizeof(int) * Np, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemcpy"));
    }
    if (h->hist_s16 && !h->hist_formf && h->L > 0 &&
        ((rc = alloc(h, &h->Qe, (size_t)h->L * Np)) || (rc = alloc(h, &h->Ke, (size_t)h->L * Np)) ||
         (rc = alloc(h, &h->Rm, sizeof(float) * DD * Np))))
        return fail(rc);
    if (h->model == LBVE_MODEL_WM &&
        ((rc = alloc(h, &h->gam_node, sizeof(double) * Np)) ||
         (rc = alloc(h, &h->gam_pt, sizeof(double) * (size_t)h->L * Np))))
        return fail(rc);
    // zero every buffer: rest state, empty history (E = 1 <=> X = 0 or Q = 1, kappa = 0, frame 1)
    // (White-Metzner: Gamma = 0 for the node and for every rest point -- no strain before t = 0)
    void* zero_bufs[] = {h->pops[0], h->pops[1], h->u_raw, h->u, h->sigma, h->kappa, h->tr_prev, h->X, h->K, h->flag,
                         h->Qe, h->Ke, h->Rm, h->gam_node, h->gam_pt};
    size_t zero_sizes[] = {h->pesz * h->Q * Np, h->pesz * h->Q * Np, fe * h->D * Np, fe * h->D * Np,
                           fe * h->NS * Np, fe * DD * Np, fe * Np, x_bytes, k_bytes, sizeof(int), (size_t)h->L * Np,
                           (size_t)h->L * Np,
                           sizeof(float) * DD * Np, sizeof(double) * Np, sizeof(double) * (size_t)h->L * Np};
    for (int i = 0; i < 15; ++i) {
        if (!zero_bufs[i]) continue;
        cudaError_t e = cudaMemset(zero_bufs[i], 0, zero_sizes[i]);
        if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemset"));
    }
    {   // the device step counter holds the index of the step in progress; the first step makes it 0
        const long long minus_one = -1;
        cudaError_t e = cudaMemcpy(h->t_dev, &minus_one, sizeof minus_one, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemcpy"));
    }
    if (h->L == 0) rc = LBVE_OK;   // no history: no sweep
    else if (h->hist_formf) {
        if (h->D == 2) rc = h->hist_s16 ? sweep_autotune<2, 6>(h) : h->hist_dbl ? sweep_autotune<2, 5>(h) : sweep_autotune<2, 4>(h);
        else rc = h->hist_s16 ? sweep_autotune<3, 6>(h) : h->hist_dbl ? sweep_autotune<3, 5>(h) : sweep_autotune<3, 4>(h);
    } else if (h->D == 2) rc = h->hist_s16 ? sweep_autotune<2, 2>(h) : h->hist_dbl ? sweep_autotune<2, 1>(h) : sweep_autotune<2, 0>(h);
    else rc = h->hist_s16 ? sweep_autotune<3, 2>(h) : h->hist_dbl ? sweep_autotune<3, 1>(h) : sweep_autotune<3, 0>(h);
    if (rc) return fail(rc);
    rc = h->pop_dbl ? init_state<double>(h, rho_init) : init_state<float>(h, rho_init);
    if (rc) return fail(rc);
    *out = h;
    return LBVE_OK;
}

TanPar tan_par(const lbve* h) {
    const lbve_channel_desc& d = h->descs[0];
    TanPar p;
    p.G_inf = Dual(d.G_inf);
    p.G_inf.d[0] = 1.0;
    p.inv_tau = Dual(1.0 / d.tau);
    p.inv_tau.d[1] = -1.0 / (d.tau * d.tau);
    p.inv_gc = Dual(std::isinf(d.gamma_c) ? 0.0 : 1.0 / d.gamma_c);
    if (!std::isinf(d.gamma_c)) p.inv_gc.d[2] = -1.0 / (d.gamma_c * d.gamma_c);
    for (int a = 0; a < 3; ++a) p.f[a] = Dual(d.rho0 * d.g[a]);
    p.f[0].d[3] = d.rho0;
    p.rho0 = d.rho0;
    p.tau_lb = d.tau_lb;
    p.trace_full = d.trace_coupling == LBVE_TRACE_FULL;
    return p;
}

template <int Q>
int tangent_step(lbve* h, int64_t n, cudaStream_t s) {
    constexpr int D = Lattice<Q>::D;
    const Geom g = geom_of(h);
    const TanPar p = tan_par(h);
    const int grid = (h->N + 127) / 128;
    const size_t smem = sweep_smem_bytes(h->L);
    for (int64_t i = 0; i < n; ++i) {
        const Dual* din = (const Dual*)h->pops[h->cur];
        Dual* dout = (Dual*)h->pops[h->cur ^ 1];
        k_moments_t<Q><<<grid, 128, 0, s>>>(din, (Dual*)h->u_raw, g, p, h->t_dev);
        LBVE_CUDA(cudaGetLastError());
        k_sweep_t<D><<<(int)(((long long)h->S * h->Npad + 127) / 128), 128, smem, s>>>(
            (Dual*)h->X, (const Dual*)h->K, (Dual*)h->part, g, p, h->t_dev, h->d.hist_B, h->d.hist_C, h->S);
        LBVE_CUDA(cudaGetLastError());
        k_history_t<D><<<grid, 128, smem, s>>>((Dual*)h->X, (Dual*)h->K, (const Dual*)h->u_raw, (Dual*)h->kappa,
                                               (Dual*)h->sigma, (const Dual*)h->part, g, p, h->t_dev, h->d.hist_B,
                                               h->d.hist_C, h->S);
        LBVE_CUDA(cudaGetLastError());
        k_collide_t<Q><<<grid, 128, 0, s>>>(din, dout, (const Dual*)h->sigma, (Dual*)h->tr_prev, (Dual*)h->rho,
                                            (Dual*)h->u, g, p);
        LBVE_CUDA(cudaGetLastError());
        h->cur ^= 1;
        h->t_host += 1;
    }
    return LBVE_OK;
}

// Value (k < 0) or derivative k of the selected fields, into device memory, lbve_fields layout.
int tangent_gather(lbve* h, uint32_t mask, int k, double* dst, cudaStream_t s) {
    const long long Np = h->Npad;
    const int N = h->N;
    size_t off = 0;
    struct Part { uint32_t bit; const void* src; int ncomp; double offset; };
    const Part parts[] = {{LBVE_FIELD_RHO, h->rho, 1, h->d.rho0},
                          {LBVE_FIELD_U, h->u, h->D, 0.0},
                          {LBVE_FIELD_SIGMA, h->sigma, h->NS, 0.0},
                          {LBVE_FIELD_KAPPA, h->kappa, h->D * h->D, 0.0}};
    for (const Part& pt : parts) {
        if (!(mask & pt.bit)) continue;
        const long long tot = (long long)pt.ncomp * N;
        if (tot > 0) {
            k_gather_t<<<(int)((tot + 255) / 256), 256, 0, s>>>((const Dual*)pt.src, Np, pt.ncomp, N, k,
                                                                 k < 0 ? pt.offset : 0.0, dst + off);
            LBVE_CUDA(cudaGetLastError());
        }
        off += (size_t)tot;
    }
    if ((mask & LBVE_FIELD_N1) && N > 0) {
        k_n1_t<<<(N + 255) / 256, 256, 0, s>>>((const Dual*)h->sigma, Np, N, k, dst + off);
        LBVE_CUDA(cudaGetLastError());
    }
    return LBVE_OK;
}

template <typename P>
__global__ void k_init_t(Dual* dn, Dual* rho, long long Npad, int N, int Q, const double* rho_init, double rho0,
                         const double* w) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const double r = rho_init ? rho_init[n] : rho0;
    for (int q = 0; q < Q; ++q) dn[q * Npad + n] = Dual(w[q] * (r - rho0));
    rho[n] = Dual(r - rho0);
}

int create_tangent(const lbve_channel_desc* desc, const double* rho_init, lbve_t** out) {
    if (!out) return LBVE_EINVAL;
    *out = nullptr;
    int rc = check_desc(desc);
    if (rc) return rc;
    if (desc->model != LBVE_MODEL_NLM || desc->x_boundary != LBVE_X_PERIODIC) return LBVE_ENOSUPPORT;
    if (desc->hist_form != LBVE_FORM_P) return LBVE_ENOSUPPORT;
    const long long Ntot = (long long)desc->nx * desc->ny * desc->nz;
    if (rho_init)
        for (long long i = 0; i < Ntot; ++i)
            if (!std::isfinite(rho_init[i]) || !(rho_init[i] > 0)) return LBVE_EINVAL;
    lbve* h = new (std::nothrow) lbve();
    if (!h) return LBVE_ENOMEM;
    h->tangent = 1;
    h->d = *desc;
    h->descs.assign(desc, desc + 1);
    h->nchan = 1;
    h->D = desc->lattice == LBVE_D2Q9 ? 2 : 3;
    h->Q = desc->lattice;
    h->NS = h->D == 2 ? 3 : 6;
    h->N = (int)Ntot;
    h->L = desc->hist_C * desc->hist_B;
    h->Npad = ((long long)h->N + 127) / 128 * 128;
    h->pop_dbl = 1;
    h->hist_dbl = 1;
    h->pesz = h->hesz = sizeof(Dual);
    h->chan_host.resize(1);
    fill_chan(*desc, 0, &h->chan_host[0]);
    const long long Np = h->Npad;
    const int DD = h->D * h->D;
    const size_t e = sizeof(Dual);
    auto fail = [&](int code) {
        free_all(h);
        delete h;
        return code;
    };
    if ((rc = alloc(h, &h->pops[0], e * h->Q * Np)) || (rc = alloc(h, &h->pops[1], e * h->Q * Np)) ||
        (rc = alloc(h, &h->u_raw, e * h->D * Np)) || (rc = alloc(h, &h->u, e * h->D * Np)) ||
        (rc = alloc(h, &h->rho, e * Np)) || (rc = alloc(h, &h->sigma, e * h->NS * Np)) ||
        (rc = alloc(h, &h->kappa, e * DD * Np)) || (rc = alloc(h, &h->tr_prev, e * Np)) ||
        (rc = alloc(h, &h->X, e * (size_t)h->L * DD * Np)) || (rc = alloc(h, &h->K, e * (size_t)h->L * DD * Np)) ||
        (rc = alloc(h, (void**)&h->t_dev, sizeof(long long))) || (rc = alloc(h, (void**)&h->flag, sizeof(int))) ||
        (rc = alloc(h, (void**)&h->chan_dev, sizeof(Chan))))
        return fail(rc);
    void* zb[] = {h->pops[0], h->pops[1], h->u_raw, h->u, h->rho, h->sigma, h->kappa, h->tr_prev, h->X, h->K};
    size_t zs[] = {e * h->Q * Np, e * h->Q * Np, e * h->D * Np, e * h->D * Np, e * Np, e * h->NS * Np, e * DD * Np,
                   e * Np, e * (size_t)h->L * DD * Np, e * (size_t)h->L * DD * Np};
    for (int i = 0; i < 10; ++i) {
        cudaError_t er = cudaMemset(zb[i], 0, zs[i]);
        if (er != cudaSuccess) return fail(cuda_fail(er, "cudaMemset"));
    }
    const long long minus_one = -1;
    cudaError_t er = cudaMemcpy(h->t_dev, &minus_one, sizeof minus_one, cudaMemcpyHostToDevice);
    if (er == cudaSuccess) er = cudaMemcpy(h->chan_dev, h->chan_host.data(), sizeof(Chan), cudaMemcpyHostToDevice);
    if (er != cudaSuccess) return fail(cuda_fail(er, "cudaMemcpy"));
    // initial populations w (rho_init - rho0), derivatives 0
    double w[19];
    for (int q = 0; q < h->Q; ++q) w[q] = h->Q == 9 ? Lattice<9>::w(q) : Lattice<19>::w(q);
    double* tmp = nullptr;
    const size_t n_tmp = h->Q + (rho_init ? (size_t)h->N : 0);
    er = dev_alloc(h, (void**)&tmp, sizeof(double) * n_tmp) == LBVE_OK ? cudaSuccess : cudaErrorMemoryAllocation;
    if (er == cudaSuccess) er = cudaMemcpy(tmp, w, sizeof(double) * h->Q, cudaMemcpyHostToDevice);
    if (er == cudaSuccess && rho_init) er = cudaMemcpy(tmp + h->Q, rho_init, sizeof(double) * h->N, cudaMemcpyHostToDevice);
    if (er == cudaSuccess) {
        k_init_t<double><<<(h->N + 255) / 256, 256>>>((Dual*)h->pops[0], (Dual*)h->rho, Np, h->N, h->Q,
                                                       rho_init ? tmp + h->Q : nullptr, h->d.rho0, tmp);
        er = cudaGetLastError();
    }
    if (er == cudaSuccess) er = cudaDeviceSynchronize();
    dev_free(h, tmp);
    if (er != cudaSuccess) return fail(cuda_fail(er, "tangent initial state"));
    const size_t smem = sweep_smem_bytes(h->L);
    if (smem > 48 * 1024) {
        er = cudaFuncSetAttribute(h->D == 2 ? (const void*)k_history_t<2> : (const void*)k_history_t<3>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (er == cudaSuccess)
            er = cudaFuncSetAttribute(h->D == 2 ? (const void*)k_sweep_t<2> : (const void*)k_sweep_t<3>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (er != cudaSuccess) return fail(cuda_fail(er, "cudaFuncSetAttribute"));
    }
    // slot chunks of the dual sweep (about 64k (node, chunk) threads, at most 32) and their partial sums
    h->S = (int)std::max(1ll, std::min<long long>({32ll, (long long)h->L, (65536ll + h->N - 1) / h->N}));
    {
        int rc2 = alloc(h, &h->part, sizeof(Dual) * (size_t)h->S * h->NS * h->Npad);
        if (rc2) return fail(rc2);
        h->part_S = h->S;
    }
    *out = h;
    return LBVE_OK;
}

int push_chan(lbve* h, int c, cudaStream_t s) {
    // the kernels read the table; stream order keeps earlier steps on `s` with the old values.  The
    // source is pageable host memory, so the copy has taken the entry when the call returns.
    LBVE_CUDA(cudaMemcpyAsync(h->chan_dev + c, &h->chan_host[c], sizeof(Chan), cudaMemcpyHostToDevice, s));
    return LBVE_OK;
}

}  // namespace

// =================================================================================================
// C ABI
// =================================================================================================
extern "C" {

int lbve_create(const lbve_channel_desc* desc, const double* rho_init, lbve_t** out) {
    return create_impl(desc, 1, rho_init, out);
}

int lbve_create_batch(const lbve_channel_desc* descs, int32_t n_channels, const double* rho_init, lbve_t** out) {
    return create_impl(descs, n_channels, rho_init, out);
}

int lbve_create_ex(const lbve_channel_desc* descs, int32_t n_channels, const double* rho_init,
                   const lbve_allocator* allocator, lbve_t** out) {
    return create_impl(descs, n_channels, rho_init, out, allocator);
}

int lbve_channel_nodes(const lbve_t* h, int32_t channel, int64_t* offset, int64_t* count) {
    if (!h || !offset || !count || channel < 0 || channel >= h->nchan) return LBVE_EINVAL;
    const lbve_channel_desc& d = h->descs[channel];
    *offset = h->chan_host[channel].off;
    *count = (int64_t)d.nx * d.ny * d.nz;
    return LBVE_OK;
}

void lbve_destroy(lbve_t* h) {
    if (!h) return;
    cudaDeviceSynchronize();
    free_all(h);
    delete h;
}

int lbve_set_force(lbve_t* h, int32_t channel, const double g[3], void* stream) {
    if (!h || !g || channel < -1 || channel >= h->nchan) return LBVE_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(g[a])) return LBVE_EINVAL;
    if (h->tangent) {   // parameters travel as kernel arguments
        for (int a = 0; a < 3; ++a) h->descs[0].g[a] = g[a];
        h->d = h->descs[0];
        return LBVE_OK;
    }
    const int c0 = channel < 0 ? 0 : channel, c1 = channel < 0 ? h->nchan : channel + 1;
    for (int c = c0; c < c1; ++c) {
        for (int a = 0; a < 3; ++a) h->descs[c].g[a] = g[a];
        fill_chan(h->descs[c], h->chan_host[c].off, &h->chan_host[c]);
        int rc = push_chan(h, c, (cudaStream_t)stream);
        if (rc) return rc;
    }
    if (channel <= 0) h->d = h->descs[0];
    return LBVE_OK;
}

int lbve_set_pressure_step(lbve_t* h, int32_t channel, double dp, void* stream) {
    if (!h || channel < -1 || channel >= h->nchan || !std::isfinite(dp)) return LBVE_EINVAL;
    if (h->tangent) return LBVE_ESTATE;
    const int c0 = channel < 0 ? 0 : channel, c1 = channel < 0 ? h->nchan : channel + 1;
    for (int c = c0; c < c1; ++c)
        if (h->descs[c].x_boundary != LBVE_X_PRESSURE) return LBVE_ESTATE;
    for (int c = c0; c < c1; ++c) {
        h->descs[c].dp = dp;
        fill_chan(h->descs[c], h->chan_host[c].off, &h->chan_host[c]);
        int rc = push_chan(h, c, (cudaStream_t)stream);
        if (rc) return rc;
    }
    if (channel <= 0) h->d = h->descs[0];
    return LBVE_OK;
}

int lbve_set_params(lbve_t* h, int32_t channel, double G_inf, double tau, double gamma_c, void* stream) {
    if (!h || channel < -1 || channel >= h->nchan) return LBVE_EINVAL;
    const int c0 = channel < 0 ? 0 : channel, c1 = channel < 0 ? h->nchan : channel + 1;
    for (int c = c0; c < c1; ++c) {
        lbve_channel_desc d = h->descs[c];
        d.G_inf = G_inf;
        d.tau = tau;
        d.gamma_c = gamma_c;
        const int rc = check_desc(&d);
        if (rc) return rc;
    }
    for (int c = c0; c < c1; ++c) {
        h->descs[c].G_inf = G_inf;
        h->descs[c].tau = tau;
        h->descs[c].gamma_c = gamma_c;
        fill_chan(h->descs[c], h->chan_host[c].off, &h->chan_host[c]);
        if (h->tangent) continue;
        int rc = push_chan(h, c, (cudaStream_t)stream);
        if (rc) return rc;
    }
    if (channel <= 0) h->d = h->descs[0];
    return LBVE_OK;
}

int lbve_step(lbve_t* h, int64_t n_steps, void* stream) {
    if (!h || n_steps < 0) return LBVE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (h->tangent) return h->Q == 9 ? tangent_step<9>(h, n_steps, s) : tangent_step<19>(h, n_steps, s);
    const int hk = h->model == LBVE_MODEL_INLM ? 3
                   : h->hist_formf ? (h->hist_s16 ? 6 : h->hist_dbl ? 5 : 4)
                   : h->hist_s16 ? 2 : (h->hist_dbl ? 1 : 0);
    if (h->Q == 9) return h->pop_dbl ? step_dispatch<9, double>(h, hk, n_steps, s) : step_dispatch<9, float>(h, hk, n_steps, s);
    return h->pop_dbl ? step_dispatch<19, double>(h, hk, n_steps, s) : step_dispatch<19, float>(h, hk, n_steps, s);
}

int lbve_get_time(const lbve_t* h, int64_t* t) {
    if (!h || !t) return LBVE_EINVAL;
    *t = h->t_host;
    return LBVE_OK;
}

int lbve_fields_count(const lbve_t* h, uint32_t mask, size_t* count) {
    if (!h || !count || (mask & ~31u)) return LBVE_EINVAL;
    *count = fields_count(h, mask);
    return LBVE_OK;
}

int lbve_set_probes(lbve_t* h, int32_t n_probes, const int64_t* nodes, int32_t every, int64_t capacity) {
    if (!h || n_probes < 0 || n_probes > 65536) return LBVE_EINVAL;
    if (h->tangent || h->rec_K) return LBVE_ENOSUPPORT;
    if (n_probes > 0) {
        if (!nodes || every < 1 || capacity < 1) return LBVE_EINVAL;
        for (int i = 0; i < n_probes; ++i)
            if (nodes[i] < 0 || nodes[i] >= h->N) return LBVE_EINVAL;
        const long long rec = 1 + (long long)n_probes * (1 + h->D + h->NS);
        if (capacity > (1ll << 40) / (rec * (long long)sizeof(double))) return LBVE_EINVAL;   // 8 TiB: nonsense
    }
    // the step graphs launch the recorder with the old buffers: let them finish, then re-capture
    LBVE_CUDA(cudaDeviceSynchronize());
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    void* old[] = {h->probe_nodes, h->probe_rec, h->probe_cnt};
    const size_t old_bytes = h->probe_cap > 0 ? sizeof(long long) * (h->probe_n + 1) +
                                                    sizeof(double) * (size_t)h->probe_cap *
                                                        (1 + (size_t)h->probe_n * (1 + h->D + h->NS))
                                              : 0;
    for (void* p : old) dev_free(h, p);
    h->bytes -= old_bytes;
    h->probe_nodes = nullptr;
    h->probe_rec = nullptr;
    h->probe_cnt = nullptr;
    h->probe_n = 0;
    h->probe_cap = 0;
    if (n_probes == 0) return LBVE_OK;
    const size_t rec = 1 + (size_t)n_probes * (1 + h->D + h->NS);
    const size_t bytes_before = h->bytes;
    int rc;
    if ((rc = alloc(h, (void**)&h->probe_nodes, sizeof(long long) * n_probes)) ||
        (rc = alloc(h, (void**)&h->probe_rec, sizeof(double) * rec * (size_t)capacity)) ||
        (rc = alloc(h, (void**)&h->probe_cnt, sizeof(long long)))) {
        for (void* p : {(void*)h->probe_nodes, (void*)h->probe_rec, (void*)h->probe_cnt}) dev_free(h, p);
        h->bytes = bytes_before;
        h->probe_nodes = nullptr;
        h->probe_rec = nullptr;
        h->probe_cnt = nullptr;
        return rc;
    }
    std::vector<long long> nn(nodes, nodes + n_probes);
    LBVE_CUDA(cudaMemcpy(h->probe_nodes, nn.data(), sizeof(long long) * n_probes, cudaMemcpyHostToDevice));
    LBVE_CUDA(cudaMemset(h->probe_cnt, 0, sizeof(long long)));
    h->probe_n = n_probes;
    h->probe_every = every;
    h->probe_cap = capacity;
    return LBVE_OK;
}

int lbve_probe_read(lbve_t* h, double* dst_host, int64_t* n_stored, int64_t* n_total, void* stream) {
    if (!h || !dst_host || !n_stored || !n_total) return LBVE_EINVAL;
    if (h->probe_n == 0) return LBVE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    long long cnt = 0;
    LBVE_CUDA(cudaMemcpyAsync(&cnt, h->probe_cnt, sizeof cnt, cudaMemcpyDeviceToHost, s));
    LBVE_CUDA(cudaStreamSynchronize(s));
    const long long k = cnt < h->probe_cap ? cnt : h->probe_cap;
    const size_t rec = 1 + (size_t)h->probe_n * (1 + h->D + h->NS);
    if (k > 0) {
        LBVE_CUDA(cudaMemcpyAsync(dst_host, h->probe_rec, sizeof(double) * rec * (size_t)k, cudaMemcpyDeviceToHost, s));
        LBVE_CUDA(cudaStreamSynchronize(s));
    }
    *n_stored = k;
    *n_total = cnt;
    return LBVE_OK;
}

int lbve_fields(lbve_t* h, uint32_t mask, double* dst, int32_t dst_is_device, void* stream) {
    if (!h || !dst || (mask & ~31u)) return LBVE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t cnt = fields_count(h, mask);
    if (h->tangent) {
        if (dst_is_device) return tangent_gather(h, mask, -1, dst, s);
        double* tmp = nullptr;
        LBVE_CUDA(cudaMallocAsync(&tmp, sizeof(double) * (cnt > 0 ? cnt : 1), s));
        int rc = tangent_gather(h, mask, -1, tmp, s);
        if (rc == LBVE_OK) {
            cudaError_t e = cudaMemcpyAsync(dst, tmp, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) rc = cuda_fail(e, "tangent fields");
        }
        cudaFreeAsync(tmp, s);
        return rc;
    }
    if (dst_is_device) return fields_impl(h, mask, dst, h->flag, s);
    if (h->stage_n < cnt) {
        dev_free(h, h->stage);
        h->stage = nullptr;
        h->stage_n = 0;
        int rc = dev_alloc(h, (void**)&h->stage, sizeof(double) * (cnt > 0 ? cnt : 1));
        if (rc) return rc;
        h->stage_n = cnt;
    }
    LBVE_CUDA(cudaMemsetAsync(h->flag, 0, sizeof(int), s));
    int rc = fields_impl(h, mask, h->stage, h->flag, s);
    if (rc) return rc;
    int flag = 0;
    LBVE_CUDA(cudaMemcpyAsync(dst, h->stage, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s));
    LBVE_CUDA(cudaMemcpyAsync(&flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    LBVE_CUDA(cudaStreamSynchronize(s));
    return flag ? LBVE_ENONFINITE : LBVE_OK;
}

int lbve_fields_ex(lbve_t* h, int32_t channel, uint32_t mask, void* dst, int32_t dst_is_device, int32_t dst_dtype,
                   void* stream) {
    if (!h || !dst || (mask & ~31u)) return LBVE_EINVAL;
    if (channel < -1 || channel >= h->nchan) return LBVE_EINVAL;
    if (dst_dtype != LBVE_F64 && dst_dtype != LBVE_F32) return LBVE_EINVAL;
    if (h->tangent) return LBVE_ENOSUPPORT;
    cudaStream_t s = (cudaStream_t)stream;
    const long long n0 = channel < 0 ? 0 : h->chan_host[channel].off;
    const int cnt = channel < 0 ? h->N : h->descs[channel].nx * h->descs[channel].ny * h->descs[channel].nz;
    const size_t vals = h->N > 0 ? fields_count(h, mask) / (size_t)h->N * (size_t)cnt : 0;
    const size_t esz = dst_dtype == LBVE_F64 ? sizeof(double) : sizeof(float);
    auto run = [&](void* d, int* flag) {
        return dst_dtype == LBVE_F64 ? fields_range_impl<double>(h, mask, n0, cnt, (double*)d, flag, s)
                                     : fields_range_impl<float>(h, mask, n0, cnt, (float*)d, flag, s);
    };
    if (dst_is_device) return run(dst, h->flag);
    const size_t need = (vals * esz + sizeof(double) - 1) / sizeof(double);   // staging, in doubles
    if (h->stage_n < need) {
        dev_free(h, h->stage);
        h->stage = nullptr;
        h->stage_n = 0;
        int rc = dev_alloc(h, (void**)&h->stage, sizeof(double) * (need > 0 ? need : 1));
        if (rc) return rc;
        h->stage_n = need;
    }
    LBVE_CUDA(cudaMemsetAsync(h->flag, 0, sizeof(int), s));
    int rc = run(h->stage, h->flag);
    if (rc) return rc;
    int flag = 0;
    LBVE_CUDA(cudaMemcpyAsync(dst, h->stage, vals * esz, cudaMemcpyDeviceToHost, s));
    LBVE_CUDA(cudaMemcpyAsync(&flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    LBVE_CUDA(cudaStreamSynchronize(s));
    return flag ? LBVE_ENONFINITE : LBVE_OK;
}

int lbve_history_apply(lbve_t* h, const double* kappa_dev, double* sigma_dev, void* stream) {
    if (!h || !kappa_dev || !sigma_dev) return LBVE_EINVAL;
    if (h->tangent) return LBVE_ENOSUPPORT;
    cudaStream_t s = (cudaStream_t)stream;
    k_advance_t<<<1, 1, 0, s>>>(h->t_dev);
    LBVE_CUDA(cudaGetLastError());
    int rc;
    const Geom g = geom_of(h);
    const int grid = (h->N + 255) / 256;
    if (h->model == LBVE_MODEL_INLM) {   // no history: the stress of Eq. (inlM) in the collision's arithmetic
        if (h->D == 2) {
            if (h->pop_dbl) k_commit<2, Instant<double>><<<grid, 256, 0, s>>>(Instant<double>{1, 4}, kappa_dev, (double*)h->sigma, (double*)h->kappa, sigma_dev, h->t_dev, g);
            else k_commit<2, Instant<float>><<<grid, 256, 0, s>>>(Instant<float>{1, 4}, kappa_dev, (double*)h->sigma, (double*)h->kappa, sigma_dev, h->t_dev, g);
        } else {
            if (h->pop_dbl) k_commit<3, Instant<double>><<<grid, 256, 0, s>>>(Instant<double>{1, 4}, kappa_dev, (double*)h->sigma, (double*)h->kappa, sigma_dev, h->t_dev, g);
            else k_commit<3, Instant<float>><<<grid, 256, 0, s>>>(Instant<float>{1, 4}, kappa_dev, (double*)h->sigma, (double*)h->kappa, sigma_dev, h->t_dev, g);
        }
    } else if (h->hist_formf) {
        const double* kin = kappa_dev;
        double* sf = (double*)h->sigma;
        double* kf = (double*)h->kappa;
        if (h->D == 2) {
            if (h->hist_s16) {
                if ((rc = launch_sweep_f16<2>(h, s))) return rc;
                k_commit<2, CommitF16><<<grid, 256, 0, s>>>(commit_f16(h), kin, sf, kf, sigma_dev, h->t_dev, g);
            } else if (h->hist_dbl) {
                if ((rc = launch_sweep_f<2, double>(h, s))) return rc;
                k_commit<2, CommitF<double>><<<grid, 256, 0, s>>>(commit_f<double>(h), kin, sf, kf, sigma_dev, h->t_dev, g);
            } else {
                if ((rc = launch_sweep_f<2, float>(h, s))) return rc;
                k_commit<2, CommitF<float>><<<grid, 256, 0, s>>>(commit_f<float>(h), kin, sf, kf, sigma_dev, h->t_dev, g);
            }
        } else {
            if (h->hist_s16) {
                if ((rc = launch_sweep_f16<3>(h, s))) return rc;
                k_commit<3, CommitF16><<<grid, 256, 0, s>>>(commit_f16(h), kin, sf, kf, sigma_dev, h->t_dev, g);
            } else if (h->hist_dbl) {
                if ((rc = launch_sweep_f<3, double>(h, s))) return rc;
                k_commit<3, CommitF<double>><<<grid, 256, 0, s>>>(commit_f<double>(h), kin, sf, kf, sigma_dev, h->t_dev, g);
            } else {
                if ((rc = launch_sweep_f<3, float>(h, s))) return rc;
                k_commit<3, CommitF<float>><<<grid, 256, 0, s>>>(commit_f<float>(h), kin, sf, kf, sigma_dev, h->t_dev, g);
            }
        }
    } else if (h->hist_s16) {
        if (h->D == 2) {
            if ((rc = launch_sweep_s16<2>(h, s))) return rc;
            k_commit<2, CommitS16><<<grid, 256, 0, s>>>(commit_s16(h), kappa_dev, (double*)h->sigma, (double*)h->kappa,
                                                        sigma_dev, h->t_dev, g);
        } else {
            if ((rc = launch_sweep_s16<3>(h, s))) return rc;
            k_commit<3, CommitS16><<<grid, 256, 0, s>>>(commit_s16(h), kappa_dev, (double*)h->sigma, (double*)h->kappa,
                                                        sigma_dev, h->t_dev, g);
        }
    } else if (h->D == 2) {
        if (h->hist_dbl) {
            if ((rc = launch_sweep<2, double>(h, s))) return rc;
            k_commit<2, CommitArgs<double>><<<grid, 256, 0, s>>>(commit_args<double>(h), kappa_dev, (double*)h->sigma,
                                                     (double*)h->kappa, sigma_dev, h->t_dev, g);
        } else {
            if ((rc = launch_sweep<2, float>(h, s))) return rc;
            k_commit<2, CommitArgs<float>><<<grid, 256, 0, s>>>(commit_args<float>(h), kappa_dev, (double*)h->sigma,
                                                    (double*)h->kappa, sigma_dev, h->t_dev, g);
        }
    } else {
        if (h->hist_dbl) {
            if ((rc = launch_sweep<3, double>(h, s))) return rc;
            k_commit<3, CommitArgs<double>><<<grid, 256, 0, s>>>(commit_args<double>(h), kappa_dev, (double*)h->sigma,
                                                     (double*)h->kappa, sigma_dev, h->t_dev, g);
        } else {
            if ((rc = launch_sweep<3, float>(h, s))) return rc;
            k_commit<3, CommitArgs<float>><<<grid, 256, 0, s>>>(commit_args<float>(h), kappa_dev, (double*)h->sigma,
                                                    (double*)h->kappa, sigma_dev, h->t_dev, g);
        }
    }
    LBVE_CUDA(cudaGetLastError());
    h->t_host += 1;
    return LBVE_OK;
}

int lbve_mass(lbve_t* h, double* sum_n, double* sum_drho, void* stream) {
    if (!h || !sum_n || !sum_drho) return LBVE_EINVAL;
    if (h->tangent) return LBVE_ENOSUPPORT;
    cudaStream_t s = (cudaStream_t)stream;
    return h->pop_dbl ? mass_impl<double>(h, sum_n, sum_drho, s) : mass_impl<float>(h, sum_n, sum_drho, s);
}

int lbve_schedule(int32_t C, int32_t B, int64_t t, int64_t* tp_out, double* w_out, int32_t* n_out) {
    if (C < 4 || B < 1 || B > LBVE_MAXB || t < 0 || !tp_out || !w_out || !n_out) return LBVE_EINVAL;
    // the same per-slot roles the history kernel evaluates, plus the point created at step t
    BlockStep bs[LBVE_MAXB];
    sched_step(B, C, (long long)t, bs);
    std::vector<std::pair<long long, double>> pts;
    pts.reserve((size_t)B * C);
    pts.emplace_back(0, 0.5);
    for (int bb = 0; bb < B; ++bb)
        for (int j = 0; j < C; ++j) {
            int age, part;
            const float w = sched_slot_role(bs, C, bb, j, &age, &part);
            if (w != 0.0f) pts.emplace_back(age, (double)w);
        }
    std::sort(pts.begin(), pts.end());
    for (size_t k = 0; k < pts.size(); ++k) {
        tp_out[k] = t - pts[k].first;
        w_out[k] = pts[k].second;
    }
    *n_out = (int32_t)pts.size();
    return LBVE_OK;
}

namespace {
// The buffers that make up the state of a handle, in checkpoint order (populations of the current
// parity only; u_raw, the sweep partials and the staging are recomputed or scratch).
struct StateBuf { void* p; size_t bytes; };
std::vector<StateBuf> state_buffers(lbve* h) {
    const long long Np = h->Npad;
    const int DD = h->D * h->D;
    const size_t fe = h->tangent ? sizeof(Dual) : sizeof(double);
    const size_t hist_elem = h->tangent ? sizeof(Dual) : (h->hist_s16 ? 2 : h->hesz);
    const int kplanes = h->hist_formf ? h->NS : DD;
    const bool f16 = h->hist_s16 && h->hist_formf;
    std::vector<StateBuf> v = {
        {h->pops[h->cur], h->pesz * h->Q * Np}, {h->u, fe * h->D * Np}, {h->rho, fe * Np},
        {h->sigma, fe * h->NS * Np}, {h->kappa, fe * DD * Np}, {h->tr_prev, fe * Np},
        {h->X, f16 ? (size_t)h->L * Np * (h->D == 2 ? 16 : 32) : hist_elem * (size_t)h->L * DD * Np},
        {h->K, f16 ? 0 : hist_elem * (size_t)h->L * kplanes * Np},
        {h->t_dev, sizeof(long long)}};
    if (h->hist_s16 && !h->hist_formf) {
        v.push_back({h->Qe, (size_t)h->L * Np});
        v.push_back({h->Ke, (size_t)h->L * Np});
        if (h->Rm) v.push_back({h->Rm, sizeof(float) * DD * Np});
    }
    if (h->gam_node) {
        v.push_back({h->gam_node, sizeof(double) * Np});
        v.push_back({h->gam_pt, sizeof(double) * (size_t)h->L * Np});
    }
    if (!h->tangent) v.push_back({h->chan_dev, sizeof(Chan) * h->nchan});
    std::vector<StateBuf> nz;   // buffers a model does not use (no history) have no bytes
    for (const StateBuf& b : v)
        if (b.p && b.bytes) nz.push_back(b);
    return nz;
}
constexpr uint64_t kCkptMagic = 0x4c42564543503031ull;   // "LBVECP01"
struct CkptHeader { uint64_t magic, total, nbuf, config; int64_t t_host; };

// Fingerprint (FNV-1a) of what must match between a checkpoint image and the handle it is restored into.
uint64_t config_fingerprint(const lbve* h) {
    uint64_t x = 1469598103934665603ull;
    auto mix = [&](long long v) {
        for (int i = 0; i < 8; ++i) { x ^= (uint64_t)((v >> (8 * i)) & 0xff); x *= 1099511628211ull; }
    };
    mix(h->tangent); mix(h->nchan); mix(h->N); mix(h->L);
    for (const lbve_channel_desc& d : h->descs) {
        mix(d.lattice); mix(d.nx); mix(d.ny); mix(d.nz); mix(d.wall_z); mix(d.hist_C); mix(d.hist_B);
        mix(d.hist_storage); mix(d.pop_precision); mix(d.trace_coupling); mix(d.model); mix(d.x_boundary);
        mix(d.hist_form);
    }
    return x;
}
}  // namespace

int lbve_checkpoint_size(lbve_t* h, size_t* bytes) {
    if (!h || !bytes) return LBVE_EINVAL;
    size_t t = sizeof(CkptHeader);
    for (const StateBuf& b : state_buffers(h)) t += (b.bytes + 255) / 256 * 256;
    *bytes = t;
    return LBVE_OK;
}

int lbve_checkpoint_save(lbve_t* h, void* dst, int32_t dst_is_device, void* stream) {
    if (!h || !dst) return LBVE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    size_t total = 0;
    lbve_checkpoint_size(h, &total);
    const std::vector<StateBuf> bufs = state_buffers(h);
    CkptHeader hd{kCkptMagic, total, bufs.size(), config_fingerprint(h), h->t_host};
    char* d = (char*)dst;
    const cudaMemcpyKind k = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    LBVE_CUDA(cudaMemcpyAsync(d, &hd, sizeof hd, dst_is_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, s));
    size_t off = sizeof(CkptHeader);
    for (const StateBuf& b : bufs) {
        LBVE_CUDA(cudaMemcpyAsync(d + off, b.p, b.bytes, k, s));
        off += (b.bytes + 255) / 256 * 256;
    }
    LBVE_CUDA(cudaStreamSynchronize(s));
    return LBVE_OK;
}

int lbve_checkpoint_restore(lbve_t* h, const void* src, int32_t src_is_device, void* stream) {
    if (!h || !src) return LBVE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    CkptHeader hd;
    LBVE_CUDA(cudaMemcpyAsync(&hd, src, sizeof hd, src_is_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, s));
    LBVE_CUDA(cudaStreamSynchronize(s));
    size_t total = 0;
    lbve_checkpoint_size(h, &total);
    std::vector<StateBuf> bufs = state_buffers(h);
    if (hd.magic != kCkptMagic || hd.total != total || hd.nbuf != bufs.size() || hd.config != config_fingerprint(h))
        return LBVE_EINVAL;
    h->cur = 0;                          // the populations are restored into buffer 0
    bufs = state_buffers(h);
    const char* c = (const char*)src;
    const cudaMemcpyKind k = src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    size_t off = sizeof(CkptHeader);
    for (const StateBuf& b : bufs) {
        LBVE_CUDA(cudaMemcpyAsync(b.p, c + off, b.bytes, k, s));
        off += (b.bytes + 255) / 256 * 256;
    }
    LBVE_CUDA(cudaStreamSynchronize(s));
    h->t_host = hd.t_host;
    if (!h->tangent) {   // the host copy of the channel table follows the restored device table
        LBVE_CUDA(cudaMemcpy(h->chan_host.data(), h->chan_dev, sizeof(Chan) * h->nchan, cudaMemcpyDeviceToHost));
        for (int ch = 0; ch < h->nchan; ++ch) {
            const Chan& cc = h->chan_host[ch];
            lbve_channel_desc& d = h->descs[ch];
            d.G_inf = cc.G_inf;
            d.tau = 1.0 / cc.inv_tau;
            d.gamma_c = cc.inv_gc == 0.0 ? INFINITY : 1.0 / cc.inv_gc;
            for (int a = 0; a < 3; ++a) d.g[a] = cc.f[a] / d.rho0;
        }
        h->d = h->descs[0];
    }
    return LBVE_OK;
}

}  // extern "C"

namespace {

int record_checkpoint(lbve* h, cudaStream_t s) {
    size_t bytes = 0;
    lbve_checkpoint_size(h, &bytes);
    const size_t idx = (size_t)(h->t_host / h->rec_K);
    if (h->ckpts.size() <= idx) h->ckpts.resize(idx + 1, nullptr);
    if (!h->ckpts[idx]) {
        int rc = dev_alloc(h, &h->ckpts[idx], bytes);
        if (rc) return rc;
    }
    return lbve_checkpoint_save(h, h->ckpts[idx], 1, s);
}

AdjPar adj_par(const lbve* h) {
    const lbve_channel_desc& d = h->descs[0];
    AdjPar p;
    p.G_inf = d.G_inf;
    p.tau = d.tau;
    p.gamma_c = d.gamma_c;
    p.inv_tau = 1.0 / d.tau;
    p.inv_gc = std::isinf(d.gamma_c) ? 0.0 : 1.0 / d.gamma_c;
    p.rho0 = d.rho0;
    p.tau_lb = d.tau_lb;
    for (int a = 0; a < 3; ++a) p.f[a] = d.rho0 * d.g[a];
    p.trace_full = d.trace_coupling == LBVE_TRACE_FULL;
    return p;
}

// Device allocation released at scope exit (the adjoint's work buffers).
struct DevBuf {
    lbve* h = nullptr;
    void* p = nullptr;
    int get(lbve* hh, size_t bytes) {
        h = hh;
        return dev_alloc(hh, &p, bytes);
    }
    ~DevBuf() { if (h) dev_free(h, p); }
};

// TP: population storage of the handle (and of the tape), TH: history storage (form P); the adjoint
// arithmetic and its buffers are double throughout.
template <int Q, typename TP, typename TH>
int backward_impl(lbve* h, const double* dL_du, const double* dL_ds, double* grad, cudaStream_t s) {
    constexpr int D = Lattice<Q>::D;
    constexpr int DD = D * D;
    constexpr int HK = sizeof(TH) == 8 ? 1 : 0;
    const int NS = h->NS;
    const long long Np = h->Npad;
    const int64_t T = h->t_host;
    const int K = h->rec_K;
    if (T < 1) return LBVE_ESTATE;
    const size_t hist_b = sizeof(TH) * (size_t)h->L * DD * Np;
    const size_t lhist_b = sizeof(TH) * (size_t)h->L * DD * Np;   // lambda of the history: the history's type
    const size_t pop_b = sizeof(TP) * h->Q * Np;
    const size_t lpop_b = sizeof(double) * h->Q * Np;
    // work buffers
    DevBuf lam_n, lamX, lamK, lam_trp, lam_kt, lam_th, seeds, tape, ur, cnt, fin, psig, plt, padj;
    // slot chunks of the split history kernels: about 32k (node, chunk) threads, at least 8 slots a chunk (the
    // per-node kernels add the chunks' partial sums in order, a chain as long as the chunk count)
    const int S = (int)std::max(1ll, std::min<long long>({64ll, (long long)std::max(1, h->L / 8),
                                                         (32768ll + h->N - 1) / h->N}));
    const size_t step_b = pop_b + 2 * hist_b + sizeof(double) * Np;   // pops, X, K, tr_prev
    size_t img = 0;
    lbve_checkpoint_size(h, &img);
    int rc;
    if ((rc = lam_n.get(h, 2 * lpop_b)) || (rc = lamX.get(h, lhist_b)) || (rc = lamK.get(h, lhist_b)) ||
        (rc = lam_trp.get(h, sizeof(double) * Np)) || (rc = lam_kt.get(h, sizeof(double) * DD * Np)) ||
        (rc = lam_th.get(h, sizeof(double) * 4 * Np)) || (rc = seeds.get(h, sizeof(double) * (D + NS) * Np)) ||
        (rc = tape.get(h, step_b * (size_t)K)) || (rc = ur.get(h, sizeof(double) * D * Np)) ||
        (rc = cnt.get(h, sizeof(long long))) || (rc = fin.get(h, img)) ||
        (rc = psig.get(h, sizeof(double) * (size_t)S * NS * Np)) || (rc = plt.get(h, sizeof(double) * DD * Np)) ||
        (rc = padj.get(h, sizeof(double) * (size_t)S * (DD + 2) * Np)))
        return rc;
    rc = lbve_checkpoint_save(h, fin.p, 1, s);   // the final state, restored at the end
    if (rc) return rc;
    LBVE_CUDA(cudaMemsetAsync(lam_n.p, 0, 2 * lpop_b, s));
    LBVE_CUDA(cudaMemsetAsync(lamX.p, 0, lhist_b, s));
    LBVE_CUDA(cudaMemsetAsync(lamK.p, 0, lhist_b, s));
    LBVE_CUDA(cudaMemsetAsync(lam_trp.p, 0, sizeof(double) * Np, s));
    LBVE_CUDA(cudaMemsetAsync(lam_th.p, 0, sizeof(double) * 4 * Np, s));
    LBVE_CUDA(cudaMemsetAsync(seeds.p, 0, sizeof(double) * (D + NS) * Np, s));
    double* seed_u = (double*)seeds.p;
    double* seed_s = seed_u + D * Np;
    for (int c = 0; c < D; ++c)
        LBVE_CUDA(cudaMemcpyAsync(seed_u + c * Np, dL_du + (size_t)c * h->N, sizeof(double) * h->N,
                                  cudaMemcpyHostToDevice, s));
    for (int c = 0; c < NS; ++c)
        LBVE_CUDA(cudaMemcpyAsync(seed_s + c * Np, dL_ds + (size_t)c * h->N, sizeof(double) * h->N,
                                  cudaMemcpyHostToDevice, s));
    const Geom g = geom_of(h);
    const AdjPar p = adj_par(h);
    // The per-node adjoint kernels are FP64 chains, and an SM's FP64 pipe completes a warp instruction in
    // (active lanes / 2) cycles: with few nodes, blocks of fewer threads spread them over more SMs, each
    // warp instruction taking fewer cycles (tpb threads a block, enough blocks to cover the SMs).
    int dev = 0, sms = 1;
    LBVE_CUDA(cudaGetDevice(&dev));
    LBVE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int tpb = 1;
    while (tpb < 32 && (h->N + tpb - 1) / tpb > sms) tpb *= 2;
    const int gridn = (h->N + tpb - 1) / tpb;
    const size_t smem = sweep_smem_bytes(h->L);
    if (smem > 32 * 1024) {   // the split kernels also hold up to 11 KB of static shared memory (their chunk sums)
        LBVE_CUDA(cudaFuncSetAttribute(k_adj_sig<D, TP, TH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        LBVE_CUDA(cudaFuncSetAttribute(k_adj_hist<D, TP, TH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    int cpb = 1;   // chunks a block of the split kernels adds itself (a power of two <= 16, <= S)
    while (cpb * 2 <= std::min(16, S)) cpb *= 2;
    const int SG = (S + cpb - 1) / cpb;
    const int grid_chunks = (int)((long long)SG * (Np / (128 / cpb)));
    DevBuf t0buf;   // the first step of the segment being processed (read by the adjoint kernels)
    if ((rc = t0buf.get(h, sizeof(long long)))) return rc;
    long long* t0dev = (long long*)t0buf.p;
#define LBVE_SEG(call)                                        \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)
    // replay steps t0 .. t1-1 from the restored image, keeping each step's state on the tape
    auto replay = [&](int64_t t0, int64_t t1, cudaStream_t st) -> int {
        for (int64_t t = t0; t < t1; ++t) {
            char* slot = (char*)tape.p + step_b * (size_t)(t - t0);
            LBVE_SEG(cudaMemcpyAsync(slot, h->pops[h->cur], pop_b, cudaMemcpyDeviceToDevice, st));
            LBVE_SEG(cudaMemcpyAsync(slot + pop_b, h->X, hist_b, cudaMemcpyDeviceToDevice, st));
            LBVE_SEG(cudaMemcpyAsync(slot + pop_b + hist_b, h->K, hist_b, cudaMemcpyDeviceToDevice, st));
            LBVE_SEG(cudaMemcpyAsync(slot + pop_b + 2 * hist_b, h->tr_prev, sizeof(double) * Np,
                                     cudaMemcpyDeviceToDevice, st));
            const int r = one_step<Q, TP, HK, TP>(h, h->cur, st);
            if (r) return r;
            h->cur ^= 1;
            h->t_host += 1;
        }
        return LBVE_OK;
    };
    // the adjoint of steps t1-1 down to t0 (lambda buffers alternate from parity lam0)
    auto adjoint = [&](int64_t t0, int64_t t1, int lam0, cudaStream_t st) -> int {
        int cl = lam0;
        for (int64_t t = t1 - 1; t >= t0; --t) {
            const char* slot = (const char*)tape.p + step_b * (size_t)(t - t0);
            const TP* pops_t = (const TP*)slot;
            k_moments<Q, TP, double><<<(h->N + h->node_tpb - 1) / h->node_tpb, h->node_tpb, 0, st>>>(pops_t, (double*)ur.p, g, (long long*)cnt.p);
            LBVE_SEG(cudaGetLastError());
            AdjArgs<TP, TH> a;
            a.n = pops_t;
            a.X = (const TH*)(slot + pop_b);
            a.K = (const TH*)(slot + pop_b + hist_b);
            a.trp = (const double*)(slot + pop_b + 2 * hist_b);
            a.u_raw = (const double*)ur.p;
            a.lam_n1 = (const double*)lam_n.p + (size_t)cl * h->Q * Np;
            a.lam_n0 = (double*)lam_n.p + (size_t)(cl ^ 1) * h->Q * Np;
            a.lamX = (TH*)lamX.p;
            a.lamK = (TH*)lamK.p;
            a.lam_trp = (double*)lam_trp.p;
            a.lam_kt = (double*)lam_kt.p;
            a.lam_theta = (double*)lam_th.p;
            a.seed_u = t == T - 1 ? seed_u : nullptr;
            a.seed_s = t == T - 1 ? seed_s : nullptr;
            a.part_sig = (double*)psig.p;
            a.lt = (double*)plt.p;
            a.part_adj = (double*)padj.p;
            a.t_off = t - t0;
            a.t0 = t0dev;
            a.B = h->d.hist_B;
            a.C = h->d.hist_C;
            a.S = S;
            a.cpb = cpb;
            a.SG = SG;
            k_adj_sig<D, TP, TH><<<grid_chunks, 128, smem, st>>>(a, g, p);
            LBVE_SEG(cudaGetLastError());
            k_adj_node<Q, TP, TH><<<gridn, tpb, 0, st>>>(a, g, p);
            LBVE_SEG(cudaGetLastError());
            k_adj_hist<D, TP, TH><<<grid_chunks, 128, smem, st>>>(a, g, p);
            LBVE_SEG(cudaGetLastError());
            k_adj_fin<D, TP, TH><<<gridn, tpb, 0, st>>>(a, g, p);
            LBVE_SEG(cudaGetLastError());
            k_adj_fd<Q, TP><<<gridn, tpb, 0, st>>>(pops_t, (const double*)lam_kt.p, a.lam_n0, (double*)lam_th.p, g, p);
            LBVE_SEG(cudaGetLastError());
            cl ^= 1;
        }
        return LBVE_OK;
    };
#undef LBVE_SEG
    // A full segment (K steps, not containing the last step, whose adjoint takes the loss seeds) is the same
    // sequence of launches for every segment: it is captured once per parity of the lambda buffers and
    // replayed; the segment's first step is written to device memory before each replay.
    cudaGraphExec_t seg_graph[2] = {nullptr, nullptr};
    auto free_graphs = [&]() {
        for (cudaGraphExec_t& ge : seg_graph)
            if (ge) { cudaGraphExecDestroy(ge); ge = nullptr; }
    };
    if (!h->graph_stream) LBVE_CUDA(cudaStreamCreateWithFlags(&h->graph_stream, cudaStreamNonBlocking));
    const int rec = h->rec_K;
    h->rec_K = 0;   // the replay below must not record
    int cur_lam = 0;
    const int64_t nseg = (T + K - 1) / K;
    for (int64_t sg = nseg - 1; sg >= 0 && rc == LBVE_OK; --sg) {
        if ((size_t)sg >= h->ckpts.size() || !h->ckpts[sg]) { rc = LBVE_ESTATE; break; }
        if ((rc = lbve_checkpoint_restore(h, h->ckpts[sg], 1, s))) break;
        const int64_t t0 = sg * K, t1 = std::min<int64_t>(T, t0 + K);
        k_set_ll<<<1, 1, 0, s>>>(t0dev, (long long)t0);
        if (cudaGetLastError() != cudaSuccess) { rc = cuda_fail(cudaErrorLaunchFailure, "k_set_ll"); break; }
        const bool graphable = t1 - t0 == K && t1 < T && !h->profiling;
        if (!graphable) {
            if ((rc = replay(t0, t1, s)) || (rc = adjoint(t0, t1, cur_lam, s))) break;
        } else {
            if (!seg_graph[cur_lam]) {
                cudaGraph_t gr = nullptr;
                cudaError_t e = cudaStreamBeginCapture(h->graph_stream, cudaStreamCaptureModeThreadLocal);
                if (e != cudaSuccess) { rc = cuda_fail(e, "cudaStreamBeginCapture"); break; }
                int rc2 = replay(t0, t1, h->graph_stream);
                if (rc2 == LBVE_OK) rc2 = adjoint(t0, t1, cur_lam, h->graph_stream);
                e = cudaStreamEndCapture(h->graph_stream, &gr);
                if (rc2 == LBVE_OK && e == cudaSuccess) e = cudaGraphInstantiate(&seg_graph[cur_lam], gr, 0);
                if (gr) cudaGraphDestroy(gr);
                if (rc2) { rc = rc2; break; }
                if (e != cudaSuccess) { rc = cuda_fail(e, "segment graph"); seg_graph[cur_lam] = nullptr; break; }
            }
            cudaError_t e = cudaGraphLaunch(seg_graph[cur_lam], s);
            if (e != cudaSuccess) { rc = cuda_fail(e, "cudaGraphLaunch"); break; }
        }
        cur_lam ^= (int)((t1 - t0) & 1);
    }
    if (rc == LBVE_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e, "backward");
    }
    free_graphs();
    h->rec_K = rec;
    if (rc) return rc;
    // dL/dtheta = sum over nodes of the per-node parts
    double* red = h->red;
    double out[4];
    for (int k = 0; k < 4; ++k) {
        LBVE_CUDA(cudaMemsetAsync(red, 0, sizeof(double), s));
        k_sum<double><<<4 * 152, 256, 0, s>>>((const double*)lam_th.p + (size_t)k * Np, Np, 1, h->N, 1.0, red);
        LBVE_CUDA(cudaGetLastError());
        LBVE_CUDA(cudaMemcpyAsync(&out[k], red, sizeof(double), cudaMemcpyDeviceToHost, s));
        LBVE_CUDA(cudaStreamSynchronize(s));
    }
    for (int k = 0; k < 4; ++k) grad[k] = out[k];
    return lbve_checkpoint_restore(h, fin.p, 1, s);
}

}  // namespace

extern "C" {

int lbve_create_adjoint(const lbve_channel_desc* desc, const double* rho_init, int32_t checkpoint_every,
                        lbve_t** out) {
    if (!desc || !out || checkpoint_every < 1) return LBVE_EINVAL;
    if ((desc->pop_precision != LBVE_F64 && desc->pop_precision != LBVE_F32) ||
        (desc->hist_storage != LBVE_F64 && desc->hist_storage != LBVE_F32))
        return LBVE_ENOSUPPORT;
    if (desc->model != LBVE_MODEL_NLM || desc->x_boundary != LBVE_X_PERIODIC) return LBVE_ENOSUPPORT;
    if (desc->hist_form != LBVE_FORM_P) return LBVE_ENOSUPPORT;
    int rc = create_impl(desc, 1, rho_init, out);
    if (rc) return rc;
    (*out)->rec_K = checkpoint_every;
    return LBVE_OK;
}

int lbve_backward(lbve_t* h, const double* dL_du, const double* dL_dsigma, double grad_out[4], void* stream) {
    if (!h || !dL_du || !dL_dsigma || !grad_out) return LBVE_EINVAL;
    if (!h->rec_K) return LBVE_ESTATE;
    cudaStream_t s = (cudaStream_t)stream;
    const int combo = (h->pop_dbl ? 2 : 0) + (h->hist_dbl ? 1 : 0);
    if (h->Q == 9) {
        switch (combo) {
            case 0: return backward_impl<9, float, float>(h, dL_du, dL_dsigma, grad_out, s);
            case 1: return backward_impl<9, float, double>(h, dL_du, dL_dsigma, grad_out, s);
            case 2: return backward_impl<9, double, float>(h, dL_du, dL_dsigma, grad_out, s);
            default: return backward_impl<9, double, double>(h, dL_du, dL_dsigma, grad_out, s);
        }
    }
    switch (combo) {
        case 0: return backward_impl<19, float, float>(h, dL_du, dL_dsigma, grad_out, s);
        case 1: return backward_impl<19, float, double>(h, dL_du, dL_dsigma, grad_out, s);
        case 2: return backward_impl<19, double, float>(h, dL_du, dL_dsigma, grad_out, s);
        default: return backward_impl<19, double, double>(h, dL_du, dL_dsigma, grad_out, s);
    }
}

int lbve_create_tangent(const lbve_channel_desc* desc, const double* rho_init, lbve_t** out) {
    return create_tangent(desc, rho_init, out);
}

int lbve_tangent_fields(lbve_t* h, uint32_t mask, double* dst_host, void* stream) {
    if (!h || !dst_host || (mask & ~31u)) return LBVE_EINVAL;
    if (!h->tangent) return LBVE_ESTATE;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t cnt = fields_count(h, mask);
    double* tmp = nullptr;
    LBVE_CUDA(cudaMallocAsync(&tmp, sizeof(double) * (cnt > 0 ? cnt : 1) * NT, s));
    int rc = LBVE_OK;
    for (int k = 0; k < NT && rc == LBVE_OK; ++k) rc = tangent_gather(h, mask, k, tmp + (size_t)k * cnt, s);
    if (rc == LBVE_OK) {
        cudaError_t e = cudaMemcpyAsync(dst_host, tmp, sizeof(double) * cnt * NT, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e, "tangent fields");
    }
    cudaFreeAsync(tmp, s);
    return rc;
}

int lbve_memory_bytes(const lbve_t* h, size_t* bytes) {
    if (!h || !bytes) return LBVE_EINVAL;
    *bytes = h->bytes;
    return LBVE_OK;
}

int lbve_sweep_config(const lbve_t* h, int32_t* slot_chunks, int32_t* ctas, int32_t* cta_tasks) {
    if (!h || !slot_chunks || !ctas || !cta_tasks) return LBVE_EINVAL;
    *slot_chunks = h->S;
    *ctas = h->sweep_grid;
    *cta_tasks = h->sweep_cta;
    return LBVE_OK;
}

int lbve_set_sweep_config(lbve_t* h, int32_t slot_chunks, int32_t cta_tasks) {
    if (!h) return LBVE_EINVAL;
    if (h->L == 0 || h->tangent || h->rec_K || !h->part) return LBVE_ENOSUPPORT;
    const long long Smax = h->L >= 16 ? h->L / 8 : 1;
    if (slot_chunks < 1 || slot_chunks > Smax || cta_tasks < 0 || cta_tasks > 2) return LBVE_EINVAL;
    if (cta_tasks == 1 && (h->hist_s16 || h->hist_formf)) return LBVE_EINVAL;   // warp tasks only
    const bool f16 = h->hist_s16 && h->hist_formf;
    if (cta_tasks == 2) {   // balanced ranges (16-bit form F only): the chunk count follows from the grid
        if (!f16) return LBVE_EINVAL;
        const long long tiles16 = h->Npad / (32 * (h->D == 2 ? 4 : 2));
        slot_chunks = f16_bal_max_pieces(tiles16, h->sweep_grid_full * 8);
        if (slot_chunks > Smax) return LBVE_EINVAL;
    }
    LBVE_CUDA(cudaDeviceSynchronize());
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    if (slot_chunks > h->part_S) {
        const size_t old_bytes = h->hesz * (size_t)h->part_S * h->part_ns * h->Npad;
        dev_free(h, h->part);
        h->bytes -= old_bytes;
        h->part = nullptr;
        h->part_S = 0;
        int rc = alloc(h, &h->part, h->hesz * (size_t)slot_chunks * h->part_ns * h->Npad);
        if (rc) return rc;
        h->part_S = slot_chunks;
    }
    const int vn = h->hist_s16 ? (h->D == 2 ? 4 : 2) : (h->hist_dbl ? 2 : 4) / (h->D == 3 ? 2 : 1);   // both forms
    const long long tiles = h->Npad / (32 * vn);
    h->S = slot_chunks;
    h->sweep_cta = cta_tasks;
    h->sweep_grid = cta_tasks == 2 ? h->sweep_grid_full
                                   : (int)std::max(1ll, std::min((long long)h->sweep_grid_full,
                                                                 cta_tasks ? tiles * slot_chunks : (tiles * slot_chunks + 7) / 8));
    return LBVE_OK;
}

const char* lbve_strerror(int status) {
    switch (status) {
        case LBVE_OK: return "ok";
        case LBVE_EINVAL: return "invalid argument";
        case LBVE_ENOMEM: return "out of device memory";
        case LBVE_ECUDA: return "CUDA error";
        case LBVE_ENONFINITE: return "non-finite value in the state";
        case LBVE_ESTATE: return "call does not fit the handle's state";
        case LBVE_ENOSUPPORT: return "combination not supported by this library";
        case LBVE_ETOOBIG: return "request exceeds the fixed staging buffer of lbve_fields_host_fixed";
        default: return "unknown status";
    }
}

const char* lbve_last_cuda_error(void) { return g_cuda_err; }

int lbve_profile(lbve_t* h, int32_t enable) {
    if (!h) return LBVE_EINVAL;
    h->profiling = enable ? 1 : 0;
    h->ev_used = 0;
    h->ev_kind.clear();
    return LBVE_OK;
}

int lbve_profile_read(lbve_t* h, double ms_out[3], int64_t launches_out[3]) {
    if (!h || !ms_out || !launches_out) return LBVE_EINVAL;
    for (int k = 0; k < KIND_COUNT; ++k) { ms_out[k] = 0.0; launches_out[k] = 0; }
    if (h->ev_used > 0) LBVE_CUDA(cudaEventSynchronize(h->ev_pool[h->ev_used - 1]));
    for (size_t i = 0; i < h->ev_kind.size(); ++i) {
        float ms = 0.0f;
        LBVE_CUDA(cudaEventElapsedTime(&ms, h->ev_pool[2 * i], h->ev_pool[2 * i + 1]));
        ms_out[h->ev_kind[i]] += ms;
        launches_out[h->ev_kind[i]] += 1;
    }
    h->ev_used = 0;
    h->ev_kind.clear();
    return LBVE_OK;
}

}  // extern "C"

// =================================================================================================
// lbve_fields_host_fixed: the host-destination field copy without any device allocation.
// The staging lives in one fixed file-scope device array; its last 32 doubles (256 bytes) hold the
// non-finite flag.  In host code the array's name is only a host-side stand-in, so the device address is
// looked up once per device with cudaGetSymbolAddress and passed to the kernels.
// =================================================================================================
static __device__ __align__(256) double g_fixed_staging[LBVE_FIXED_STAGING_DOUBLES + 32];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_fixed_mu;
// Per device: the array's device address and the id of the CUDA context it was looked up in.  A context
// that has been torn down (cudaDeviceReset) and made again gets a new id, and the address is looked up
// again in the new context.
struct FixedSlot { unsigned long long ctx_id; double* ptr; };
FixedSlot g_fixed[kMaxDevices] = {};

// Id of the calling thread's current CUDA context (0 if there is none or the driver cannot say).  The two
// driver queries are resolved once through the runtime's entry-point lookup.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool resolved = false;
    if (!resolved) {
        resolved = true;
        cudaDriverEntryPointQueryResult q1, q2;
        void* f1 = nullptr;
        void* f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            get_current = (CtxGetCurrentFn)f1;
            get_id = (CtxGetIdFn)f2;
        }
        cudaGetLastError();   // a failed lookup leaves no sticky error behind
    }
    if (!get_current || !get_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the fixed staging array on the current device: looked up on the first call on a
// device, and again when the device's context has changed since (or its id cannot be read).
int fixed_staging_ptr(double** out) {
    int dev = -1;
    LBVE_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return LBVE_ENOSUPPORT;
    std::lock_guard<std::mutex> lock(g_fixed_mu);
    FixedSlot& slot = g_fixed[dev];
    unsigned long long id = current_context_id();
    if (!slot.ptr || id == 0 || slot.ctx_id != id) {
        double* p = nullptr;
        LBVE_CUDA(cudaGetSymbolAddress((void**)&p, g_fixed_staging));
        if (id == 0) id = current_context_id();   // the lookup makes the device's context current
        slot.ptr = p;
        slot.ctx_id = id;
    }
    *out = slot.ptr;
    return LBVE_OK;
}

}  // namespace

extern "C" int lbve_fields_host_fixed(lbve_t* h, uint32_t mask, double* dst_host, void* stream) {
    if (!h || !dst_host || (mask & ~31u)) return LBVE_EINVAL;
    if (h->tangent) return LBVE_ENOSUPPORT;
    const size_t cnt = fields_count(h, mask);
    if (cnt > (size_t)LBVE_FIXED_STAGING_DOUBLES) return LBVE_ETOOBIG;
    cudaStream_t s = (cudaStream_t)stream;
    double* stage = nullptr;
    int rc = fixed_staging_ptr(&stage);
    if (rc) return rc;
    int* flag = reinterpret_cast<int*>(stage + LBVE_FIXED_STAGING_DOUBLES);
    LBVE_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
    if ((rc = fields_impl(h, mask, stage, flag, s))) return rc;
    int flag_host = 0;
    LBVE_CUDA(cudaMemcpyAsync(dst_host, stage, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s));
    LBVE_CUDA(cudaMemcpyAsync(&flag_host, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    LBVE_CUDA(cudaStreamSynchronize(s));
    return flag_host ? LBVE_ENONFINITE : LBVE_OK;
}
