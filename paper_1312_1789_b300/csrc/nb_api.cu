// nb_api.cu -- host side of libnb: the C ABI declared in include/nb.h.
//
// Owns the device state, sequences the kernels of one block step on the
// context's stream, validates arguments on the host and turns the status word
// the kernels raise into NB_ERR_* codes at every synchronisation point.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "nb_internal.cuh"

using namespace nb;

namespace {

void* (*g_alloc)(size_t, void*) = nullptr;
void (*g_free)(void*, void*) = nullptr;
void* g_user = nullptr;
// per host thread, like errno: concurrent context-free calls keep their own message
thread_local char g_err[512] = "";

int set_err(nb_ctx* c, int code, const char* fmt, ...)
{
    char* dst = c ? c->err : g_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return code;
}

const char* code_name(int code)
{
    switch (code) {
    case NB_OK: return "ok";
    case NB_ERR_ARG: return "invalid argument";
    case NB_ERR_CUDA: return "CUDA error";
    case NB_ERR_NOT_SYNC: return "particles not synchronised";
    case NB_ERR_DT_UNDERFLOW: return "time step below dt_min";
    case NB_ERR_TIMEOUT: return "device wait timed out";
    case NB_ERR_NAN: return "non-finite value";
    case NB_ERR_NOMEM: return "out of device memory";
    default: return "unknown";
    }
}

#define NB_CUDA(c, call)                                                                                       \
    do {                                                                                                       \
        cudaError_t e_ = (call);                                                                               \
        if (e_ != cudaSuccess)                                                                                 \
            return set_err((c), NB_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                           __LINE__);                                                                          \
    } while (0)

#define NB_TRY(expr)                \
    do {                            \
        int r_ = (expr);            \
        if (r_ != NB_OK) return r_; \
    } while (0)

template <typename T>
int dalloc(nb_ctx* c, T** p, size_t count)
{
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 256;
    void* q = nullptr;
    if (c->alloc_fn) {
        q = c->alloc_fn(bytes, c->alloc_user);
        if (!q) return set_err(c, NB_ERR_NOMEM, "allocator returned NULL for %zu bytes", bytes);
    } else {
        cudaError_t e = cudaMalloc(&q, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_err(c, NB_ERR_NOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
        }
    }
    *p = static_cast<T*>(q);
    return NB_OK;
}

void dfree(nb_ctx* c, void* p)
{
    if (!p) return;
    if (c->free_fn) c->free_fn(p, c->alloc_user);
    else cudaFree(p);
}

bool finite_all(const double* a, size_t n)
{
    for (size_t k = 0; k < n; ++k)
        if (!std::isfinite(a[k])) return false;
    return true;
}

bool is_pow2(double x)
{
    if (!(x > 0.0) || !std::isfinite(x)) return false;
    int e;
    return std::frexp(x, &e) == 0.5;
}

// ------------------------------------------------------------- profiling
cudaEvent_t prof_event(nb_ctx* c)
{
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Fold completed event pairs into the per-phase totals (stream synchronised).
void prof_fold(nb_ctx* c)
{
    for (auto& r : c->prof_recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) c->prof_ms[r.phase] += ms;
        else cudaGetLastError();
        c->ev_pool.push_back(r.a);
        c->ev_pool.push_back(r.b);
    }
    c->prof_recs.clear();
}

// Run one launcher (nk kernels) as phase `phase`, counting and, when profiling
// is on, bracketing it with events on the context's stream.
// NVTX range of a scope (a no-op unless a profiler is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

const char* const PHASE_RANGE[NB_NPHASES] = {"nb:sched", "nb:predict", "nb:force",
                                             "nb:reduce", "nb:correct", "nb:other"};

template <typename F>
cudaError_t timed(nb_ctx* c, int phase, int nk, F&& launch)
{
    c->n_launch += nk;
    NvtxRange range(PHASE_RANGE[phase]);
    if (!c->prof_on) return launch();
    cudaEvent_t a = prof_event(c), b = prof_event(c);
    if (a) cudaEventRecord(a, c->stream);
    const cudaError_t e = launch();
    if (b) cudaEventRecord(b, c->stream);
    if (a && b) c->prof_recs.push_back({a, b, phase});
    c->prof_n[phase] += nk;
    return e;
}

// Read the device scalars (waits for the stream) and turn a raised status into
// an error code; the status word is cleared for the next call.
// After a device error: clear the status word.
int clear_device_status(nb_ctx* c, cudaStream_t st)
{
    NB_CUDA(c, cudaMemsetAsync(&c->sc->status, 0, sizeof(int), st));
    NB_CUDA(c, cudaStreamSynchronize(st));
    return NB_OK;
}

int sync_scalars(nb_ctx* c)
{
    NB_CUDA(c, cudaMemcpyAsync(c->h_sc, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream));
    NB_CUDA(c, cudaStreamSynchronize(c->stream));
    if (!c->prof_recs.empty()) prof_fold(c);
    const int st = c->h_sc->status;
    if (st != NB_OK) {
        NB_TRY(clear_device_status(c, c->stream));
        return set_err(c, st, "device kernel reported: %s", code_name(st));
    }
    return NB_OK;
}

// Launch shape of the force: FORCE_NT i-particles per CTA; the j range is
// split so that small active sets still fill every SM (j-split), capped by the
// partial-sum buffer.
// j tiles of later force launches: the nb_force range when `ranged` and a
// range is set, else the whole store.
void set_launch_tiles(nb_ctx* c, bool ranged)
{
    if (ranged && c->jr_end > 0) {
        c->lt0 = (int)(c->jr_begin / JT);
        c->ltn = (int)((c->jr_end + JT - 1) / JT) - c->lt0;
    } else {
        c->lt0 = 0;
        c->ltn = (int)(c->np / JT);
    }
}

void choose_shape(nb_ctx* c, int order, int64_t n_act, int* itiles, int* jsplit, int* ni_out)
{
    const int ntiles = c->ltn;
    const long long cap_splits = (long long)(c->partial_cap / ((size_t)ncomp(order) * (size_t)n_act));
    const int pi = (c->pred_prec >= 0 ? c->pred_prec : c->prec) == NB_MIXED ? 1 : 0;
    int ni, it, js;
    if (order == c->order && c->jsplit_force <= 0 && tuned_shape(c->tune[pi], c->tune_n[pi], n_act, &ni, &it, &js)) {
        // autotuned class shape
    } else {
        ni = force_ni(c, n_act);
        it = (int)((n_act + ni - 1) / ni);
        js = c->jsplit_force > 0
                 ? c->jsplit_force
                 : makespan_split(it, ntiles, shape_slots(c, order, ni, pi == 1), cap_splits);
    }
    if (js > ntiles) js = ntiles;
    if (js > cap_splits) js = (int)cap_splits;
    if (js < 1) js = 1;
    *ni_out = ni;
    *itiles = it;
    *jsplit = js;
}

// ranged: sum over the nb_force j range only (nb_set_jrange); the start-up
// and energy passes always sum over every particle.
int run_force(nb_ctx* c, int order, const int32_t* idx_dev, int64_t n_act, bool ranged = false)
{
    int it, js, ni;
    set_launch_tiles(c, ranged);
    choose_shape(c, order, n_act, &it, &js, &ni);
    NB_CUDA(c, timed(c, NB_PHASE_FORCE, 1, [&] { return launch_force(c, order, idx_dev, n_act, js, it, ni); }));
    if (js > 1)
        NB_CUDA(c, timed(c, NB_PHASE_REDUCE, 1, [&] { return launch_force_reduce(c, order, idx_dev, n_act, js); }));
    c->last_itiles = it;
    c->last_jsplit = js;
    c->last_threads = ni;
    c->F_order = order;
    c->F_n = n_act;
    return NB_OK;
}

// ------------------------------------------------- device-driven cycles
void destroy_graph(nb_ctx* c)
{
    if (c->graph_exec) {
        cudaGraphExecDestroy(c->graph_exec);
        c->graph_exec = nullptr;
    }
}

// Capture graph_cycles device-driven block cycles (scheduler with the
// predictor and the shape gate, persistent force, reduction, corrector) into
// one CUDA graph.
// Every kernel reads n_act / t_blk / the launch shape from the device
// scalars, so the graph replays with no host round trip.
int build_graph(nb_ctx* c)
{
    destroy_graph(c);
    int grid[2] = {0, 0};
    c->pred_prec = c->prec;
    NB_CUDA(c, launch_force_dyn(c, grid, true));
    // the split rule sees the same slot counts as in host-driven cycles, so
    // a block gets the same shape (and the same summation order) in both
    int slots[4];
    const int variants[4] = {4, 32, FORCE_NT, 2 * FORCE_NT};
    for (int k = 0; k < 4; ++k) slots[k] = shape_slots(c, c->order, variants[k], c->prec == NB_MIXED);
    if (!c->graph_stream) NB_CUDA(c, cudaStreamCreateWithFlags(&c->graph_stream, cudaStreamNonBlocking));
    cudaStream_t saved = c->stream;
    c->stream = c->graph_stream;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->graph_stream, cudaStreamCaptureModeThreadLocal);
    // every kernel of the cycle may be scheduled while its predecessor runs
    // (programmatic dependent launch; each waits for it before reading)
    c->pdl = 1;
    for (int r = 0; e == cudaSuccess && r < c->graph_cycles; ++r) {
        if ((e = launch_sched_predict(c, true, slots)) != cudaSuccess) break;
        if ((e = launch_force_dyn(c, grid, false)) != cudaSuccess) break;
        if ((e = launch_force_reduce_dyn(c)) != cudaSuccess) break;
        if ((e = launch_correct(c, nullptr, nullptr, c->sc)) != cudaSuccess) break;
    }
    c->pdl = 0;
    const cudaError_t e2 = cudaStreamEndCapture(c->graph_stream, &g);
    c->stream = saved;
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph_exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        destroy_graph(c);
        return set_err(c, NB_ERR_CUDA, "block-cycle graph capture failed: %s", cudaGetErrorString(e));
    }
    return NB_OK;
}

int step_until_graph(nb_ctx* c, double t_end, int64_t* n_blocks, int64_t* n_inter)
{
    if (!c->graph_exec) NB_TRY(build_graph(c));
    NB_CUDA(c, cudaStreamSynchronize(c->stream));
    DevScalars* h = c->h_sc;
    NB_CUDA(c, cudaMemcpy(h, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost));
    h->t_end = t_end;
    h->idle = 0;
    h->blocks = 0;
    h->inter = 0;
    NB_CUDA(c, cudaMemcpy(c->sc, h, sizeof(DevScalars), cudaMemcpyHostToDevice));
    // scheduler 2 (the second predicts and sets the launch shape), persistent
    // force (two kernels on the mixed path), reduction, corrector
    const long long per_cycle = 2 + (c->prec == NB_MIXED ? 2 : 1) + 1 + 1;
    for (;;) {
        NvtxRange range("nb:graph replay");
        NB_CUDA(c, cudaGraphLaunch(c->graph_exec, c->graph_stream));
        c->n_launch += per_cycle * c->graph_cycles;
        NB_CUDA(c, cudaMemcpyAsync(h, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->graph_stream));
        NB_CUDA(c, cudaStreamSynchronize(c->graph_stream));
        if (h->status != NB_OK) {
            const int st = h->status;
            NB_TRY(clear_device_status(c, c->graph_stream));
            return set_err(c, st, "device kernel reported: %s", code_name(st));
        }
        if (h->idle) break;
    }
    if (n_blocks) *n_blocks = h->blocks;
    if (n_inter) *n_inter = h->inter;
    c->have_pred = c->have_force = c->have_sched = 0;
    c->F_order = -1;
    return NB_OK;
}

int do_predict(nb_ctx* c, double t)
{
    // a j range with a scheduled block: the rank's records and the block's
    // active particles, which is all its force reads
    const bool ranged = c->jr_end > 0 && c->have_sched;
    if (ranged) {
        const int64_t r1 = std::min<int64_t>(c->np, (c->jr_end + JT - 1) / JT * JT);  // padding of the last tile
        NB_CUDA(c, timed(c, NB_PHASE_PREDICT, 1, [&] {
            return launch_predict_ranged(c, t, c->jr_begin, r1, c->act_idx, c->sched_n);
        }));
    } else {
        NB_CUDA(c, timed(c, NB_PHASE_PREDICT, 1, [&] { return launch_predict(c, t); }));
    }
    c->pred_ranged = ranged ? 1 : 0;
    c->pred_prec = c->prec;
    c->have_pred = 1;
    c->t_pred = t;
    return NB_OK;
}

}  // namespace

void nb::set_global_error(const char* msg) { snprintf(g_err, sizeof g_err, "%s", msg); }

extern "C" {

const char* nb_version(void) { return "libnb 0.1 (sm_103a)"; }

const char* nb_last_error(const nb_ctx* c) { return c ? c->err : g_err; }

int nb_set_allocator(void* (*alloc)(size_t, void*), void (*free_)(void*, void*), void* user)
{
    if ((alloc == nullptr) != (free_ == nullptr)) return set_err(nullptr, NB_ERR_ARG, "alloc and free must be set together");
    g_alloc = alloc;
    g_free = free_;
    g_user = user;
    return NB_OK;
}

void nb_destroy(nb_ctx* c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    void* ptrs[] = {c->m, c->eps2, c->x, c->v, c->d, c->t, c->dt, c->pot, c->jstore, c->act_idx, c->all_idx,
                    c->chunk_cnt, c->chunk_min, c->chunk_off, c->d_tune, c->stage, c->sc, c->nact_hist, c->red,
                    c->f_idx, c->partial, c->F};
    for (void* p : ptrs) dfree(c, p);
    if (c->h_sc) cudaFreeHost(c->h_sc);
    if (c->h_red) cudaFreeHost(c->h_red);
    for (auto& r : c->prof_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    destroy_graph(c);
    if (c->graph_stream) cudaStreamDestroy(c->graph_stream);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    delete c;
}

int nb_create(nb_ctx** out, int64_t n, int order, double eps)
{
    if (!out) return set_err(nullptr, NB_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > (1LL << 28)) return set_err(nullptr, NB_ERR_ARG, "n = %lld outside [1, 2^28]", (long long)n);
    if (!(order == 4 || order == 6 || order == 8)) return set_err(nullptr, NB_ERR_ARG, "order %d not 4, 6 or 8", order);
    if (!(eps >= 0.0) || !std::isfinite(eps)) return set_err(nullptr, NB_ERR_ARG, "eps must be finite and >= 0");
    nb_ctx* c = new (std::nothrow) nb_ctx();
    if (!c) return set_err(nullptr, NB_ERR_NOMEM, "host allocation failed");
    c->alloc_fn = g_alloc;
    c->free_fn = g_free;
    c->alloc_user = g_user;
    c->n = n;
    c->np = (n + JT - 1) / JT * JT;
    c->order = order;
    c->eps = eps;
    int rc = NB_OK;
    auto fail = [&](int code) {
        snprintf(g_err, sizeof g_err, "%s", c->err);
        nb_destroy(c);
        return code;
    };
    if (cudaGetDevice(&c->dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->dev) != cudaSuccess) {
        cudaGetLastError();
        set_err(c, NB_ERR_CUDA, "no usable CUDA device");
        return fail(NB_ERR_CUDA);
    }
    const size_t np = (size_t)c->np;
    const int nc = ncomp(order);
    const size_t rec = (size_t)(fp64_rw(order) > mixed_rw(order) ? fp64_rw(order) : mixed_rw(order)) * 16;
    int sched_per = 1;
    sched_layout(n, c->sm_count, &sched_per, &c->n_chunks);
    c->red_len = 4 * c->sm_count + 8;
    if (c->red_len < 2 * c->sm_count) c->red_len = 2 * c->sm_count;
    // j-split partial sums: room for the 16 splits the split rule allows a
    // full block (SPLIT_FLOOR; 1.5 GB at 2^20, order 6) up to 2^21 particles,
    // for a full block of any size, and for the many splits of small blocks
    const size_t span = (size_t)2 * 16 * c->sm_count * FORCE_NT;
    const size_t floor_rows = std::min((size_t)SPLIT_FLOOR * (size_t)n, (size_t)SPLIT_FLOOR << 21);
    c->partial_cap = (size_t)nc * std::max({floor_rows, (size_t)n, span});
    if ((rc = dalloc(c, &c->m, np)) || (rc = dalloc(c, &c->eps2, np)) || (rc = dalloc(c, &c->x, 3 * np)) ||
        (rc = dalloc(c, &c->v, 3 * np)) || (rc = dalloc(c, &c->d, 18 * np)) || (rc = dalloc(c, &c->t, np)) ||
        (rc = dalloc(c, &c->dt, np)) || (rc = dalloc(c, &c->pot, np)) ||
        (rc = dalloc(c, reinterpret_cast<unsigned char**>(&c->jstore), np * rec)) ||
        (rc = dalloc(c, &c->act_idx, (size_t)n)) || (rc = dalloc(c, &c->all_idx, (size_t)n)) ||
        (rc = dalloc(c, &c->f_idx, (size_t)n)) || (rc = dalloc(c, &c->chunk_cnt, (size_t)c->n_chunks)) ||
        (rc = dalloc(c, &c->chunk_min, (size_t)c->n_chunks)) || (rc = dalloc(c, &c->chunk_off, (size_t)c->n_chunks)) ||
        (rc = dalloc(c, &c->d_tune, (size_t)2 * TUNE_MAX)) ||
        (rc = dalloc(c, &c->sc, 1)) || (rc = dalloc(c, &c->nact_hist, (size_t)NB_NACT_CLASSES)) ||
        (rc = dalloc(c, &c->red, (size_t)c->red_len)) ||
        (rc = dalloc(c, &c->partial, c->partial_cap)) || (rc = dalloc(c, &c->F, (size_t)nc * (size_t)n)))
        return fail(rc);
    if (cudaMallocHost(&c->h_sc, sizeof(DevScalars)) != cudaSuccess ||
        cudaMallocHost(&c->h_red, 4 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        set_err(c, NB_ERR_NOMEM, "pinned host allocation failed");
        return fail(NB_ERR_NOMEM);
    }
    std::vector<int32_t> iota((size_t)n);
    for (int64_t k = 0; k < n; ++k) iota[(size_t)k] = (int32_t)k;
    if (cudaMemcpy(c->all_idx, iota.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(c->sc, 0, sizeof(DevScalars)) != cudaSuccess ||
        cudaMemset(c->nact_hist, 0, NB_NACT_CLASSES * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(c->m, 0, np * 8) != cudaSuccess ||
        cudaMemset(c->d_tune, 0, sizeof(TuneEntry) * 2 * TUNE_MAX) != cudaSuccess ||
        cudaMemset(c->x, 0, 3 * np * 8) != cudaSuccess || cudaMemset(c->v, 0, 3 * np * 8) != cudaSuccess ||
        cudaMemset(c->d, 0, 18 * np * 8) != cudaSuccess || cudaMemset(c->t, 0, np * 8) != cudaSuccess ||
        cudaMemset(c->dt, 0, np * 8) != cudaSuccess || cudaMemset(c->pot, 0, np * 8) != cudaSuccess) {
        cudaGetLastError();
        set_err(c, NB_ERR_CUDA, "device initialisation failed");
        return fail(NB_ERR_CUDA);
    }
    std::vector<double> e2(np, eps * eps);
    if (cudaMemcpy(c->eps2, e2.data(), np * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        set_err(c, NB_ERR_CUDA, "device initialisation failed");
        return fail(NB_ERR_CUDA);
    }
    *out = c;
    return NB_OK;
}

int nb_set_stream(nb_ctx* c, void* stream)
{
    if (!c) return NB_ERR_ARG;
    c->stream = static_cast<cudaStream_t>(stream);
    return NB_OK;
}

int nb_set_precision(nb_ctx* c, int mode)
{
    if (!c) return NB_ERR_ARG;
    if (mode != NB_FP64 && mode != NB_MIXED) return set_err(c, NB_ERR_ARG, "precision %d not NB_FP64 or NB_MIXED", mode);
    if (c->prec != mode) destroy_graph(c);
    c->prec = mode;
    return NB_OK;
}

int nb_set_softening(nb_ctx* c, const double* eps_i)
{
    if (!c) return NB_ERR_ARG;
    std::vector<double> e2((size_t)c->np, c->eps * c->eps);
    if (eps_i) {
        for (int64_t k = 0; k < c->n; ++k) {
            if (!(eps_i[k] >= 0.0) || !std::isfinite(eps_i[k]))
                return set_err(c, NB_ERR_ARG, "eps_i[%lld] must be finite and >= 0", (long long)k);
            e2[(size_t)k] = eps_i[k] * eps_i[k];
        }
    }
    NB_CUDA(c, cudaMemcpyAsync(c->eps2, e2.data(), e2.size() * 8, cudaMemcpyHostToDevice, c->stream));
    NB_CUDA(c, cudaStreamSynchronize(c->stream));
    destroy_graph(c);
    c->pair_eps = eps_i != nullptr;
    c->eps2_max = 0.0;
    for (int64_t k = 0; k < c->n; ++k) c->eps2_max = std::max(c->eps2_max, e2[(size_t)k]);
    c->have_pred = 0;
    return NB_OK;
}

int nb_set_params(nb_ctx* c, double eta, double eta_s, double dt_max, double dt_min)
{
    if (!c) return NB_ERR_ARG;
    if (!(eta > 0.0) || !std::isfinite(eta) || !(eta_s > 0.0) || !std::isfinite(eta_s))
        return set_err(c, NB_ERR_ARG, "eta and eta_s must be positive and finite");
    if (!is_pow2(dt_max)) return set_err(c, NB_ERR_ARG, "dt_max must be a power of two");
    if (!(dt_min > 0.0) || !(dt_min <= dt_max)) return set_err(c, NB_ERR_ARG, "need 0 < dt_min <= dt_max");
    destroy_graph(c);
    c->eta = eta;
    c->eta_s = eta_s;
    c->dt_max = dt_max;
    c->dt_min = dt_min;
    return NB_OK;
}

int nb_set_graph(nb_ctx* c, int cycles)
{
    if (!c) return NB_ERR_ARG;
    if (cycles < 0 || cycles > 4096) return set_err(c, NB_ERR_ARG, "cycles must be in [0, 4096]");
    if (cycles > 0 && c->jr_end > 0) return set_err(c, NB_ERR_ARG, "graph cycles need the whole j range");
    destroy_graph(c);
    c->graph_cycles = cycles;
    return NB_OK;
}

// Time one force launch shape (force + split reduction) on the all-particle
// list prefix of length na: best of reps runs, milliseconds.
static int time_shape(nb_ctx* c, int64_t na, int ni, int js, int reps, cudaEvent_t e0, cudaEvent_t e1, float* best)
{
    const int it = (int)((na + ni - 1) / ni);
    *best = INFINITY;
    for (int r = -1; r < reps; ++r) {  // r = -1: untimed warm-up
        NB_CUDA(c, cudaEventRecord(e0, c->stream));
        NB_CUDA(c, launch_force(c, c->order, c->all_idx, na, js, it, ni));
        if (js > 1) NB_CUDA(c, launch_force_reduce(c, c->order, c->all_idx, na, js));
        NB_CUDA(c, cudaEventRecord(e1, c->stream));
        NB_CUDA(c, cudaEventSynchronize(e1));
        float ms = 0.f;
        NB_CUDA(c, cudaEventElapsedTime(&ms, e0, e1));
        if (r >= 0 && ms < *best) *best = ms;
    }
    c->n_launch += (int64_t)(reps + 1) * (js > 1 ? 2 : 1);
    return sync_scalars(c);
}

// The same for a device-driven cycle: the shape written into the device
// scalars, the persistent force kernels and the split reduction, as a
// replayed cycle runs them (the active list must hold particles 0..na-1).
static int time_shape_dyn(nb_ctx* c, int64_t na, int ni, int js, int reps, cudaEvent_t e0, cudaEvent_t e1,
                          float* best)
{
    DevScalars* h = c->h_sc;
    NB_CUDA(c, cudaMemcpyAsync(h, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream));
    NB_CUDA(c, cudaStreamSynchronize(c->stream));
    h->idle = 0;
    h->n_act = na;
    h->ni = ni;
    h->itiles = (int)((na + ni - 1) / ni);
    h->jsplit = js;
    NB_CUDA(c, cudaMemcpyAsync(c->sc, h, sizeof(DevScalars), cudaMemcpyHostToDevice, c->stream));
    int grid[2] = {0, 0};
    NB_CUDA(c, launch_force_dyn(c, grid, true));
    *best = INFINITY;
    for (int r = -1; r < reps; ++r) {  // r = -1: untimed warm-up
        NB_CUDA(c, cudaEventRecord(e0, c->stream));
        NB_CUDA(c, launch_force_dyn(c, grid, false));
        NB_CUDA(c, launch_force_reduce_dyn(c));
        NB_CUDA(c, cudaEventRecord(e1, c->stream));
        NB_CUDA(c, cudaEventSynchronize(e1));
        float ms = 0.f;
        NB_CUDA(c, cudaEventElapsedTime(&ms, e0, e1));
        if (r >= 0 && ms < *best) *best = ms;
    }
    c->n_launch += (int64_t)(reps + 1) * (c->prec == NB_MIXED ? 3 : 2);
    return sync_scalars(c);
}

// A tuned shape must be this much faster than the analytic rule's to be kept.
constexpr float TUNE_MARGIN = 0.97f;

int nb_autotune(nb_ctx* c, int reps)
{
    if (!c) return NB_ERR_ARG;
    if (!c->have_particles) return set_err(c, NB_ERR_ARG, "nb_autotune before nb_set_particles");
    if (c->jr_end > 0) return set_err(c, NB_ERR_ARG, "nb_autotune needs the whole j range (nb_set_jrange(0, 0))");
    const int pi = c->prec == NB_MIXED ? 1 : 0;
    destroy_graph(c);
    c->tune_n[pi] = 0;
    if (reps > 0) {
        // the store every candidate reads: all particles predicted to the next block time
        double tb;
        int64_t na0;
        NB_TRY(nb_next_block(c, &tb, nullptr, &na0));
        NB_TRY(do_predict(c, tb));
        // graph mode set: time the persistent kernels its cycles run, on the
        // active list 0..n-1
        const bool dyn = c->graph_cycles > 0;
        if (dyn)
            NB_CUDA(c, cudaMemcpyAsync(c->act_idx, c->all_idx, (size_t)c->n * sizeof(int32_t),
                                       cudaMemcpyDeviceToDevice, c->stream));
        cudaEvent_t e0, e1;
        NB_CUDA(c, cudaEventCreate(&e0));
        NB_CUDA(c, cudaEventCreate(&e1));
        set_launch_tiles(c, false);
        const int ntiles = (int)(c->np / JT), nc = ncomp(c->order);
        const bool mixed = c->prec == NB_MIXED;
        int ncls = 0;
        while (ncls < TUNE_MAX && (1LL << ncls) <= c->n) ++ncls;
        // classes past this per-call time are left to the analytic rule
        const float budget_ms = 60.f;
        int rc = NB_OK;
        float prev_best = 0.f;
        for (int k = 0; k < ncls && rc == NB_OK; ++k) {
            TuneEntry& e = c->tune[pi][k];
            e = TuneEntry{0, 0, 0, 0.f};
            if (k > 0 && 2.f * prev_best > budget_ms) continue;
            const int64_t na = 1LL << k;
            const long long cap_splits = (long long)(c->partial_cap / ((size_t)nc * (size_t)na));
            int cand[4], nv = 0;
            if (na <= 64) cand[nv++] = 4;
            if (na <= 512) cand[nv++] = 32;
            if (!mixed || na <= 16384) cand[nv++] = FORCE_NT;
            if (mixed && na >= 64) cand[nv++] = 2 * FORCE_NT;
            // the analytic rule's own shape for this size (one of the candidates)
            const int r16_ni = force_ni(c, na);
            float best = INFINITY, r16_ms = INFINITY;
            for (int v = 0; v < nv && rc == NB_OK; ++v) {
                const int ni = cand[v];
                const int it = (int)((na + ni - 1) / ni);
                const int base = makespan_split(it, ntiles, shape_slots(c, c->order, ni, mixed), cap_splits);
                const long long js_rule = std::max(1LL, std::min<long long>(std::min<long long>(base, ntiles),
                                                                            cap_splits));
                const int mult[8][2] = {{1, 4}, {1, 2}, {1, 1}, {2, 1}, {4, 1}, {8, 1}, {16, 1}, {0, 1}};
                int tried[8], nt = 0;
                for (int q = 0; q < 8 && rc == NB_OK; ++q) {
                    long long js = mult[q][0] == 0 ? 1 : (long long)base * mult[q][0] / mult[q][1];
                    if (js > ntiles) js = ntiles;
                    if (js > cap_splits) js = cap_splits;
                    if (js < 1) js = 1;
                    bool dup = false;
                    for (int u = 0; u < nt; ++u) dup = dup || tried[u] == (int)js;
                    if (dup) continue;
                    tried[nt++] = (int)js;
                    float ms;
                    rc = dyn ? time_shape_dyn(c, na, ni, (int)js, reps, e0, e1, &ms)
                             : time_shape(c, na, ni, (int)js, reps, e0, e1, &ms);
                    if (rc == NB_OK && ni == r16_ni && js == js_rule) r16_ms = ms;
                    if (rc == NB_OK && ms < best) {
                        best = ms;
                        e = TuneEntry{ni, (int)js, it, ms};
                    }
                }
            }
            // a class keeps a tuned shape only if it beat the analytic rule's
            // by TUNE_MARGIN at the class's size: the rule adapts the split to
            // every size of the class, a tuned shape only scales it
            if (!(best < TUNE_MARGIN * r16_ms)) e = TuneEntry{0, 0, 0, r16_ms};
            prev_best = best;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        c->have_pred = c->have_force = c->have_sched = 0;
        c->F_order = -1;
        NB_TRY(rc);
        c->tune_n[pi] = ncls;
    }
    NB_CUDA(c, cudaMemcpy(c->d_tune + pi * TUNE_MAX, c->tune[pi], sizeof(TuneEntry) * TUNE_MAX,
                          cudaMemcpyHostToDevice));
    return NB_OK;
}

int nb_set_tuning(nb_ctx* c, int n_classes, const int32_t* ni, const int32_t* js)
{
    if (!c) return NB_ERR_ARG;
    if (n_classes < 0 || n_classes > TUNE_MAX || (n_classes > 0 && (!ni || !js)))
        return set_err(c, NB_ERR_ARG, "need 0 <= n_classes <= %d and both arrays", TUNE_MAX);
    const bool mixed = c->prec == NB_MIXED;
    for (int k = 0; k < n_classes; ++k) {
        const bool ok = ni[k] == 0 || ni[k] == 4 || ni[k] == 32 || ni[k] == FORCE_NT || (mixed && ni[k] == 2 * FORCE_NT);
        if (!ok || (ni[k] != 0 && js[k] < 1))
            return set_err(c, NB_ERR_ARG, "class %d: variant %d / split %d not valid here", k, ni[k], js[k]);
    }
    const int pi = mixed ? 1 : 0;
    destroy_graph(c);
    for (int k = 0; k < TUNE_MAX; ++k) {
        TuneEntry e{0, 0, 0, 0.f};
        if (k < n_classes && ni[k] > 0) e = TuneEntry{ni[k], js[k], (int)(((1LL << k) + ni[k] - 1) / ni[k]), 0.f};
        c->tune[pi][k] = e;
    }
    c->tune_n[pi] = n_classes;
    NB_CUDA(c, cudaMemcpy(c->d_tune + pi * TUNE_MAX, c->tune[pi], sizeof(TuneEntry) * TUNE_MAX,
                          cudaMemcpyHostToDevice));
    return NB_OK;
}

int nb_get_tuning(nb_ctx* c, int* n_classes, int32_t* ni, int32_t* js, double* ms)
{
    if (!c) return NB_ERR_ARG;
    const int pi = c->prec == NB_MIXED ? 1 : 0;
    if (n_classes) *n_classes = c->tune_n[pi];
    for (int k = 0; k < TUNE_MAX; ++k) {
        const TuneEntry& e = c->tune[pi][k];
        const bool on = k < c->tune_n[pi];
        if (ni) ni[k] = on ? e.ni : 0;
        if (js) js[k] = on ? e.js : 0;
        if (ms) ms[k] = on ? (double)e.ms : 0.0;
    }
    return NB_OK;
}

int nb_selftest_wait(nb_ctx* c, double seconds)
{
    if (!c) return NB_ERR_ARG;
    if (!(seconds > 0.0) || seconds > 5.0) return set_err(c, NB_ERR_ARG, "seconds must be in (0, 5]");
    int khz = 0;
    NB_CUDA(c, cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, c->dev));
    const long long cycles = (long long)(seconds * 1e3 * (double)(khz > 0 ? khz : 2000000));
    NB_CUDA(c, launch_wait_probe(c, cycles));
    c->n_launch += 1;
    NB_TRY(sync_scalars(c));
    return set_err(c, NB_ERR_CUDA, "the probe's wait completed although nothing arrives");
}

int nb_selftest_convert(nb_ctx* c, int64_t n, uint64_t seed, int64_t* mismatches)
{
    if (!c || !mismatches) return NB_ERR_ARG;
    if (n < 0) return set_err(c, NB_ERR_ARG, "n must be >= 0");
    unsigned long long* bad = nullptr;
    NB_CUDA(c, cudaMalloc(&bad, sizeof(unsigned long long)));
    unsigned long long h = 0;
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess) e = launch_convert_check(c, n, (unsigned long long)seed, bad);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, bad, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(bad);
    if (e != cudaSuccess) return set_err(c, NB_ERR_CUDA, "conversion self-check: %s", cudaGetErrorString(e));
    c->n_launch += 1;
    *mismatches = (int64_t)h;
    return NB_OK;
}

int nb_set_jsplit(nb_ctx* c, int js)
{
    if (!c) return NB_ERR_ARG;
    if (js < 0) return set_err(c, NB_ERR_ARG, "j_splits must be >= 0");
    if (js != c->jsplit_force) destroy_graph(c);
    c->jsplit_force = js;
    return NB_OK;
}

int nb_set_jrange(nb_ctx* c, int64_t j_begin, int64_t j_end)
{
    if (!c) return NB_ERR_ARG;
    if (j_begin == 0 && (j_end == 0 || j_end == c->n)) {
        if (c->pred_ranged) c->have_pred = 0;  // the store holds only the old share
        c->jr_begin = c->jr_end = 0;
        return NB_OK;
    }
    if (j_begin < 0 || j_end <= j_begin || j_end > c->n || j_begin % JT != 0 || (j_end % JT != 0 && j_end != c->n))
        return set_err(c, NB_ERR_ARG, "j range [%lld, %lld) must lie in [0, %lld) and start and end on multiples of %d "
                       "(or end at n)", (long long)j_begin, (long long)j_end, (long long)c->n, JT);
    if (c->graph_cycles > 0) return set_err(c, NB_ERR_ARG, "a j range cannot be combined with graph cycles");
    if (j_begin != c->jr_begin || j_end != c->jr_end) c->have_pred = 0;  // a new share: predict again
    c->jr_begin = j_begin;
    c->jr_end = j_end;
    return NB_OK;
}

int nb_copy_force(nb_ctx* c, double* dst, int64_t* ncomp_out, int64_t* n_act_out)
{
    if (!c || !dst) return NB_ERR_ARG;
    if (!c->have_force || c->F_order != c->order) return set_err(c, NB_ERR_ARG, "no force result held (call nb_force first)");
    const size_t cnt = (size_t)ncomp(c->order) * (size_t)c->F_n;
    NB_CUDA(c, cudaMemcpyAsync(dst, c->F, cnt * sizeof(double), cudaMemcpyDefault, c->stream));
    if (ncomp_out) *ncomp_out = ncomp(c->order);
    if (n_act_out) *n_act_out = c->F_n;
    return NB_OK;
}

int nb_reduce_force(nb_ctx* c, const double* parts, int n_parts)
{
    if (!c || !parts || n_parts < 1) return set_err(c, NB_ERR_ARG, "parts must be non-NULL and n_parts >= 1");
    if (!c->have_force || c->F_order != c->order)
        return set_err(c, NB_ERR_ARG, "nb_reduce_force needs a preceding nb_force");
    NB_CUDA(c, timed(c, NB_PHASE_REDUCE, 1, [&] { return launch_parts_reduce(c, c->order, parts, c->F_n, n_parts); }));
    return NB_OK;
}

int nb_get_launch(nb_ctx* c, int* it, int* js, int* nt)
{
    if (!c) return NB_ERR_ARG;
    if (it) *it = c->last_itiles;
    if (js) *js = c->last_jsplit;
    if (nt) *nt = c->last_threads;
    return NB_OK;
}

// Host [n][3] -> device [3][np]
static int upload_vec(nb_ctx* c, double* dst, const double* src)
{
    std::vector<double> tmp((size_t)3 * c->np, 0.0);
    for (int64_t i = 0; i < c->n; ++i)
        for (int k = 0; k < 3; ++k) tmp[(size_t)k * c->np + i] = src[3 * i + k];
    NB_CUDA(c, cudaMemcpyAsync(dst, tmp.data(), tmp.size() * 8, cudaMemcpyHostToDevice, c->stream));
    NB_CUDA(c, cudaStreamSynchronize(c->stream));
    return NB_OK;
}

int nb_set_particles(nb_ctx* c, const double* m, const double* x, const double* v)
{
    NvtxRange range("nb_set_particles");
    if (!c || !m || !x || !v) return c ? set_err(c, NB_ERR_ARG, "m, x and v are required") : NB_ERR_ARG;
    const size_t n = (size_t)c->n, np = (size_t)c->np;
    for (size_t k = 0; k < n; ++k)
        if (!(m[k] >= 0.0) || !std::isfinite(m[k])) return set_err(c, NB_ERR_ARG, "masses must be finite and >= 0");
    if (!finite_all(x, 3 * n) || !finite_all(v, 3 * n)) return set_err(c, NB_ERR_NAN, "non-finite position or velocity");
    std::vector<double> mm(np, 0.0);
    for (size_t k = 0; k < n; ++k) mm[k] = m[k];
    NB_CUDA(c, cudaMemcpyAsync(c->m, mm.data(), np * 8, cudaMemcpyHostToDevice, c->stream));
    NB_TRY(upload_vec(c, c->x, x));
    NB_TRY(upload_vec(c, c->v, v));
    NB_CUDA(c, cudaMemsetAsync(c->d, 0, 18 * np * 8, c->stream));
    NB_CUDA(c, cudaMemsetAsync(c->t, 0, np * 8, c->stream));
    NB_CUDA(c, cudaMemsetAsync(c->dt, 0, np * 8, c->stream));
    NB_CUDA(c, cudaMemsetAsync(c->pot, 0, np * 8, c->stream));
    NB_CUDA(c, cudaMemsetAsync(&c->sc->status, 0, sizeof(int), c->stream));
    c->have_particles = 1;
    c->have_force = 0;
    c->have_sched = 0;
    // Start-up: at t = 0 only positions and velocities are known.  The order-4
    // pass gives acc and jerk; with those as the predicted acc the order-6 pass
    // gives snap; with acc and jerk the order-8 pass gives crackle.
    for (int pass = 4; pass <= c->order; pass += 2) {
        NB_TRY(do_predict(c, 0.0));
        NB_TRY(run_force(c, pass, c->all_idx, c->n));
        NB_CUDA(c, timed(c, NB_PHASE_OTHER, 1, [&] { return launch_startup_store(c, pass); }));
    }
    NB_CUDA(c, timed(c, NB_PHASE_OTHER, 1, [&] { return launch_startup_dt(c); }));
    c->have_pred = 0;
    c->F_order = -1;
    return sync_scalars(c);
}

int nb_next_block(nb_ctx* c, double* t_blk, int32_t* idx_out, int64_t* n_act)
{
    if (!c) return NB_ERR_ARG;
    if (!c->have_particles) return set_err(c, NB_ERR_ARG, "nb_next_block before nb_set_particles");
    NB_CUDA(c, timed(c, NB_PHASE_SCHED, 2, [&] { return launch_sched(c); }));
    NB_TRY(sync_scalars(c));
    c->sched_t = c->h_sc->t_blk;
    c->sched_n = c->h_sc->n_act;
    c->have_sched = 1;
    if (t_blk) *t_blk = c->sched_t;
    if (n_act) *n_act = c->sched_n;
    if (idx_out) {
        NB_CUDA(c, cudaMemcpyAsync(idx_out, c->act_idx, sizeof(int32_t) * (size_t)c->sched_n, cudaMemcpyDeviceToHost,
                                   c->stream));
        NB_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return NB_OK;
}

int nb_predict(nb_ctx* c, double t)
{
    if (!c) return NB_ERR_ARG;
    if (!c->have_particles) return set_err(c, NB_ERR_ARG, "nb_predict before nb_set_particles");
    if (!std::isfinite(t)) return set_err(c, NB_ERR_ARG, "t must be finite");
    c->have_force = 0;
    return do_predict(c, t);
}

int nb_force(nb_ctx* c, const int32_t* idx, int64_t n_act)
{
    if (!c) return NB_ERR_ARG;
    if (!c->have_pred) return set_err(c, NB_ERR_ARG, "nb_force needs a preceding nb_predict");
    if (!idx) {
        if (!c->have_sched) return set_err(c, NB_ERR_ARG, "nb_force(NULL) needs a preceding nb_next_block");
        if (n_act <= 0) n_act = c->sched_n;
        if (n_act != c->sched_n)
            return set_err(c, NB_ERR_ARG, "n_act %lld differs from the scheduled %lld", (long long)n_act,
                           (long long)c->sched_n);
        NB_CUDA(c, cudaMemcpyAsync(c->f_idx, c->act_idx, sizeof(int32_t) * (size_t)n_act, cudaMemcpyDeviceToDevice,
                                   c->stream));
    } else {
        if (n_act < 1 || n_act > c->n) return set_err(c, NB_ERR_ARG, "n_act = %lld outside [1, n]", (long long)n_act);
        if (c->pred_ranged)
            return set_err(c, NB_ERR_ARG, "after a j-range prediction nb_force takes the scheduled list (NULL)");
        cudaPointerAttributes pa;
        bool on_device = false;
        if (cudaPointerGetAttributes(&pa, idx) == cudaSuccess)
            on_device = pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged;
        else
            cudaGetLastError();
        if (on_device) {
            NB_CUDA(c, cudaMemcpyAsync(c->f_idx, idx, sizeof(int32_t) * (size_t)n_act, cudaMemcpyDeviceToDevice,
                                       c->stream));
        } else {
            for (int64_t k = 0; k < n_act; ++k)
                if (idx[k] < 0 || idx[k] >= c->n)
                    return set_err(c, NB_ERR_ARG, "active_idx[%lld] = %d out of range", (long long)k, idx[k]);
            NB_CUDA(c, cudaMemcpyAsync(c->f_idx, idx, sizeof(int32_t) * (size_t)n_act, cudaMemcpyHostToDevice,
                                       c->stream));
        }
    }
    NB_TRY(run_force(c, c->order, c->f_idx, n_act, true));
    c->f_n = n_act;
    c->f_t = c->t_pred;
    c->f_order = c->order;
    c->have_force = 1;
    return NB_OK;
}

int nb_correct(nb_ctx* c)
{
    if (!c) return NB_ERR_ARG;
    if (!c->have_force || c->F_order != c->order)
        return set_err(c, NB_ERR_ARG, "nb_correct needs a preceding nb_force");
    NB_CUDA(c, timed(c, NB_PHASE_CORRECT, 1, [&] { return launch_correct(c); }));
    c->have_force = 0;
    c->have_pred = 0;
    c->have_sched = 0;
    c->F_order = -1;
    return NB_OK;
}

// Scheduler with the predictor fused into its second pass: leaves the
// scheduled block and the predicted store exactly as nb_next_block followed
// by nb_predict(t_blk) would.
static int next_block_predicted(nb_ctx* c, double* tb, int64_t* na)
{
    if (!c->have_particles) return set_err(c, NB_ERR_ARG, "block step before nb_set_particles");
    NB_CUDA(c, timed(c, NB_PHASE_SCHED, 2, [&] { return launch_sched_predict(c, false); }));
    NB_TRY(sync_scalars(c));
    c->sched_t = c->h_sc->t_blk;
    c->sched_n = c->h_sc->n_act;
    c->have_sched = 1;
    c->pred_prec = c->prec;
    c->have_pred = 1;
    c->pred_ranged = 0;  // the fused predictor covers every particle
    c->t_pred = c->sched_t;
    c->have_force = 0;
    *tb = c->sched_t;
    *na = c->sched_n;
    return NB_OK;
}

// A block step corrects with the force it computed, so it needs the whole
// j range; with a range set, step with nb_force, the exchange of the partial
// sums and nb_reduce_force.
static int need_whole_range(nb_ctx* c)
{
    if (c->jr_end > 0) return set_err(c, NB_ERR_ARG, "block steps need the whole j range (nb_set_jrange(0, 0))");
    return NB_OK;
}

int nb_block_step(nb_ctx* c, double* t_blk, int64_t* n_act)
{
    NvtxRange range("nb_block_step");
    if (!c) return NB_ERR_ARG;
    NB_TRY(need_whole_range(c));
    double tb = 0.0;
    int64_t na = 0;
    NB_TRY(next_block_predicted(c, &tb, &na));
    NB_TRY(nb_force(c, nullptr, na));
    NB_TRY(nb_correct(c));
    if (t_blk) *t_blk = tb;
    if (n_act) *n_act = na;
    return NB_OK;
}

int nb_step_until(nb_ctx* c, double t_end, int64_t* n_blocks, int64_t* n_inter)
{
    NvtxRange range("nb_step_until");
    if (!c) return NB_ERR_ARG;
    NB_TRY(need_whole_range(c));
    if (!std::isfinite(t_end)) return set_err(c, NB_ERR_ARG, "t_end must be finite");
    if (!c->have_particles) return set_err(c, NB_ERR_ARG, "nb_step_until before nb_set_particles");
    if (c->graph_cycles > 0) return step_until_graph(c, t_end, n_blocks, n_inter);
    int64_t nb = 0, ni = 0;
    for (;;) {
        double tb = 0.0;
        int64_t na = 0;
        NB_TRY(next_block_predicted(c, &tb, &na));
        if (tb > t_end) break;
        NB_TRY(nb_force(c, nullptr, na));
        NB_TRY(nb_correct(c));
        ++nb;
        ni += na * c->n;
    }
    if (n_blocks) *n_blocks = nb;
    if (n_inter) *n_inter = ni;
    return sync_scalars(c);
}

int nb_energy(nb_ctx* c, double* ekin, double* epot)
{
    NvtxRange range("nb_energy");
    if (!c) return NB_ERR_ARG;
    if (!c->have_particles) return set_err(c, NB_ERR_ARG, "nb_energy before nb_set_particles");
    const int g = energy_grid(c);
    NB_CUDA(c, timed(c, NB_PHASE_OTHER, 2, [&] { return launch_energy_sums(c, 0); }));
    NB_CUDA(c, cudaMemcpyAsync(c->h_red, c->red + 4 * g, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    NB_TRY(sync_scalars(c));
    const double tmin = c->h_red[2], tmax = c->h_red[3];
    if (tmin != tmax)
        return set_err(c, NB_ERR_NOT_SYNC, "particles at different times (%.17g .. %.17g)", tmin, tmax);
    // potential from the positions at the common time (prediction by 0)
    c->have_force = 0;
    NB_TRY(do_predict(c, tmin));
    NB_TRY(run_force(c, 0, c->all_idx, c->n));
    NB_CUDA(c, timed(c, NB_PHASE_OTHER, 2, [&] { return launch_energy_sums(c, 1); }));
    NB_CUDA(c, cudaMemcpyAsync(c->h_red, c->red + 4 * g, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    NB_TRY(sync_scalars(c));
    if (ekin) *ekin = c->h_red[0];
    if (epot) *epot = c->h_red[1];
    return NB_OK;
}

// Device staging buffer for the state in the caller's particle order.
static int ensure_stage(nb_ctx* c)
{
    if (!c->stage) NB_TRY(dalloc(c, &c->stage, (size_t)26 * (size_t)c->n));
    return NB_OK;
}

int nb_get_state(nb_ctx* c, double* x, double* v, double* d, double* t, double* dt)
{
    if (!c) return NB_ERR_ARG;
    NB_TRY(sync_scalars(c));
    NB_TRY(ensure_stage(c));
    const size_t n = (size_t)c->n;
    NB_CUDA(c, launch_state_out(c));
    const double* st = c->stage;
    if (x) NB_CUDA(c, cudaMemcpyAsync(x, st, 3 * n * 8, cudaMemcpyDeviceToHost, c->stream));
    if (v) NB_CUDA(c, cudaMemcpyAsync(v, st + 3 * n, 3 * n * 8, cudaMemcpyDeviceToHost, c->stream));
    if (d) NB_CUDA(c, cudaMemcpyAsync(d, st + 6 * n, 18 * n * 8, cudaMemcpyDeviceToHost, c->stream));
    if (t) NB_CUDA(c, cudaMemcpyAsync(t, st + 24 * n, n * 8, cudaMemcpyDeviceToHost, c->stream));
    if (dt) NB_CUDA(c, cudaMemcpyAsync(dt, st + 25 * n, n * 8, cudaMemcpyDeviceToHost, c->stream));
    NB_CUDA(c, cudaStreamSynchronize(c->stream));
    return NB_OK;
}

int nb_set_state(nb_ctx* c, const double* x, const double* v, const double* d, const double* t, const double* dt)
{
    if (!c) return NB_ERR_ARG;
    if (!x || !v || !d || !t || !dt) return set_err(c, NB_ERR_ARG, "x, v, d, t and dt are required");
    NB_TRY(sync_scalars(c));
    NB_TRY(ensure_stage(c));
    const size_t n = (size_t)c->n;
    double* st = c->stage;
    NB_CUDA(c, cudaMemcpyAsync(st, x, 3 * n * 8, cudaMemcpyHostToDevice, c->stream));
    NB_CUDA(c, cudaMemcpyAsync(st + 3 * n, v, 3 * n * 8, cudaMemcpyHostToDevice, c->stream));
    NB_CUDA(c, cudaMemcpyAsync(st + 6 * n, d, 18 * n * 8, cudaMemcpyHostToDevice, c->stream));
    NB_CUDA(c, cudaMemcpyAsync(st + 24 * n, t, n * 8, cudaMemcpyHostToDevice, c->stream));
    NB_CUDA(c, cudaMemcpyAsync(st + 25 * n, dt, n * 8, cudaMemcpyHostToDevice, c->stream));
    NB_CUDA(c, launch_state_in(c));
    c->n_launch += 2;
    const int st_code = sync_scalars(c);
    if (st_code == NB_ERR_NAN) return set_err(c, NB_ERR_NAN, "non-finite state");
    if (st_code == NB_ERR_ARG) return set_err(c, NB_ERR_ARG, "every dt must be > 0");
    NB_TRY(st_code);
    c->have_particles = 1;
    c->have_pred = c->have_force = c->have_sched = 0;
    c->F_order = -1;
    return NB_OK;
}

int nb_get_force(nb_ctx* c, double* acc, double* jerk, double* snap, double* crackle, double* pot)
{
    if (!c) return NB_ERR_ARG;
    if (c->F_order < 4) return set_err(c, NB_ERR_ARG, "no force result held (call nb_force first)");
    NB_TRY(sync_scalars(c));
    const int o = c->F_order, nc = ncomp(o);
    const size_t fn = (size_t)c->F_n;
    std::vector<double> tmp((size_t)nc * fn);
    NB_CUDA(c, cudaMemcpyAsync(tmp.data(), c->F, tmp.size() * 8, cudaMemcpyDeviceToHost, c->stream));
    NB_CUDA(c, cudaStreamSynchronize(c->stream));
    double* outs[4] = {acc, jerk, snap, crackle};
    for (int q = 0; q < 4; ++q) {
        if (!outs[q]) continue;
        for (size_t p = 0; p < fn; ++p)
            for (int k = 0; k < 3; ++k) outs[q][3 * p + k] = (q < o / 2) ? tmp[(size_t)(3 * q + k) * fn + p] : 0.0;
    }
    if (pot)
        for (size_t p = 0; p < fn; ++p) pot[p] = tmp[(size_t)pot_comp(o) * fn + p];
    return NB_OK;
}

int nb_get_pair_warps(nb_ctx* c, int64_t* n_warps)
{
    if (!c || !n_warps) return NB_ERR_ARG;
    unsigned long long v = 0;
    NB_CUDA(c, cudaMemcpyAsync(&v, &c->sc->pair_warps, sizeof v, cudaMemcpyDeviceToHost, c->stream));
    NB_CUDA(c, cudaMemsetAsync(&c->sc->pair_warps, 0, sizeof v, c->stream));
    NB_CUDA(c, cudaStreamSynchronize(c->stream));
    *n_warps = (int64_t)v;
    return NB_OK;
}

int nb_get_predicted(nb_ctx* c, double* xp, double* vp, double* ap, double* jp)
{
    if (!c) return NB_ERR_ARG;
    if (!c->have_pred) return set_err(c, NB_ERR_ARG, "no predicted store (call nb_predict first)");
    NB_TRY(sync_scalars(c));
    const size_t n = (size_t)c->n;
    const bool mixed = c->pred_prec == NB_MIXED;
    const int rw = mixed ? mixed_rw(c->order) : fp64_rw(c->order);
    std::vector<unsigned char> raw(n * rw * 16);
    NB_CUDA(c, cudaMemcpyAsync(raw.data(), c->jstore, raw.size(), cudaMemcpyDeviceToHost, c->stream));
    NB_CUDA(c, cudaStreamSynchronize(c->stream));
    for (size_t i = 0; i < n; ++i) {
        const unsigned char* r = raw.data() + i * rw * 16;
        if (mixed) {
            const float* f = reinterpret_cast<const float*>(r);
            for (int k = 0; k < 3; ++k) {
                if (xp) xp[3 * i + k] = (double)f[k] + (double)f[4 + k];
                if (vp) vp[3 * i + k] = f[8 + k];
                if (ap) ap[3 * i + k] = c->order >= 6 ? f[12 + k] : 0.0;
                if (jp) jp[3 * i + k] = c->order >= 8 ? f[16 + k] : 0.0;
            }
        } else {
            const double* q = reinterpret_cast<const double*>(r);
            for (int k = 0; k < 3; ++k) {
                if (xp) xp[3 * i + k] = q[k];
                if (vp) vp[3 * i + k] = q[4 + k];
                if (ap) ap[3 * i + k] = c->order >= 6 ? q[8 + k] : 0.0;
                if (jp) jp[3 * i + k] = c->order >= 8 ? q[12 + k] : 0.0;
            }
        }
    }
    return NB_OK;
}

int nb_set_block_step(nb_ctx* c, double dt)
{
    if (!c) return NB_ERR_ARG;
    if (!c->have_particles) return set_err(c, NB_ERR_ARG, "nb_set_block_step before nb_set_particles");
    if (!is_pow2(dt) || dt > c->dt_max) return set_err(c, NB_ERR_ARG, "dt must be a power of two <= dt_max");
    NB_CUDA(c, timed(c, NB_PHASE_OTHER, 1, [&] { return launch_set_dt(c, dt); }));
    c->have_sched = 0;
    return NB_OK;
}

int nb_set_noise_floor(nb_ctx* c, int prec, const double* eps)
{
    if (!c) return NB_ERR_ARG;
    if ((prec != NB_FP64 && prec != NB_MIXED) || !eps) return set_err(c, NB_ERR_ARG, "bad precision or NULL eps");
    for (int k = 0; k < 4; ++k)
        if (!(eps[k] >= 0.0) || !std::isfinite(eps[k])) return set_err(c, NB_ERR_ARG, "eps must be finite and >= 0");
    destroy_graph(c);
    for (int k = 0; k < 4; ++k) c->noise[prec].e[k] = eps[k];
    return NB_OK;
}

int nb_get_noise_floor(nb_ctx* c, int prec, double* eps)
{
    if (!c) return NB_ERR_ARG;
    if ((prec != NB_FP64 && prec != NB_MIXED) || !eps) return set_err(c, NB_ERR_ARG, "bad precision or NULL eps");
    for (int k = 0; k < 4; ++k) eps[k] = c->noise[prec].e[k];
    return NB_OK;
}

int nb_set_profiling(nb_ctx* c, int enable)
{
    if (!c) return NB_ERR_ARG;
    NB_CUDA(c, cudaStreamSynchronize(c->stream));
    prof_fold(c);
    for (int k = 0; k < NB_NPHASES; ++k) {
        c->prof_ms[k] = 0.0;
        c->prof_n[k] = 0;
    }
    c->prof_on = enable != 0;
    return NB_OK;
}

int nb_get_nact_histogram(nb_ctx* c, int64_t* counts, int reset)
{
    if (!c) return NB_ERR_ARG;
    unsigned long long h[NB_NACT_CLASSES];
    NB_CUDA(c, cudaMemcpyAsync(h, c->nact_hist, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    if (reset) NB_CUDA(c, cudaMemsetAsync(c->nact_hist, 0, sizeof h, c->stream));
    NB_CUDA(c, cudaStreamSynchronize(c->stream));
    if (counts)
        for (int k = 0; k < NB_NACT_CLASSES; ++k) counts[k] = (int64_t)h[k];
    return NB_OK;
}

int nb_get_profile(nb_ctx* c, double* ms, int64_t* launches, int64_t* total)
{
    if (!c) return NB_ERR_ARG;
    NB_CUDA(c, cudaStreamSynchronize(c->stream));
    prof_fold(c);
    for (int k = 0; k < NB_NPHASES; ++k) {
        if (ms) ms[k] = c->prof_ms[k];
        if (launches) launches[k] = c->prof_n[k];
    }
    if (total) *total = c->n_launch;
    return NB_OK;
}

}  // extern "C"
