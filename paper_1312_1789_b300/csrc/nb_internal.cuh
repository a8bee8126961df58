// nb_internal.cuh -- shared definitions of libnb's CUDA sources (sm_103a).
//
// Device state is structure-of-arrays FP64 in HBM, padded to np = a multiple of
// the force kernel's j tile:
//   m[np], eps2[np]                 mass and squared softening
//   x[3][np], v[3][np]              position, velocity   (component-major)
//   d[6][3][np]                     acc, jerk, snap, crackle, a^(4), a^(5)
//   t[np], dt[np]                   particle time and block step
//   pot[np]                         potential of the last force
// The predictor writes the j-particle store read by the force kernel, one
// fixed-size record per particle (see the record layouts below).
#pragma once

#include <cuda_runtime.h>
#include <cmath>
#include <stdint.h>

#include <vector>

#include "nb.h"

namespace nb {

// j tile of the force kernel: records staged per bulk copy.
constexpr int JT = 128;
// threads per force CTA; each holds 1 or 2 i-particles (IPT).
constexpr int FORCE_NT = 128;
// the mixed force uses two i-particles per thread from this active-set size on
constexpr int IPT2_MIN_NACT = 512;

// Launch variant of the mixed force, named by its i-particles per CTA:
//   256: two per thread (n_act >= IPT2_MIN_NACT);
//   128: one per thread (256 < n_act < IPT2_MIN_NACT);
//   32, 4: j-parallel -- 4 or 32 threads share an i-particle, each taking
//          every 4th / 32nd record of a j tile, so that a few active
//          particles still keep a CTA's threads busy (n_act <= 256: at most
//          eight i-tiles of 32; n_act <= 24: at most six of 4).
// The thresholds are where the autotuner's measurements switch variant on
// the 65k and the 2^20 stores.
__host__ __device__ inline int mixed_ni(long long n_act)
{
    if (n_act >= IPT2_MIN_NACT) return 2 * FORCE_NT;
    if (n_act > 256) return FORCE_NT;
    return n_act > 24 ? 32 : 4;
}

// The FP64 force has the one-per-thread and the two j-parallel variants,
// with the same thresholds.
__host__ __device__ inline int fp64_ni(long long n_act)
{
    const int ni = mixed_ni(n_act);
    return ni > FORCE_NT ? FORCE_NT : ni;
}
// stages of the force kernel's shared-memory ring.
constexpr int NSTAGE = 3;
// spin limit of a bounded mbarrier wait, in SM clock cycles (~2 s at 2 GHz).
constexpr long long WAIT_LIMIT_CYCLES = 4000000000LL;

// Record sizes in 16-byte words.
// Mixed record (float4 words), 48 / 64 / 80 bytes for orders 4 / 6 / 8:
//   w0 = (x_hi.xyz, m)   w1 = (x_lo.xyz, eps2)   w2 = (v.xyz, 0)
//   w3 = (a.xyz, 0)      [order >= 6]            w4 = (jerk.xyz, 0) [order 8]
// FP64 record (double2 words), 64 / 96 / 128 bytes:
//   w0 = (x.x, x.y)  w1 = (x.z, m)  w2 = (v.x, v.y)  w3 = (v.z, eps2)
//   w4 = (a.x, a.y)  w5 = (a.z, 0)  [order >= 6]
//   w6 = (j.x, j.y)  w7 = (j.z, 0)  [order 8]
__host__ __device__ constexpr int mixed_rw(int order) { return order == 4 ? 3 : order == 6 ? 4 : 5; }
__host__ __device__ constexpr int fp64_rw(int order) { return order == 4 ? 4 : order == 6 ? 6 : 8; }
// components of a force result: acc, jerk[, snap[, crackle]] x 3, then pot,
// then (orders >= 4) the acc magnitude scale B = sum_j m_j / R_ij^2, an upper
// bound of sum_j |A_ij| that sets the rounding level of the acc total.
__host__ __device__ constexpr int ncomp(int order) { return order == 0 ? 1 : 3 * (order / 2) + 2; }
__host__ __device__ constexpr int pot_comp(int order) { return order == 0 ? 0 : 3 * (order / 2); }

// j-split count of a force launch with the shortest makespan.  it i-tiles x s
// splits of equal work run in waves of `slots` CTAs and take
// ceil(it*s/slots)/s of the one-split time.  For w waves the best s is the
// largest with it*s <= w*slots, so only those candidates (in increasing s,
// clamped to s_max) are scored; a candidate replaces the running best only
// when its span is over 0.5% shorter.  s_max bounds s by the j tiles, the
// partial buffer (cap_splits) and about four waves' worth of splits, but
// allows 16 at any size: a large block split 16 ways ran faster than the
// wave count predicts (full blocks of 2^20, 2^18 and 2^16 particles 1.5-1.8 %
// faster than with the 1, 4 and 9 splits of a four-wave bound and 1 % ties;
// shorter j ranges per split keep the concurrent CTAs on fewer j tiles and
// even out the last wave).
// Integer arithmetic only: the host and the device-driven gate agree exactly.
constexpr long long SPLIT_FLOOR = 16;
__host__ __device__ inline int makespan_split(int it, int ntiles, int slots, long long cap_splits)
{
    if (it < 1) it = 1;
    if (slots < 1) slots = 1;
    long long s_max = 4LL * slots / it + 4;
    if (s_max < SPLIT_FLOOR) s_max = SPLIT_FLOOR;
    if (s_max > ntiles) s_max = ntiles;
    if (s_max > cap_splits) s_max = cap_splits;
    if (s_max <= 1) return 1;
    long long best_s = 1, best_w = (it + slots - 1) / slots;
    const long long w_last = ((long long)it * s_max + slots - 1) / slots;
    for (long long w = best_w; w <= w_last; ++w) {
        long long s = w * slots / it;
        if (s > s_max) s = s_max;
        if (s <= best_s) continue;
        const long long ws = ((long long)it * s + slots - 1) / slots;
        // ws / s < 0.995 * best_w / best_s
        if (1000 * ws * best_s < 995 * best_w * s) {
            best_s = s;
            best_w = ws;
        }
    }
    return (int)best_s;
}

// Autotuned launch shape of one active-set size class (nb_autotune): the
// variant ni and split count js measured best at the class's representative
// size, where the force took `it` i-tiles and `ms` milliseconds.
constexpr int TUNE_MAX = 32;
struct TuneEntry {
    int ni, js, it;
    float ms;
};

// Shape of an n_act block from the tuned table (ntab classes; false: no
// entry): class floor(log2(n_act)) (the last class serves larger sets), its
// variant, and the split count that keeps its number of CTAs it * js.
__host__ __device__ inline bool tuned_shape(const TuneEntry* tab, int ntab, long long n_act, int* ni, int* it,
                                            int* js)
{
    if (ntab <= 0 || n_act <= 0) return false;
    int k = 0;
    while (k + 1 < ntab && (n_act >> (k + 1)) > 0) ++k;
    const TuneEntry e = tab[k];
    if (e.ni <= 0) return false;
    *ni = e.ni;
    *it = (int)((n_act + e.ni - 1) / e.ni);
    const long long ctas = (long long)e.js * e.it;
    long long s = (ctas + *it / 2) / *it;
    *js = (int)(s < 1 ? 1 : s);
    return true;
}

// Scalars shared between the scheduler, the kernels and the host.
struct DevScalars {
    long long n_act;  // size of the active list
    double t_blk;     // block time
    int status;       // first error raised by a kernel (NB_OK if none)
    int idle;         // device-driven cycle: the block is past t_end, do nothing
    double t_end;     // device-driven cycle: stop time
    int itiles, jsplit, ni;        // device-driven cycle: force launch shape
    int n_items;                   // ensemble cycle: force work items
    long long blocks, inter;       // device-driven cycle: blocks (cycles) taken, interactions
    int stepped;                   // ensemble cycle: clusters stepped in the last cycle
    int next_item;                 // ensemble cycle: next force item to hand out
    unsigned long long pair_warps; // mixed force: warps that took the per-pair softening form
    // scheduler: the first pass's last CTA publishes the block time's order
    // key and the number of matches (sched_ticket counts the CTAs done)
    unsigned long long tb_key;
    int n_match;
    unsigned int sched_ticket;
};

// Threshold of the dominant-softening test.  A warp whose i-particles all
// have the system's largest eps^2 takes the pair value eps_i^2 without a
// per-pair max.  The test compares the float eps^2 of the j-store, which the
// predictor converts toward zero, so the threshold takes the same
// conversion: rounded to nearest it can lie above every stored value, and no
// warp would take the uniform path.
inline float eps2_threshold(double e2max)
{
    float f = (float)e2max;
    if (std::fabs((double)f) > std::fabs(e2max)) f = std::nextafter(f, 0.0f);
    return f;
}

// Launch-shape gate of a device-driven cycle, applied by the thread that
// publishes the cycle's t_blk and n_act: close the cycle when the block lies
// past t_end, otherwise pick the force launch shape exactly as the host rule
// does for a block of that size (the autotuned table if any, else the same
// variant rule, slot counts and makespan split; a forced split).  slots = the
// resident CTAs the split rule plans for with 4, 32, FORCE_NT and 2 FORCE_NT
// i-particles per CTA (shape_slots).
struct GateArgs {
    long long n;     // particles (interactions per active particle)
    long long cap;   // partial-sum buffer, doubles
    int ntiles;      // j tiles of the store
    int nc;          // force components
    int mixed;       // precision of the force
    int js_force;    // forced split (0: none)
    int4 slots;
    const TuneEntry* tab;
    int ntab;
};

__device__ __forceinline__ void cycle_gate_apply(DevScalars* sc, double tb, long long na, const GateArgs& g)
{
    if (!(tb <= sc->t_end) || na <= 0) {
        sc->idle = 1;
        return;
    }
    sc->idle = 0;
    const long long cap_splits = g.cap / ((long long)g.nc * na);
    int ni, it, js;
    if (g.js_force > 0 || !tuned_shape(g.tab, g.ntab, na, &ni, &it, &js)) {
        ni = g.mixed ? mixed_ni(na) : fp64_ni(na);
        const int sl = ni == 4 ? g.slots.x : ni == 32 ? g.slots.y : ni == FORCE_NT ? g.slots.z : g.slots.w;
        it = (int)((na + ni - 1) / ni);
        js = g.js_force > 0 ? g.js_force : makespan_split(it, g.ntiles, sl, cap_splits);
    }
    sc->ni = ni;
    sc->itiles = it;
    if (js > g.ntiles) js = g.ntiles;
    if (js > cap_splits) js = (int)cap_splits;
    sc->jsplit = js < 1 ? 1 : js;
    sc->blocks += 1;
    sc->inter += na * g.n;
}

// Relative precision of the force components (acc, jerk, snap, crackle) that
// sets the noise floor of interpolated derivatives in the time-step criterion.
struct NoiseEps {
    double e[4];
};

__device__ __forceinline__ void raise_status(DevScalars* sc, int code)
{
    atomicCAS(&sc->status, NB_OK, code);
}

// ------------------------------------------- programmatic dependent launch
// The kernels of a block cycle start with pdl_wait() then pdl_release().
// Launched with programmatic stream serialization (launch_k, pdl = true), a
// kernel's CTAs may become resident while its predecessor in the stream still
// runs: pdl_wait() holds them until that grid has completed and its writes are
// visible, so nothing is read early.  pdl_release() lets the next kernel's
// CTAs be scheduled once every CTA of this grid has started.  Launched
// without the attribute, both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ------------------------------------------------------------ bulk copies
__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// One-dimensional TMA bulk copy global -> shared; completion is signalled on bar.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of bar to complete, giving up after WAIT_LIMIT_CYCLES.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  long long limit_cycles = WAIT_LIMIT_CYCLES)
{
    if (mbar_try_wait(bar, parity)) return true;
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit_cycles) return false;
    }
    return true;
}

// ------------------------------------------------------ double-single sums
// Error-free sum (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// (hi, lo) += x, compensated.
__device__ __forceinline__ void ds_add(float& hi, float& lo, float x)
{
    float s, e;
    two_sum(hi, x, s, e);
    hi = s;
    lo += e;
}

// (hi, lo) += (bh, bl), compensated (double-single sum).
__device__ __forceinline__ void ds_add_ds(float& hi, float& lo, float bh, float bl)
{
    float s, e;
    two_sum(hi, bh, s, e);
    e += lo + bl;
    hi = s + e;
    lo = e - (hi - s);
}

}  // namespace nb

// ------------------------------------------------------------ the context
struct nb_ctx {
    int dev = 0;
    int64_t n = 0;   // particles
    int64_t np = 0;  // padded to a multiple of nb::JT
    int order = 6;
    int prec = NB_MIXED;
    int pred_prec = -1;  // precision of the store written by the last predict
    double eps = 0.0;
    int pair_eps = 0;  // per-particle softening in use
    double eps2_max = 0.0;  // largest eps_i^2 (per-particle softening)
    double eta = 0.2, eta_s = 0.01, dt_max = 1.0 / 16, dt_min = 0x1p-40;
    // noise floors per precision [NB_FP64, NB_MIXED]: FP64 none (the plain
    // criterion); mixed from the measured error of the FP32 force chain
    nb::NoiseEps noise[2] = {{{0.0, 0.0, 0.0, 0.0}}, {{5e-7, 1e-6, 2e-6, 2e-5}}};
    cudaStream_t stream = nullptr;
    int jsplit_force = 0;
    int sm_count = 148;

    // state (FP64 SoA)
    double *m = nullptr, *eps2 = nullptr, *x = nullptr, *v = nullptr, *d = nullptr;
    double *t = nullptr, *dt = nullptr, *pot = nullptr;
    // j-particle store
    void* jstore = nullptr;
    // scheduler
    int32_t* act_idx = nullptr;   // [n] active list
    int32_t* all_idx = nullptr;   // [n] 0..n-1
    int32_t* chunk_cnt = nullptr; // scheduler: per-chunk match counts
    unsigned long long* chunk_min = nullptr;  // scheduler: per-chunk minima of t + dt (order keys)
    int32_t* chunk_off = nullptr; // scheduler: per-chunk offsets of the matches in the active list
    double* stage = nullptr;      // state I/O staging, 26 n doubles (allocated on first use)
    int n_chunks = 0;
    nb::DevScalars* sc = nullptr;
    unsigned long long* nact_hist = nullptr;  // [NB_NACT_CLASSES] corrector passes by floor(log2(n_act))
    nb::DevScalars* h_sc = nullptr;  // pinned
    double* red = nullptr;           // reduction scratch [red_len]
    int red_len = 0;
    double* h_red = nullptr;         // pinned, 4 doubles (energy sums, time range)
    // force
    int32_t* f_idx = nullptr;  // [n] list of the last force
    int64_t f_n = 0;
    double f_t = 0.0;
    int f_order = 0;
    double* partial = nullptr;  // j-split partial sums
    size_t partial_cap = 0;     // doubles
    double* F = nullptr;        // [ncomp][n] reduced force, list order
    // j range of nb_force (nb_set_jrange): particles [jr_begin, jr_end); jr_end = 0: all
    int64_t jr_begin = 0, jr_end = 0;
    // the last prediction covered the j range and the scheduled block only
    int pred_ranged = 0;
    // j tiles of the force launch in progress: [lt0, lt0 + ltn) (run_force sets them)
    int lt0 = 0, ltn = 0;
    int have_particles = 0, have_pred = 0, have_force = 0;
    double t_pred = 0.0;
    int F_order = -1;           // order of the result held in F (-1: none)
    int64_t F_n = 0;            // its list length
    int64_t sched_n = 0;        // result of the last scheduler pass
    double sched_t = 0.0;
    int have_sched = 0;
    int last_itiles = 0, last_jsplit = 0, last_threads = 0;
    // profiling: event pairs around launches, folded into totals at syncs
    struct ProfRec {
        cudaEvent_t a, b;
        int phase;
    };
    int prof_on = 0;
    std::vector<ProfRec> prof_recs;
    std::vector<cudaEvent_t> ev_pool;
    double prof_ms[NB_NPHASES] = {0};
    int64_t prof_n[NB_NPHASES] = {0};
    int64_t n_launch = 0;  // kernel launches since creation
    // autotuned launch shapes per precision (nb_autotune); device copy for the gate
    nb::TuneEntry tune[2][nb::TUNE_MAX] = {};
    int tune_n[2] = {0, 0};
    nb::TuneEntry* d_tune = nullptr;  // [2][TUNE_MAX]
    // device-driven cycles captured in a CUDA graph (nb_set_graph)
    int pdl = 0;  // launch the cycle's kernels with programmatic stream serialization
    int graph_cycles = 0;
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t graph_stream = nullptr;
    // allocator captured at creation
    void* (*alloc_fn)(size_t, void*) = nullptr;
    void (*free_fn)(void*, void*) = nullptr;
    void* alloc_user = nullptr;
    char err[512] = {0};
};

namespace nb {

// Launchers (k_*.cu); each returns cudaGetLastError() of its launches.
cudaError_t launch_sched(nb_ctx* c);
// Scheduler whose second pass also predicts every particle to the new block
// time (use_t_end: not past sc->t_end).
cudaError_t launch_sched_predict(nb_ctx* c, bool use_t_end, const int* shape_slots = nullptr);
// tpc, cid (ensembles): per-cluster prediction time and cluster of each slot; NULL for one system.
// dyn (device-driven cycle): take the time from dyn->t_blk and do nothing when dyn->idle.
cudaError_t launch_predict(nb_ctx* c, double t, const double* tpc = nullptr, const int32_t* cid = nullptr,
                           const DevScalars* dyn = nullptr);
// ni: the launch variant, i-particles per CTA (force_ni).  A one-split
// launch writes the result to c->F itself; otherwise launch_force_reduce
// adds the split partials into c->F.
cudaError_t launch_force(nb_ctx* c, int order, const int32_t* idx, int64_t n_act, int jsplit, int itiles, int ni);
cudaError_t launch_force_reduce(nb_ctx* c, int order, const int32_t* idx, int64_t n_act, int jsplit);
// c->F = the n_parts force results parts[n_parts][ncomp][n_act] added in part
// order (no sign change: each part is already a finished result).
cudaError_t launch_parts_reduce(nb_ctx* c, int order, const double* parts, int64_t n_act, int n_parts);
// Prediction of the records [r0, r1) and of the listed particles outside
// them (nl entries of a device list): a rank's j share and the block's active set.
cudaError_t launch_predict_ranged(nb_ctx* c, double t, int64_t r0, int64_t r1, const int32_t* list, int64_t nl);
// Self-check of the corrector's cvt conversions against the integer forms
// (nb_selftest_convert): *bad (device) += mismatches over n seeded inputs.
cudaError_t launch_convert_check(nb_ctx* c, int64_t n, unsigned long long seed, unsigned long long* bad);
// Corrector of the last force (dyn: of the block in the device scalars).
cudaError_t launch_correct(nb_ctx* c, const double* tfc = nullptr, const int32_t* cid = nullptr,
                           const DevScalars* dyn = nullptr);
// Device-driven block cycle (CUDA-graph capturable): shape gate, persistent
// force over device-chosen items, split reduction; all read n_act / t_blk on
// the device.
// shape_slots[4]: SMs x occupancy of the per-launch kernels with 4, 32, 128, 256 i-particles per CTA
cudaError_t launch_force_dyn(nb_ctx* c, int* grid /*[2]*/, bool query_only);
cudaError_t launch_force_reduce_dyn(nb_ctx* c);
cudaError_t launch_wait_probe(nb_ctx* c, long long limit_cycles);
cudaError_t launch_startup_store(nb_ctx* c, int order);
cudaError_t launch_startup_dt(nb_ctx* c);
cudaError_t launch_energy_sums(nb_ctx* c, int with_pot);
cudaError_t launch_set_dt(nb_ctx* c, double dt);
// State I/O through c->stage: validate and scatter into the state (nothing
// written if any value is invalid), or gather the state into it.
cudaError_t launch_state_in(nb_ctx* c);
cudaError_t launch_state_out(nb_ctx* c);
int force_occupancy(nb_ctx* c, int order, int ni);
int shape_slots(nb_ctx* c, int order, int ni, bool mixed);
int force_ni(const nb_ctx* c, int64_t n_act);
void sched_layout(int64_t n, int sm_count, int* per, int* nch);
int energy_grid(const nb_ctx* c);
// Message returned by nb_last_error(NULL) (calls made without a context).
void set_global_error(const char* msg);


// Launch kern<<<grid, block, smem, st>>>(args...), with programmatic stream
// serialization when pdl is set (the kernel must start with pdl_wait()).
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool pdl,
                     Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}
}  // namespace nb
