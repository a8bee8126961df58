// nb_batch.cu -- ensembles of independent clusters advanced together.
//
// Many small systems (clusters) are integrated side by side: every cycle
// advances each unfinished cluster by one of its own hierarchical blocks
// (abstract: individual block time-steps; each cluster has its own block
// time).  One launch per kernel serves all clusters: the force kernel runs
// over a table of (cluster, i-tile, j-split) items whose j range is the
// cluster's own particles, so a cycle costs the same handful of launches for
// 256 clusters as for one.
//
// Layout: the clusters are concatenated cluster-major, each padded to whole j
// tiles (JT records).  Padding slots have m = 0, eps2 = 1 and t = +inf: the
// scheduler never activates them and the force kernel sees exact zeros.
// cid[slot] is the slot's cluster, -1 for padding.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "force_kernels.cuh"

using namespace nb;

namespace {

struct BatchItem {
    int list_off;  // first position in the active list
    int count;     // i-particles of this item (<= ni)
    int jt0;       // first j tile (global)
    int nt;        // j tiles
    int split;     // row of the partial sums
    int ni;        // launch variant: 4, 32, FORCE_NT or (mixed) 2 FORCE_NT i-particles per CTA
    int pad[2];
};

}  // namespace

struct nb_batch {
    nb_ctx* c = nullptr;  // the padded concatenation
    int K = 0;
    std::vector<int64_t> nk, off, pk, roff;  // real sizes, slot offsets, padded sizes, offsets in the real list
    int64_t n_real = 0;
    int32_t* cid = nullptr;       // [np]
    int32_t* real_idx = nullptr;  // [n_real] the real slots, ascending
    int64_t* d_off = nullptr;     // [K]
    int64_t* d_nk = nullptr;      // [K]
    double* tblk = nullptr;       // [K] block time of each cluster (+inf: idle)
    unsigned long long* kmin = nullptr;  // [K] its first-pass key (all ones between cycles)
    int32_t* kstart = nullptr;    // [K] first position of the cluster in the active list
    int32_t* kcount = nullptr;    // [K] active particles of the cluster
    int32_t* ksplit = nullptr;    // [K] j-splits of the cluster this cycle
    int32_t* chunk_cnt = nullptr;
    BatchItem* items = nullptr;   // host-planned items (start-up, energy)
    size_t items_cap = 0;
    // device-driven cycle: plan and items built on the device
    int64_t* d_pk = nullptr;      // [K] padded sizes
    int32_t* kni = nullptr;       // [K] launch variant of the cluster this cycle
    int32_t* koff = nullptr;      // [K] first item of the cluster this cycle
    BatchItem* d_items = nullptr;
    int d_items_cap = 0;
    int force_slots = 0;          // SMs x occupancy of the persistent force kernel
    int waves = 4;                // the plan's waves of force items (nb_batch_autotune)
    int graph_cycles = 0;
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t graph_stream = nullptr;
    double* esum = nullptr;  // [3K] per-cluster kinetic, potential, sync flag
    // pinned mirrors
    double* h_tblk = nullptr;
    int32_t* h_kstart = nullptr;
    int32_t* h_kcount = nullptr;
    int32_t* h_ksplit = nullptr;
    BatchItem* h_items = nullptr;
    double* h_esum = nullptr;
    char err[512] = {0};
};

namespace {

int berr(nb_batch* b, int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b->err, sizeof b->err, fmt, ap);
    va_end(ap);
    return code;
}

#define B_CUDA(b, call)                                                                                        \
    do {                                                                                                       \
        cudaError_t e_ = (call);                                                                               \
        if (e_ != cudaSuccess) return berr((b), NB_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
    } while (0)

#define B_TRY(expr)                 \
    do {                            \
        int r_ = (expr);            \
        if (r_ != NB_OK) return r_; \
    } while (0)

// ------------------------------------------------------------------ kernels
constexpr int BNT = 256;

constexpr int BPER = 8;
constexpr int BCHUNK = BNT * BPER;

// Order-preserving key of a non-NaN double (k(a) < k(b) <=> a < b), and back.
constexpr unsigned long long KEY_EMPTY = ~0ull;
__device__ __forceinline__ unsigned long long time_key(double x)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double key_time(unsigned long long k)
{
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k));
}

// Block time of each cluster, first pass: min_i (t_i + dt_i) over the
// cluster's particles, as keys into kmin[k] (atomicMin).  CTA = BCHUNK slots,
// warp w = 256 consecutive slots as 8 groups of 32; clusters start on
// multiples of JT (a multiple of 32), so a group's real slots share one
// cluster and a warp meets at most a few clusters, flushing its running
// minimum when the cluster changes.  The only FP64 operation is the sum
// t + dt (the FP64 pipe runs at 1/64 of the FP32 rate here); comparisons run
// on the keys.
__global__ void __launch_bounds__(BNT) k_batch_tmin(const double* __restrict__ t, const double* __restrict__ dt,
                                                    const int32_t* __restrict__ cid, int64_t n,
                                                    unsigned long long* __restrict__ kmin, DevScalars* sc)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t s0 = (int64_t)blockIdx.x * BCHUNK + (int64_t)warp * 256;
    int cur = -1;
    unsigned long long cmin = KEY_EMPTY;
    bool bad = false;
    auto flush = [&]() {
        if (lane == 0 && cur >= 0 && cmin != KEY_EMPTY) atomicMin(&kmin[cur], cmin);
    };
    // all eight groups' loads first, then the reductions and flushes
    int kg[8];
    unsigned long long kv[8];
#pragma unroll
    for (int g = 0; g < 8; ++g) {
        const int64_t i = s0 + g * 32 + lane;
        kg[g] = i < n ? cid[i] : -1;
        kv[g] = KEY_EMPTY;
        if (kg[g] >= 0) {
            const double tn = t[i] + dt[i];
            if (tn == tn) kv[g] = time_key(tn);
            else bad = true;
        }
    }
#pragma unroll
    for (int g = 0; g < 8; ++g) {
        const int k = kg[g];
        unsigned long long key = kv[g];
        const int gk = __reduce_max_sync(0xffffffffu, k);
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long y = __shfl_xor_sync(0xffffffffu, key, o);
            key = y < key ? y : key;
        }
        if (gk < 0) continue;
        if (gk != cur) {
            flush();
            cur = gk;
            cmin = key;
        } else if (key < cmin) {
            cmin = key;
        }
    }
    flush();
    if (bad) raise_status(sc, NB_ERR_NAN);
}

// Second pass: tblk[k] from the key, +inf past t_end (the cluster idles);
// the key is reset for the next cycle.
__global__ void k_batch_tfinal(int K, unsigned long long* __restrict__ kmin, double* __restrict__ tblk,
                               const DevScalars* __restrict__ sc)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const unsigned long long key = kmin[k];
    kmin[k] = KEY_EMPTY;
    const double b = key == KEY_EMPTY ? INFINITY : key_time(key);
    tblk[k] = b <= sc->t_end ? b : INFINITY;
}

// t_i + dt_i == tblk[k] as bits (both sides exact dyadic sums; no FP64 compare)
__device__ __forceinline__ bool batch_active(const double* t, const double* dt, const int32_t* cid,
                                             const double* tblk, int64_t i)
{
    const int k = cid[i];
    return k >= 0 && __double_as_longlong(t[i] + dt[i]) == __double_as_longlong(tblk[k]);
}

__global__ void k_batch_count(const double* __restrict__ t, const double* __restrict__ dt,
                              const int32_t* __restrict__ cid, const double* __restrict__ tblk, int64_t n,
                              int32_t* __restrict__ cnt)
{
    __shared__ int wc[BNT / 32];
    const int64_t base = (int64_t)blockIdx.x * BCHUNK;
    int c = 0;
    for (int it = 0; it < BPER; ++it) {
        const int64_t i = base + it * BNT + threadIdx.x;
        if (i < n && batch_active(t, dt, cid, tblk, i)) ++c;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) wc[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < BNT / 32; ++w) s += wc[w];
        cnt[blockIdx.x] = s;
    }
}

__global__ void k_batch_scatter(const double* __restrict__ t, const double* __restrict__ dt,
                                const int32_t* __restrict__ cid, const double* __restrict__ tblk, int64_t n,
                                const int32_t* __restrict__ cnt, int nchunks, int32_t* __restrict__ idx,
                                DevScalars* sc)
{
    __shared__ int wtot[BNT / 32];
    __shared__ int s_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int o = 0;
    for (int k = threadIdx.x; k < (int)blockIdx.x; k += BNT) o += cnt[k];
    for (int s = 16; s > 0; s >>= 1) o += __shfl_xor_sync(0xffffffffu, o, s);
    if (lane == 0) wtot[warp] = o;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < BNT / 32; ++w) s += wtot[w];
        s_base = s;
    }
    __syncthreads();
    int base = s_base;
    const int64_t c0 = (int64_t)blockIdx.x * BCHUNK;
    for (int it = 0; it < BPER; ++it) {
        __syncthreads();
        const int64_t i = c0 + it * BNT + threadIdx.x;
        const bool f = i < n && batch_active(t, dt, cid, tblk, i);
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (lane == 0) wtot[warp] = __popc(bal);
        __syncthreads();
        int woff = 0, tot = 0;
        for (int w = 0; w < BNT / 32; ++w) {
            const int x = wtot[w];
            if (w < warp) woff += x;
            tot += x;
        }
        if (f) idx[base + woff + __popc(bal & ((1u << lane) - 1u))] = (int32_t)i;
        base += tot;
    }
    if (blockIdx.x == nchunks - 1 && threadIdx.x == 0) {
        sc->n_act = base;
        sc->idle = base == 0;
    }
}

__global__ void k_batch_counts(int K, const int32_t* __restrict__ kstart, int32_t* __restrict__ kcount)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < K && kcount[k] > 0) kcount[k] -= kstart[k];
}

// One item per CTA, in the item's launch variant (the cluster's active-set
// size picks it with the rule of a single system, mixed_ni: two i-particles
// per thread in packed FP32x2 lanes from 512 active on).
template <int ORDER, int RW>
__global__ void __launch_bounds__(FORCE_NT, dyn_min_ctas(ORDER)) k_batch_force_mixed(const float4* __restrict__ js,
                                                                   const int32_t* __restrict__ list,
                                                                   const BatchItem* __restrict__ items, int n_act,
                                                                   int n, float eps2max, double* __restrict__ partial,
                                                                   DevScalars* sc)
{
    const BatchItem it = items[blockIdx.x];
    const int lim = it.list_off + it.count;
    if (it.ni == 2 * FORCE_NT)
        xs_item<ORDER, RW, true>(js, list, it.list_off, lim, n, it.jt0, it.nt, it.split, n_act, 0.0f, eps2max, partial,
                                 sc, TileSum{});
    else if (it.ni == FORCE_NT)
        force_block_mixed<ORDER, RW, true, 1>(js, list, it.list_off, lim, n, it.jt0, it.nt, it.split, n_act, 0.0f,
                                              eps2max, partial, sc);
    else if (it.ni == FORCE_NT / 4)
        force_block_mixed_jp<ORDER, RW, true, 4>(js, list, it.list_off, lim, n, it.jt0, it.nt, it.split, n_act, 0.0f,
                                                 eps2max, partial, sc);
    else
        force_block_mixed_jp<ORDER, RW, true, 32>(js, list, it.list_off, lim, n, it.jt0, it.nt, it.split, n_act,
                                                  0.0f, eps2max, partial, sc);
}

// ------------------------------------------------ device-driven cycle
// Segment of each cluster in the (cluster-major, ascending) active list; the
// cycle's active-set size lives in sc->n_act, a fixed grid strides.
__global__ void k_batch_bounds_dyn(const int32_t* __restrict__ list, const DevScalars* __restrict__ sc,
                                   const int32_t* __restrict__ cid, int32_t* __restrict__ kstart,
                                   int32_t* __restrict__ kcount)
{
    const int n_act = (int)sc->n_act;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_act; p += gridDim.x * blockDim.x) {
        const int k = cid[list[p]];
        if (p == 0 || cid[list[p - 1]] != k) kstart[k] = p;
        if (p == n_act - 1 || cid[list[p + 1]] != k) kcount[k] = p + 1;
    }
}

// Plan of the cycle's force (one CTA): each cluster with cnt active takes the
// launch variant ni = mixed_ni(cnt) (fp64_ni(cnt) in FP64) and
// s j-splits, s = ceil(min(cnt, ni) * pk / target) in [1, pk / JT], with
// target = max(work / (waves slots), FORCE_NT * JT) and work = sum cnt * pk:
// items of about equal work, about `waves` waves of them (4 unless
// nb_batch_autotune measured another count faster).  The largest split is then
// capped by the partial-sum buffer.  The force kernel hands items out in
// table order, so the table lists the heavy items first: clusters whose item
// work min(cnt, ni) pk / s is at least target / 2, then at least target / 8,
// then the rest (cluster order within a class), and the short items fill the
// gaps at the end.  Writes ksplit, kni, koff (first item of each cluster),
// n_items, the item counter, the clusters stepped and the interactions of
// the cycle.
__global__ void __launch_bounds__(BNT) k_batch_plan(int K, const int32_t* __restrict__ kcount,
                                                    const int64_t* __restrict__ pk, const int64_t* __restrict__ nk,
                                                    int slots, int waves, long long cap, int nc, int mixed,
                                                    int items_cap,
                                                    int32_t* __restrict__ ksplit, int32_t* __restrict__ kni,
                                                    int32_t* __restrict__ koff, DevScalars* sc)
{
    __shared__ long long s_ll[BNT / 32];
    __shared__ int s_i[BNT / 32];
    __shared__ double s_target;
    __shared__ int s_smax;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (sc->idle) {
        if (tid == 0) {
            sc->n_items = 0;
            sc->next_item = 0;
            sc->stepped = 0;
        }
        return;
    }
    auto block_sum = [&](long long v) {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        __syncthreads();
        if (lane == 0) s_ll[warp] = v;
        __syncthreads();
        long long t = 0;
        for (int w = 0; w < BNT / 32; ++w) t += s_ll[w];
        return t;
    };
    long long work = 0, inter = 0, stepped = 0;
    for (int k = tid; k < K; k += BNT) {
        const long long cnt = kcount[k];
        if (cnt > 0) {
            work += cnt * pk[k];
            inter += cnt * nk[k];
            ++stepped;
        }
    }
    work = block_sum(work);
    inter = block_sum(inter);
    stepped = block_sum(stepped);
    if (tid == 0) s_target = fmax((double)work / ((double)waves * slots), (double)FORCE_NT * JT);
    __syncthreads();
    const double target = s_target;
    int smax = 1;
    for (int k = tid; k < K; k += BNT) {
        const int cnt = kcount[k];
        const int ni = mixed ? mixed_ni(cnt) : fp64_ni(cnt);
        const int jt = (int)(pk[k] / JT);
        int sk = 1;
        if (cnt > 0) {
            sk = (int)ceil((double)min(cnt, ni) * (double)pk[k] / target);
            sk = max(1, min(sk, jt));
        }
        ksplit[k] = sk;
        kni[k] = ni;
        smax = max(smax, sk);
    }
    for (int o = 16; o > 0; o >>= 1) smax = max(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    __syncthreads();
    if (lane == 0) s_i[warp] = smax;
    __syncthreads();
    if (tid == 0) {
        int m = 1;
        for (int w = 0; w < BNT / 32; ++w) m = max(m, s_i[w]);
        const long long n_act = sc->n_act;
        while (m > 1 && (long long)m * nc * n_act > cap) --m;
        s_smax = m;
    }
    __syncthreads();
    const int scap = s_smax;
    for (int k = tid; k < K; k += BNT) ksplit[k] = min(ksplit[k], scap);
    // items per cluster and their exclusive scan, one class after another,
    // BNT clusters at a time (thread tid keeps clusters tid + BNT m)
    auto item_class = [&](int k) {
        const long long cnt = kcount[k];
        const double w = (double)min(cnt, (long long)kni[k]) * (double)pk[k] / ksplit[k];
        return w >= 0.5 * target ? 0 : w >= 0.125 * target ? 1 : 2;
    };
    int running = 0;
    for (int cls = 0; cls < 3; ++cls)
        for (int base = 0; base < K; base += BNT) {
            const int k = base + tid;
            int items = 0;
            if (k < K) {
                const int cnt = kcount[k];
                if (cnt > 0 && item_class(k) == cls) items = (cnt + kni[k] - 1) / kni[k] * ksplit[k];
            }
            int incl = items;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            __syncthreads();
            if (lane == 31) s_i[warp] = incl;
            __syncthreads();
            int wbase = 0, tot = 0;
            for (int w = 0; w < BNT / 32; ++w) {
                if (w < warp) wbase += s_i[w];
                tot += s_i[w];
            }
            if (items > 0) koff[k] = running + wbase + incl - items;
            running += tot;
        }
    if (tid == 0) {
        if (running > items_cap) {
            raise_status(sc, NB_ERR_ARG);
            running = items_cap;
        }
        sc->n_items = running;
        sc->next_item = 0;
        sc->stepped = (int)stepped;
        sc->blocks += stepped > 0 ? 1 : 0;
        sc->inter += inter;
    }
}

// Items of cluster k = blockIdx.x in (i-tile, split) order at koff[k].
__global__ void __launch_bounds__(BNT) k_batch_items(const int32_t* __restrict__ kstart,
                                                     const int32_t* __restrict__ kcount,
                                                     const int32_t* __restrict__ ksplit,
                                                     const int32_t* __restrict__ kni, const int32_t* __restrict__ koff,
                                                     const int64_t* __restrict__ off, const int64_t* __restrict__ pk,
                                                     int items_cap, BatchItem* __restrict__ items)
{
    const int k = blockIdx.x;
    const int cnt = kcount[k];
    if (cnt <= 0) return;
    const int sk = ksplit[k], ni = kni[k], it = (cnt + ni - 1) / ni;
    const int jt = (int)(pk[k] / JT), jt0 = (int)(off[k] / JT), o = koff[k];
    for (int q = threadIdx.x; q < it * sk; q += BNT) {
        if (o + q >= items_cap) return;
        const int i_tile = q / sk, s = q - i_tile * sk;
        BatchItem e{};
        e.list_off = kstart[k] + i_tile * ni;
        e.count = min(ni, cnt - i_tile * ni);
        const int a = (int)((long long)s * jt / sk), b = (int)((long long)(s + 1) * jt / sk);
        e.jt0 = jt0 + a;
        e.nt = b - a;
        e.split = s;
        e.ni = ni;
        items[o + q] = e;
    }
}

// Persistent force over the cycle's items (count in sc->n_items): each CTA
// takes the next item from a counter, so that CTAs that drew short items take
// more of them.
template <int ORDER, int RW>
__global__ void __launch_bounds__(FORCE_NT, dyn_min_ctas(ORDER)) k_batch_force_mixed_dyn(const float4* __restrict__ js,
                                                                       const int32_t* __restrict__ list,
                                                                       const BatchItem* __restrict__ items, int n,
                                                                       float eps2max, double* __restrict__ partial,
                                                                       DevScalars* sc)
{
    if (sc->idle) return;
    const int n_items = sc->n_items, n_act = (int)sc->n_act;
    __shared__ int s_w;
    if (threadIdx.x == 0) s_w = atomicAdd(&sc->next_item, 1);
    __syncthreads();
    for (int w = s_w; w < n_items; w = s_w) {
        const BatchItem it = items[w];
        const int lim = it.list_off + it.count;
        if (it.ni == 2 * FORCE_NT)
            xs_item<ORDER, RW, true>(js, list, it.list_off, lim, n, it.jt0, it.nt, it.split, n_act, 0.0f, eps2max,
                                     partial, sc, TileSum{});
        else if (it.ni == FORCE_NT)
            force_block_mixed<ORDER, RW, true, 1>(js, list, it.list_off, lim, n, it.jt0, it.nt, it.split, n_act, 0.0f,
                                                  eps2max, partial, sc);
        else if (it.ni == FORCE_NT / 4)
            force_block_mixed_jp<ORDER, RW, true, 4>(js, list, it.list_off, lim, n, it.jt0, it.nt, it.split, n_act,
                                                     0.0f, eps2max, partial, sc);
        else
            force_block_mixed_jp<ORDER, RW, true, 32>(js, list, it.list_off, lim, n, it.jt0, it.nt, it.split, n_act,
                                                      0.0f, eps2max, partial, sc);
        // the next item: taken after every thread has read w (the item's own
        // barriers lie between), published by the barrier below
        if (threadIdx.x == 0) s_w = atomicAdd(&sc->next_item, 1);
        if (__syncthreads_or(threadIdx.x == 0 && *(volatile int*)&sc->status != 0)) return;
    }
}

template <int ORDER, int RW>
__global__ void __launch_bounds__(FORCE_NT) k_batch_force_fp64_dyn(const double2* __restrict__ js,
                                                                   const int32_t* __restrict__ list,
                                                                   const BatchItem* __restrict__ items, int n,
                                                                   double* __restrict__ partial, DevScalars* sc)
{
    if (sc->idle) return;
    const int n_items = sc->n_items, n_act = (int)sc->n_act;
    __shared__ int s_w;
    if (threadIdx.x == 0) s_w = atomicAdd(&sc->next_item, 1);
    __syncthreads();
    for (int w = s_w; w < n_items; w = s_w) {
        const BatchItem it = items[w];
        const int lim = it.list_off + it.count;
        if (it.ni == FORCE_NT)
            force_block_fp64<ORDER, RW, true, 1>(js, list, it.list_off, lim, n, it.jt0, it.nt, it.split, n_act, 0.0,
                                                 partial, sc);
        else if (it.ni == FORCE_NT / 4)
            force_block_fp64<ORDER, RW, true, 4>(js, list, it.list_off, lim, n, it.jt0, it.nt, it.split, n_act, 0.0,
                                                 partial, sc);
        else
            force_block_fp64<ORDER, RW, true, 32>(js, list, it.list_off, lim, n, it.jt0, it.nt, it.split, n_act, 0.0,
                                                  partial, sc);
        // the next item: taken after every thread has read w (the item's own
        // barriers lie between), published by the barrier below
        if (threadIdx.x == 0) s_w = atomicAdd(&sc->next_item, 1);
        if (__syncthreads_or(threadIdx.x == 0 && *(volatile int*)&sc->status != 0)) return;
    }
}

// F[c][p] = sum over the particle's cluster splits (fixed order); a fixed
// grid strides over the (component, particle) pairs of the cycle, one sum
// per thread (eleven times the parallelism of a thread per particle, which
// left the many-split sums waiting on memory).
template <int NC, int PC>
__global__ void k_batch_reduce_dyn(const double* __restrict__ partial, const int32_t* __restrict__ list,
                                   const int32_t* __restrict__ cid, const int32_t* __restrict__ ksplit,
                                   const DevScalars* __restrict__ sc, double* __restrict__ F)
{
    if (sc->idle) return;
    const int n_act = (int)sc->n_act;
    const long long total = (long long)NC * n_act;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(q / n_act), p = (int)(q - (long long)c * n_act);
        const int S = ksplit[cid[list[p]]];
        const double* src = partial + (size_t)c * n_act + p;
        const size_t stride = (size_t)NC * n_act;
        double s = 0.0;
#pragma unroll 8
        for (int sp = 0; sp < S; ++sp) s += src[(size_t)sp * stride];
        F[(size_t)c * n_act + p] = c == PC ? -s : s;
    }
}

template <int ORDER, int RW>
__global__ void __launch_bounds__(FORCE_NT) k_batch_force_fp64(const double2* __restrict__ js,
                                                               const int32_t* __restrict__ list,
                                                               const BatchItem* __restrict__ items, int n_act, int n,
                                                               double* __restrict__ partial, DevScalars* sc)
{
    const BatchItem it = items[blockIdx.x];
    force_block_fp64<ORDER, RW, true>(js, list, it.list_off, it.list_off + it.count, n, it.jt0, it.nt, it.split,
                                      n_act, 0.0, partial, sc);
}

// F[c][p] = sum over the particle's cluster splits (fixed order); potential negated.
template <int NC, int PC>
__global__ void k_batch_reduce(const double* __restrict__ partial, const int32_t* __restrict__ list,
                               const int32_t* __restrict__ cid, const int32_t* __restrict__ ksplit, int n_act,
                               double* __restrict__ F)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_act) return;
    const int S = ksplit[cid[list[p]]];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        double s = 0.0;
        for (int sp = 0; sp < S; ++sp) s += partial[((size_t)sp * NC + c) * n_act + p];
        F[(size_t)c * n_act + p] = c == PC ? -s : s;
    }
}

template <int PASS>
__global__ void k_batch_startup_store(const double* __restrict__ F, const int32_t* __restrict__ list, int n_act,
                                      int64_t np, double* __restrict__ d, double* __restrict__ pot)
{
    constexpr int MM = PASS / 2;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_act) return;
    const int64_t i = list[p];
#pragma unroll
    for (int k = 0; k < MM; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) d[(k * 3 + c) * np + i] = F[(size_t)(3 * k + c) * n_act + p];
    pot[i] = F[(size_t)(3 * MM) * n_act + p];
}

// Start-up step eta_s |a| / |jerk| quantised at t = 0 (same rule as one system).
__global__ void k_batch_startup_dt(const double* __restrict__ d, const int32_t* __restrict__ list, int n_act,
                                   int64_t np, double* __restrict__ t, double* __restrict__ dtv, double eta_s,
                                   double dt_max, double dt_min, DevScalars* sc)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_act) return;
    const int64_t i = list[p];
    double na = 0.0, nj = 0.0;
    for (int c = 0; c < 3; ++c) {
        const double a = d[(0 * 3 + c) * np + i], j = d[(1 * 3 + c) * np + i];
        na += a * a;
        nj += j * j;
    }
    na = sqrt(na);
    nj = sqrt(nj);
    double lim = nj > 0.0 ? eta_s * na / nj : INFINITY;
    double dtn;
    if (!(lim == lim)) {
        raise_status(sc, NB_ERR_NAN);
        dtn = dt_max;
    } else if (lim >= dt_max) dtn = dt_max;
    else if (lim < dt_min) {
        raise_status(sc, NB_ERR_DT_UNDERFLOW);
        dtn = dt_min;
    } else dtn = __longlong_as_double(__double_as_longlong(lim) & 0xFFF0000000000000LL);
    t[i] = 0.0;
    dtv[i] = dtn;
}

// Per-cluster energy sums (one CTA per cluster) over the real list segment
// [roff, roff + nk): kinetic, potential (pot in list order), and whether all
// of the cluster's particles share one time.
__global__ void k_batch_energy(const double* __restrict__ m, const double* __restrict__ v,
                               const double* __restrict__ t, const double* __restrict__ pot_list,
                               const int32_t* __restrict__ list, const int64_t* __restrict__ roff,
                               const int64_t* __restrict__ nk, int64_t np, double* __restrict__ out)
{
    __shared__ double sk[BNT / 32], sp[BNT / 32], sd[BNT / 32];
    const int k = blockIdx.x;
    const int64_t r0 = roff[k];
    const double t0 = t[list[r0]];
    double ek = 0.0, ep = 0.0, dev = 0.0;
    for (int64_t p = r0 + threadIdx.x; p < r0 + nk[k]; p += BNT) {
        const int64_t i = list[p];
        const double vx = v[i], vy = v[np + i], vz = v[2 * np + i];
        ek += 0.5 * m[i] * (vx * vx + vy * vy + vz * vz);
        if (pot_list) ep += 0.5 * m[i] * pot_list[p];
        dev = fmax(dev, fabs(t[i] - t0));
    }
    for (int o = 16; o > 0; o >>= 1) {
        ek += __shfl_xor_sync(0xffffffffu, ek, o);
        ep += __shfl_xor_sync(0xffffffffu, ep, o);
        dev = fmax(dev, __shfl_xor_sync(0xffffffffu, dev, o));
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        sk[w] = ek;
        sp[w] = ep;
        sd[w] = dev;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0, c = 0;
        for (int q = 0; q < BNT / 32; ++q) {
            a += sk[q];
            b += sp[q];
            c = fmax(c, sd[q]);
        }
        out[3 * k] = a;
        out[3 * k + 1] = b;
        out[3 * k + 2] = c;
    }
}

// Block time of each cluster = the time of its first particle (for energy).
__global__ void k_batch_first_time(const double* __restrict__ t, const int64_t* __restrict__ off, int K,
                                   double* __restrict__ tblk)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < K) tblk[k] = t[off[k]];
}

// ------------------------------------------------------------------- host
template <typename T>
int balloc(nb_batch* b, T** p, size_t count)
{
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count * sizeof(T), 256));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return berr(b, NB_ERR_NOMEM, "cudaMalloc failed: %s", cudaGetErrorString(e));
    }
    *p = static_cast<T*>(q);
    return NB_OK;
}

int bsync(nb_batch* b)
{
    nb_ctx* c = b->c;
    B_CUDA(b, cudaMemcpyAsync(c->h_sc, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream));
    B_CUDA(b, cudaStreamSynchronize(c->stream));
    if (c->h_sc->status != NB_OK) {
        const int st = c->h_sc->status;
        B_CUDA(b, cudaMemsetAsync(&c->sc->status, 0, sizeof(int), c->stream));
        B_CUDA(b, cudaStreamSynchronize(c->stream));
        return berr(b, st, "device kernel reported error %d", st);
    }
    return NB_OK;
}

// Occupancy of a batch force kernel (configured once per kernel).
template <typename K>
int occ_of(K kern, size_t smem)
{
    static std::map<const void*, int> cache;
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    const void* key = reinterpret_cast<const void*>(kern);
    auto f = cache.find(key);
    if (f != cache.end()) return f->second;
    int occ = 1;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, FORCE_NT, smem) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    cache[key] = occ;
    return occ;
}

// Launch the batched force kernel (computed order `order`, stored layout of
// the context) for `nitems` items; occ_only: return the occupancy instead.
template <int SO>
int batch_force_dispatch(nb_batch* b, int order, const int32_t* list, int n_act, int nitems, bool occ_only)
{
    nb_ctx* c = b->c;
    const bool mixed = c->pred_prec == NB_MIXED;
#define BCASE(O)                                                                                                  \
    if (order == O) {                                                                                             \
        if (mixed) {                                                                                              \
            constexpr int RW = mixed_rw(SO);                                                                      \
            const size_t smem = xs_smem(O, RW, 1);                                                                \
            auto kern = k_batch_force_mixed<O, RW>;                                                            \
            const int occ = occ_of(kern, smem);                                                                   \
            if (occ_only) return occ;                                                                             \
            kern<<<nitems, FORCE_NT, smem, c->stream>>>(reinterpret_cast<const float4*>(c->jstore), list,         \
                                                        b->items, n_act, (int)c->n,                               \
                                                        eps2_threshold(c->eps2_max),                              \
                                                        c->partial, c->sc);                                       \
        } else {                                                                                                  \
            constexpr int RW = fp64_rw(SO);                                                                       \
            const size_t smem = (size_t)NSTAGE * JT * RW * 16;                                                    \
            auto kern = k_batch_force_fp64<O, RW>;                                                                \
            const int occ = occ_of(kern, smem);                                                                   \
            if (occ_only) return occ;                                                                             \
            kern<<<nitems, FORCE_NT, smem, c->stream>>>(reinterpret_cast<const double2*>(c->jstore), list,        \
                                                        b->items, n_act, (int)c->n, c->partial, c->sc);           \
        }                                                                                                         \
        return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ERR_CUDA;                                           \
    }
    BCASE(0)
    BCASE(4)
    if constexpr (SO >= 6) {
        BCASE(6)
    }
    if constexpr (SO >= 8) {
        BCASE(8)
    }
#undef BCASE
    return NB_ERR_ARG;
}

int batch_force_call(nb_batch* b, int order, const int32_t* list, int n_act, int nitems, bool occ_only)
{
    switch (b->c->order) {
    case 4: return batch_force_dispatch<4>(b, order, list, n_act, nitems, occ_only);
    case 6: return batch_force_dispatch<6>(b, order, list, n_act, nitems, occ_only);
    default: return batch_force_dispatch<8>(b, order, list, n_act, nitems, occ_only);
    }
}

int batch_reduce(nb_batch* b, int order, const int32_t* list, int n_act)
{
    nb_ctx* c = b->c;
    const int g = (n_act + 255) / 256;
#define BRED(O) \
    k_batch_reduce<ncomp(O), pot_comp(O)><<<g, 256, 0, c->stream>>>(c->partial, list, b->cid, b->ksplit, n_act, c->F)
    if (order == 0) BRED(0);
    else if (order == 4) BRED(4);
    else if (order == 6) BRED(6);
    else BRED(8);
#undef BRED
    c->n_launch += 1;
    return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}

// Force of the listed particles, given each cluster's segment of the list
// (h_start/h_count on the host); j ranges are the clusters' own tiles.
int batch_force(nb_batch* b, int order, const int32_t* list, int n_act, const int32_t* h_start,
                const int32_t* h_count)
{
    nb_ctx* c = b->c;
    const int nc = ncomp(order);
    // split each cluster's j range so that items carry similar work
    double work = 0.0;
    for (int k = 0; k < b->K; ++k) work += (double)h_count[k] * (double)b->pk[k];
    const int occ = batch_force_call(b, order, list, n_act, 0, true);
    const double target = std::max(work / (4.0 * occ * c->sm_count), (double)FORCE_NT * JT);
    int smax = 1;
    size_t nitems = 0;
    const bool mixed = c->pred_prec == NB_MIXED;  // the kernel batch_force_call launches
    auto variant = [&](int count) { return mixed ? mixed_ni(count) : FORCE_NT; };
    for (int k = 0; k < b->K; ++k) {
        b->h_ksplit[k] = 1;
        if (h_count[k] <= 0) continue;
        const int jt = (int)(b->pk[k] / JT), ni = variant(h_count[k]);
        const double item_work = (double)std::min(h_count[k], ni) * (double)b->pk[k];
        int s = (int)std::ceil(item_work / target);
        s = std::max(1, std::min(s, jt));
        b->h_ksplit[k] = s;
        smax = std::max(smax, s);
        nitems += (size_t)((h_count[k] + ni - 1) / ni) * s;
    }
    while (smax > 1 && (size_t)smax * nc * (size_t)n_act > c->partial_cap) {
        --smax;
        for (int k = 0; k < b->K; ++k) b->h_ksplit[k] = std::min(b->h_ksplit[k], smax);
    }
    if (nitems == 0) return NB_OK;
    if (nitems > b->items_cap) {
        if (b->items) cudaFree(b->items);
        if (b->h_items) cudaFreeHost(b->h_items);
        b->items = nullptr;
        b->h_items = nullptr;
        b->items_cap = nitems * 2;
        B_TRY(balloc(b, &b->items, b->items_cap));
        B_CUDA(b, cudaMallocHost(&b->h_items, b->items_cap * sizeof(BatchItem)));
    }
    size_t q = 0;
    for (int k = 0; k < b->K; ++k) {
        if (h_count[k] <= 0) continue;
        const int jt = (int)(b->pk[k] / JT), jt0 = (int)(b->off[k] / JT), s_k = b->h_ksplit[k];
        const int ni = variant(h_count[k]);
        for (int i0 = 0; i0 < h_count[k]; i0 += ni)
            for (int s = 0; s < s_k; ++s) {
                BatchItem it{};
                it.list_off = h_start[k] + i0;
                it.count = std::min(ni, h_count[k] - i0);
                it.ni = ni;
                const int a = (int)((long long)s * jt / s_k), e = (int)((long long)(s + 1) * jt / s_k);
                it.jt0 = jt0 + a;
                it.nt = e - a;
                it.split = s;
                b->h_items[q++] = it;
            }
    }
    B_CUDA(b, cudaMemcpyAsync(b->items, b->h_items, nitems * sizeof(BatchItem), cudaMemcpyHostToDevice, c->stream));
    B_CUDA(b, cudaMemcpyAsync(b->ksplit, b->h_ksplit, b->K * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    if (batch_force_call(b, order, list, n_act, (int)nitems, false) != NB_OK)
        return berr(b, NB_ERR_CUDA, "batch force launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    c->n_launch += 1;
    B_TRY(batch_reduce(b, order, list, n_act));
    c->F_order = order;
    c->F_n = n_act;
    // the item table and splits are read asynchronously: keep them until done
    B_CUDA(b, cudaStreamSynchronize(c->stream));
    return NB_OK;
}

// ------------------------------------------------ device-driven cycle (host)
// scheduler 4 (block times 2, count, scatter), bounds 2, plan, items,
// predictor, force, reduction, corrector
constexpr int BATCH_CYCLE_LAUNCHES = 12;
// largest wave count of the force plan (the item buffer is sized for it)
constexpr int BATCH_WAVES_MAX = 8;
// a wave count replaces the default only when it is this much faster
constexpr double BATCH_TUNE_MARGIN = 0.97;

void batch_destroy_graph(nb_batch* b)
{
    if (b->graph_exec) {
        cudaGraphExecDestroy(b->graph_exec);
        b->graph_exec = nullptr;
    }
}

template <int SO>
int batch_force_dyn_o(nb_batch* b, bool occ_only)
{
    nb_ctx* c = b->c;
    if (c->prec == NB_MIXED) {
        constexpr int RW = mixed_rw(SO);
        const size_t smem = xs_smem(SO, RW, 1);
        auto kern = k_batch_force_mixed_dyn<SO, RW>;
        if (occ_only) return occ_of(kern, smem);
        kern<<<b->force_slots, FORCE_NT, smem, c->stream>>>(reinterpret_cast<const float4*>(c->jstore), c->act_idx,
                                                             b->d_items, (int)c->n, eps2_threshold(c->eps2_max),
                                                             c->partial, c->sc);
    } else {
        constexpr int RW = fp64_rw(SO);
        const size_t smem = (size_t)NSTAGE * JT * RW * 16;
        auto kern = k_batch_force_fp64_dyn<SO, RW>;
        if (occ_only) return occ_of(kern, smem);
        kern<<<b->force_slots, FORCE_NT, smem, c->stream>>>(reinterpret_cast<const double2*>(c->jstore), c->act_idx,
                                                             b->d_items, (int)c->n, c->partial, c->sc);
    }
    return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}

int batch_force_dyn(nb_batch* b, bool occ_only)
{
    switch (b->c->order) {
    case 4: return batch_force_dyn_o<4>(b, occ_only);
    case 6: return batch_force_dyn_o<6>(b, occ_only);
    default: return batch_force_dyn_o<8>(b, occ_only);
    }
}

// Slots of the persistent force in the current precision and an item buffer
// that holds every plan: items <= waves slots + np/64 + 8K (each cluster's
// split count rounds up by at most one, its i-tiles number at most
// cnt/128 + 8), waves <= BATCH_WAVES_MAX.
int batch_prepare(nb_batch* b)
{
    nb_ctx* c = b->c;
    const int slots = c->sm_count * batch_force_dyn(b, true);
    const long long need = 2LL * BATCH_WAVES_MAX * slots + c->np / 32 + 8LL * b->K + 1024;
    if (slots != b->force_slots || need > b->d_items_cap) {
        batch_destroy_graph(b);
        b->force_slots = slots;
    }
    if (need > b->d_items_cap) {
        B_CUDA(b, cudaStreamSynchronize(c->stream));
        if (b->d_items) cudaFree(b->d_items);
        b->d_items = nullptr;
        b->d_items_cap = 0;
        B_TRY(balloc(b, &b->d_items, (size_t)need));
        b->d_items_cap = (int)need;
    }
    c->pred_prec = c->prec;
    return NB_OK;
}

// t_end of the coming cycles, counters cleared.
int batch_reset_scalars(nb_batch* b, double t_end, cudaStream_t st)
{
    nb_ctx* c = b->c;
    DevScalars* h = c->h_sc;
    B_CUDA(b, cudaStreamSynchronize(c->stream));
    B_CUDA(b, cudaMemcpy(h, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost));
    h->t_end = t_end;
    h->idle = 0;
    h->blocks = 0;
    h->inter = 0;
    h->stepped = 0;
    B_CUDA(b, cudaMemcpyAsync(c->sc, h, sizeof(DevScalars), cudaMemcpyHostToDevice, st));
    B_CUDA(b, cudaStreamSynchronize(st));
    return NB_OK;
}

// The launches of one ensemble cycle, every size read on the device: block
// time per cluster (idle past t_end), active list, cluster segments, the
// force plan and its items, predictor, persistent force, reduction,
// corrector.
// The first launches of an ensemble cycle: block time per cluster (idle
// past t_end), active list, cluster segments.
cudaError_t batch_cycle_front(nb_batch* b)
{
    nb_ctx* c = b->c;
    const int K = b->K, nch = (int)((c->n + BCHUNK - 1) / BCHUNK), g = c->sm_count * 4;
    k_batch_tmin<<<nch, BNT, 0, c->stream>>>(c->t, c->dt, b->cid, c->n, b->kmin, c->sc);
    k_batch_tfinal<<<(K + 255) / 256, 256, 0, c->stream>>>(K, b->kmin, b->tblk, c->sc);
    k_batch_count<<<nch, BNT, 0, c->stream>>>(c->t, c->dt, b->cid, b->tblk, c->n, b->chunk_cnt);
    k_batch_scatter<<<nch, BNT, 0, c->stream>>>(c->t, c->dt, b->cid, b->tblk, c->n, b->chunk_cnt, nch, c->act_idx,
                                                c->sc);
    cudaError_t e = cudaMemsetAsync(b->kcount, 0, K * sizeof(int32_t), c->stream);
    if (e != cudaSuccess) return e;
    k_batch_bounds_dyn<<<g, 256, 0, c->stream>>>(c->act_idx, c->sc, b->cid, b->kstart, b->kcount);
    k_batch_counts<<<(K + 255) / 256, 256, 0, c->stream>>>(K, b->kstart, b->kcount);
    return cudaGetLastError();
}

// The force plan with `waves` waves of items, and its item table.
cudaError_t batch_cycle_plan(nb_batch* b, int waves)
{
    nb_ctx* c = b->c;
    const int K = b->K;
    k_batch_plan<<<1, BNT, 0, c->stream>>>(K, b->kcount, b->d_pk, b->d_nk, b->force_slots, waves,
                                           (long long)c->partial_cap, ncomp(c->order), c->prec == NB_MIXED,
                                           b->d_items_cap, b->ksplit, b->kni, b->koff, c->sc);
    k_batch_items<<<K, BNT, 0, c->stream>>>(b->kstart, b->kcount, b->ksplit, b->kni, b->koff, b->d_off, b->d_pk,
                                            b->d_items_cap, b->d_items);
    return cudaGetLastError();
}

// The persistent force over the planned items and the reduction over each
// cluster's splits.
cudaError_t batch_cycle_force(nb_batch* b)
{
    nb_ctx* c = b->c;
    const int g = c->sm_count * 4;
    if (batch_force_dyn(b, false) != NB_OK) return cudaGetLastError();
#define BRED(O)                                                                                                   \
    k_batch_reduce_dyn<ncomp(O), pot_comp(O)><<<2 * g, 256, 0, c->stream>>>(c->partial, c->act_idx, b->cid,         \
                                                                            b->ksplit, c->sc, c->F)
    if (c->order == 4) BRED(4);
    else if (c->order == 6) BRED(6);
    else BRED(8);
#undef BRED
    return cudaGetLastError();
}

cudaError_t batch_cycle_launches(nb_batch* b)
{
    nb_ctx* c = b->c;
    cudaError_t e;
    if ((e = batch_cycle_front(b)) != cudaSuccess) return e;
    if ((e = batch_cycle_plan(b, b->waves)) != cudaSuccess) return e;
    if ((e = launch_predict(c, 0.0, b->tblk, b->cid, c->sc)) != cudaSuccess) return e;
    if ((e = batch_cycle_force(b)) != cudaSuccess) return e;
    if ((e = launch_correct(c, b->tblk, b->cid, c->sc)) != cudaSuccess) return e;
    c->n_launch += BATCH_CYCLE_LAUNCHES;
    return cudaGetLastError();
}

int batch_build_graph(nb_batch* b)
{
    nb_ctx* c = b->c;
    batch_destroy_graph(b);
    if (!b->graph_stream) B_CUDA(b, cudaStreamCreateWithFlags(&b->graph_stream, cudaStreamNonBlocking));
    cudaStream_t saved = c->stream;
    const int64_t launches = c->n_launch;
    c->stream = b->graph_stream;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->graph_stream, cudaStreamCaptureModeThreadLocal);
    for (int r = 0; e == cudaSuccess && r < b->graph_cycles; ++r) e = batch_cycle_launches(b);
    const cudaError_t e2 = cudaStreamEndCapture(b->graph_stream, &g);
    c->stream = saved;
    c->n_launch = launches;  // counted per replay
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph_exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        batch_destroy_graph(b);
        return berr(b, NB_ERR_CUDA, "ensemble cycle graph capture failed: %s", cudaGetErrorString(e));
    }
    return NB_OK;
}

}  // namespace

extern "C" {

const char* nb_batch_last_error(const nb_batch* b) { return b ? b->err : "NULL batch"; }

void nb_batch_destroy(nb_batch* b)
{
    if (!b) return;
    if (b->c) cudaStreamSynchronize(b->c->stream);
    batch_destroy_graph(b);
    if (b->graph_stream) cudaStreamDestroy(b->graph_stream);
    void* d[] = {b->cid,    b->real_idx, b->d_off, b->d_nk,    b->tblk, b->kmin, b->kstart, b->kcount,
                 b->ksplit, b->chunk_cnt, b->items, b->esum, b->d_pk, b->kni,  b->koff,   b->d_items};
    for (void* p : d)
        if (p) cudaFree(p);
    void* h[] = {b->h_tblk, b->h_kstart, b->h_kcount, b->h_ksplit, b->h_items, b->h_esum};
    for (void* p : h)
        if (p) cudaFreeHost(p);
    nb_destroy(b->c);
    delete b;
}

int nb_batch_create(nb_batch** out, int n_clusters, const int64_t* n_per_cluster, int order, double eps)
{
    if (!out) return NB_ERR_ARG;
    *out = nullptr;
    if (n_clusters < 1 || !n_per_cluster) return NB_ERR_ARG;
    nb_batch* b = new (std::nothrow) nb_batch();
    if (!b) return NB_ERR_NOMEM;
    b->K = n_clusters;
    int64_t slots = 0;
    for (int k = 0; k < n_clusters; ++k) {
        const int64_t nk = n_per_cluster[k];
        if (nk < 1) {
            delete b;
            return NB_ERR_ARG;
        }
        b->nk.push_back(nk);
        b->off.push_back(slots);
        b->pk.push_back((nk + JT - 1) / JT * JT);
        b->roff.push_back(b->n_real);
        b->n_real += nk;
        slots += b->pk.back();
    }
    int rc = nb_create(&b->c, slots, order, eps);
    if (rc != NB_OK) {
        delete b;
        return rc;
    }
    const int K = n_clusters;
    if ((rc = balloc(b, &b->cid, (size_t)b->c->np)) || (rc = balloc(b, &b->real_idx, (size_t)b->n_real)) ||
        (rc = balloc(b, &b->d_off, K)) || (rc = balloc(b, &b->d_nk, K)) || (rc = balloc(b, &b->tblk, K)) ||
        (rc = balloc(b, &b->kmin, K)) ||
        (rc = balloc(b, &b->kstart, K)) || (rc = balloc(b, &b->kcount, K)) || (rc = balloc(b, &b->ksplit, K)) ||
        (rc = balloc(b, &b->kni, K)) || (rc = balloc(b, &b->koff, K)) || (rc = balloc(b, &b->d_pk, K)) ||
        (rc = balloc(b, &b->chunk_cnt, (size_t)((slots + BCHUNK - 1) / BCHUNK))) ||
        (rc = balloc(b, &b->esum, 3 * (size_t)K))) {
        nb_batch_destroy(b);
        return rc;
    }
    if (cudaMallocHost(&b->h_tblk, K * sizeof(double)) || cudaMallocHost(&b->h_kstart, K * sizeof(int32_t)) ||
        cudaMallocHost(&b->h_kcount, K * sizeof(int32_t)) || cudaMallocHost(&b->h_ksplit, K * sizeof(int32_t)) ||
        cudaMallocHost(&b->h_esum, 3 * K * sizeof(double))) {
        cudaGetLastError();
        nb_batch_destroy(b);
        return NB_ERR_NOMEM;
    }
    std::vector<int32_t> cid((size_t)b->c->np, -1), real;
    real.reserve((size_t)b->n_real);
    for (int k = 0; k < K; ++k)
        for (int64_t i = 0; i < b->nk[k]; ++i) {
            cid[(size_t)(b->off[k] + i)] = k;
            real.push_back((int32_t)(b->off[k] + i));
        }
    if (cudaMemcpy(b->cid, cid.data(), cid.size() * 4, cudaMemcpyHostToDevice) ||
        cudaMemcpy(b->real_idx, real.data(), real.size() * 4, cudaMemcpyHostToDevice) ||
        cudaMemcpy(b->d_off, b->off.data(), K * 8, cudaMemcpyHostToDevice) ||
        cudaMemcpy(b->d_nk, b->nk.data(), K * 8, cudaMemcpyHostToDevice) ||
        cudaMemcpy(b->d_pk, b->pk.data(), K * 8, cudaMemcpyHostToDevice) ||
        cudaMemset(b->kmin, 0xFF, K * sizeof(unsigned long long))) {
        cudaGetLastError();
        nb_batch_destroy(b);
        return NB_ERR_CUDA;
    }
    b->c->pair_eps = 1;
    *out = b;
    return NB_OK;
}

int nb_batch_set_stream(nb_batch* b, void* stream) { return b ? nb_set_stream(b->c, stream) : NB_ERR_ARG; }

int nb_batch_set_precision(nb_batch* b, int mode)
{
    if (!b) return NB_ERR_ARG;
    batch_destroy_graph(b);
    return nb_set_precision(b->c, mode);
}

int nb_batch_set_params(nb_batch* b, double eta, double eta_s, double dt_max, double dt_min)
{
    if (!b) return NB_ERR_ARG;
    batch_destroy_graph(b);
    int rc = nb_set_params(b->c, eta, eta_s, dt_max, dt_min);
    if (rc != NB_OK) berr(b, rc, "%s", nb_last_error(b->c));
    return rc;
}

int nb_batch_set_particles(nb_batch* b, const double* m, const double* x, const double* v)
{
    if (!b || !m || !x || !v) return NB_ERR_ARG;
    nb_ctx* c = b->c;
    batch_destroy_graph(b);
    const size_t np = (size_t)c->np;
    std::vector<double> hm(np, 0.0), he(np, 1.0), hx(3 * np, 0.0), hv(3 * np, 0.0), ht(np, INFINITY), hdt(np, 0.0);
    const double e2 = c->eps * c->eps;
    double e2max = 0.0;
    for (int k = 0; k < b->K; ++k)
        for (int64_t i = 0; i < b->nk[k]; ++i) {
            const size_t r = (size_t)(b->roff[k] + i), s = (size_t)(b->off[k] + i);
            if (!(m[r] >= 0.0) || !std::isfinite(m[r])) return berr(b, NB_ERR_ARG, "masses must be finite and >= 0");
            hm[s] = m[r];
            he[s] = e2;
            ht[s] = 0.0;
            for (int q = 0; q < 3; ++q) {
                if (!std::isfinite(x[3 * r + q]) || !std::isfinite(v[3 * r + q]))
                    return berr(b, NB_ERR_NAN, "non-finite position or velocity");
                hx[q * np + s] = x[3 * r + q];
                hv[q * np + s] = v[3 * r + q];
            }
            e2max = std::max(e2max, e2);
        }
    B_CUDA(b, cudaMemcpyAsync(c->m, hm.data(), np * 8, cudaMemcpyHostToDevice, c->stream));
    B_CUDA(b, cudaMemcpyAsync(c->eps2, he.data(), np * 8, cudaMemcpyHostToDevice, c->stream));
    B_CUDA(b, cudaMemcpyAsync(c->x, hx.data(), 3 * np * 8, cudaMemcpyHostToDevice, c->stream));
    B_CUDA(b, cudaMemcpyAsync(c->v, hv.data(), 3 * np * 8, cudaMemcpyHostToDevice, c->stream));
    B_CUDA(b, cudaMemcpyAsync(c->t, ht.data(), np * 8, cudaMemcpyHostToDevice, c->stream));
    B_CUDA(b, cudaMemcpyAsync(c->dt, hdt.data(), np * 8, cudaMemcpyHostToDevice, c->stream));
    B_CUDA(b, cudaMemsetAsync(c->d, 0, 18 * np * 8, c->stream));
    B_CUDA(b, cudaMemsetAsync(c->pot, 0, np * 8, c->stream));
    B_CUDA(b, cudaMemsetAsync(b->tblk, 0, b->K * sizeof(double), c->stream));
    B_CUDA(b, cudaMemsetAsync(&c->sc->status, 0, sizeof(int), c->stream));
    B_CUDA(b, cudaStreamSynchronize(c->stream));
    c->eps2_max = e2max;
    c->have_particles = 1;
    // start-up passes on every real particle (each cluster against itself)
    std::vector<int32_t> hs(b->K), hc(b->K);
    for (int k = 0; k < b->K; ++k) {
        hs[k] = (int32_t)b->roff[k];
        hc[k] = (int32_t)b->nk[k];
    }
    const int nr = (int)b->n_real, g = (nr + 255) / 256;
    for (int pass = 4; pass <= c->order; pass += 2) {
        B_CUDA(b, launch_predict(c, 0.0, b->tblk, b->cid));
        c->pred_prec = c->prec;
        c->n_launch += 1;
        B_TRY(batch_force(b, pass, b->real_idx, nr, hs.data(), hc.data()));
        if (pass == 4) k_batch_startup_store<4><<<g, 256, 0, c->stream>>>(c->F, b->real_idx, nr, c->np, c->d, c->pot);
        else if (pass == 6) k_batch_startup_store<6><<<g, 256, 0, c->stream>>>(c->F, b->real_idx, nr, c->np, c->d, c->pot);
        else k_batch_startup_store<8><<<g, 256, 0, c->stream>>>(c->F, b->real_idx, nr, c->np, c->d, c->pot);
    }
    k_batch_startup_dt<<<g, 256, 0, c->stream>>>(c->d, b->real_idx, nr, c->np, c->t, c->dt, c->eta_s, c->dt_max,
                                                 c->dt_min, c->sc);
    B_CUDA(b, cudaGetLastError());
    return bsync(b);
}

int nb_batch_set_waves(nb_batch* b, int waves)
{
    if (!b) return NB_ERR_ARG;
    if (waves < 1 || waves > BATCH_WAVES_MAX) return berr(b, NB_ERR_ARG, "waves must be in [1, %d]", BATCH_WAVES_MAX);
    if (waves != b->waves) batch_destroy_graph(b);
    b->waves = waves;
    return NB_OK;
}

int nb_batch_get_waves(nb_batch* b, int* waves)
{
    if (!b || !waves) return NB_ERR_ARG;
    *waves = b->waves;
    return NB_OK;
}

int nb_batch_autotune(nb_batch* b, int cycles, int reps, double* ms_per_wave)
{
    if (!b) return NB_ERR_ARG;
    nb_ctx* c = b->c;
    if (!c->have_particles) return berr(b, NB_ERR_ARG, "nb_batch_autotune before nb_batch_set_particles");
    if (cycles < 1 || reps < 1) return berr(b, NB_ERR_ARG, "cycles and reps must be >= 1");
    B_TRY(batch_prepare(b));
    B_TRY(batch_reset_scalars(b, INFINITY, c->stream));
    cudaEvent_t e0, e1;
    B_CUDA(b, cudaEventCreate(&e0));
    B_CUDA(b, cudaEventCreate(&e1));
    double total[BATCH_WAVES_MAX + 1] = {0};
    int rc = NB_OK;
    for (int cyc = 0; cyc < cycles && rc == NB_OK; ++cyc) {
        cudaError_t e = batch_cycle_front(b);
        if (e == cudaSuccess) e = launch_predict(c, 0.0, b->tblk, b->cid, c->sc);
        // each candidate: its plan, then its force and reduction, best of reps
        for (int w = 1; w <= BATCH_WAVES_MAX && e == cudaSuccess; w *= 2) {
            if ((e = batch_cycle_plan(b, w)) != cudaSuccess) break;
            float best = INFINITY;
            for (int r = 0; r < reps && e == cudaSuccess; ++r) {
                // the force hands out items from a counter the plan reset
                if ((e = cudaMemsetAsync(&c->sc->next_item, 0, sizeof(int), c->stream)) != cudaSuccess) break;
                cudaEventRecord(e0, c->stream);
                if ((e = batch_cycle_force(b)) != cudaSuccess) break;
                cudaEventRecord(e1, c->stream);
                if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                best = std::min(best, ms);
            }
            total[w] += best;
        }
        // the cycle itself, with the wave count in use
        if (e == cudaSuccess) e = batch_cycle_plan(b, b->waves);
        if (e == cudaSuccess) e = cudaMemsetAsync(&c->sc->next_item, 0, sizeof(int), c->stream);
        if (e == cudaSuccess) e = batch_cycle_force(b);
        if (e == cudaSuccess) e = launch_correct(c, b->tblk, b->cid, c->sc);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = berr(b, NB_ERR_CUDA, "autotune cycle failed: %s", cudaGetErrorString(e));
            break;
        }
        rc = bsync(b);
        if (rc == NB_OK && c->h_sc->idle) break;  // every cluster at t = +inf: cannot happen before t_end
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    B_TRY(rc);
    int w_min = 4;
    for (int w = 1; w <= BATCH_WAVES_MAX; w *= 2)
        if (total[w] < total[w_min]) w_min = w;
    const int best_w = total[w_min] < BATCH_TUNE_MARGIN * total[4] ? w_min : 4;
    if (ms_per_wave)
        for (int k = 0, w = 1; w <= BATCH_WAVES_MAX; ++k, w *= 2) ms_per_wave[k] = total[w];
    return nb_batch_set_waves(b, best_w);
}

int nb_batch_cycle(nb_batch* b, double t_end, int* n_stepped, int64_t* n_inter)
{
    if (!b) return NB_ERR_ARG;
    nb_ctx* c = b->c;
    if (!c->have_particles) return berr(b, NB_ERR_ARG, "nb_batch_cycle before nb_batch_set_particles");
    if (!std::isfinite(t_end)) return berr(b, NB_ERR_ARG, "t_end must be finite");
    B_TRY(batch_prepare(b));
    B_TRY(batch_reset_scalars(b, t_end, c->stream));
    B_CUDA(b, batch_cycle_launches(b));
    B_TRY(bsync(b));
    if (n_stepped) *n_stepped = c->h_sc->stepped;
    if (n_inter) *n_inter = c->h_sc->inter;
    return NB_OK;
}

int nb_batch_set_graph(nb_batch* b, int cycles)
{
    if (!b) return NB_ERR_ARG;
    if (cycles < 0 || cycles > 4096) return berr(b, NB_ERR_ARG, "cycles must be in [0, 4096]");
    batch_destroy_graph(b);
    b->graph_cycles = cycles;
    return NB_OK;
}

int nb_batch_step_until(nb_batch* b, double t_end, int64_t* n_cycles, int64_t* n_inter)
{
    if (!b) return NB_ERR_ARG;
    nb_ctx* c = b->c;
    if (!c->have_particles) return berr(b, NB_ERR_ARG, "nb_batch_step_until before nb_batch_set_particles");
    if (!std::isfinite(t_end)) return berr(b, NB_ERR_ARG, "t_end must be finite");
    int64_t cycles = 0, inter = 0;
    if (b->graph_cycles > 0) {
        B_TRY(batch_prepare(b));
        if (!b->graph_exec) B_TRY(batch_build_graph(b));
        B_CUDA(b, cudaStreamSynchronize(c->stream));
        B_TRY(batch_reset_scalars(b, t_end, b->graph_stream));
        DevScalars* h = c->h_sc;
        for (;;) {
            B_CUDA(b, cudaGraphLaunch(b->graph_exec, b->graph_stream));
            c->n_launch += (int64_t)b->graph_cycles * BATCH_CYCLE_LAUNCHES;
            B_CUDA(b, cudaMemcpyAsync(h, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, b->graph_stream));
            B_CUDA(b, cudaStreamSynchronize(b->graph_stream));
            if (h->status != NB_OK) {
                const int st = h->status;
                B_CUDA(b, cudaMemsetAsync(&c->sc->status, 0, sizeof(int), b->graph_stream));
                B_CUDA(b, cudaStreamSynchronize(b->graph_stream));
                return berr(b, st, "device kernel reported error %d", st);
            }
            if (h->idle) break;
        }
        cycles = h->blocks;
        inter = h->inter;
    } else {
        for (;;) {
            int stepped = 0;
            int64_t ni = 0;
            B_TRY(nb_batch_cycle(b, t_end, &stepped, &ni));
            if (stepped == 0) break;
            ++cycles;
            inter += ni;
        }
    }
    if (n_cycles) *n_cycles = cycles;
    if (n_inter) *n_inter = inter;
    return bsync(b);
}

int nb_batch_energy(nb_batch* b, double* ekin, double* epot)
{
    if (!b) return NB_ERR_ARG;
    nb_ctx* c = b->c;
    const int K = b->K, nr = (int)b->n_real;
    int64_t* d_roff = nullptr;
    B_TRY(balloc(b, &d_roff, K));
    cudaMemcpyAsync(d_roff, b->roff.data(), K * 8, cudaMemcpyHostToDevice, c->stream);
    k_batch_first_time<<<(K + 255) / 256, 256, 0, c->stream>>>(c->t, b->d_off, K, b->tblk);
    B_CUDA(b, launch_predict(c, 0.0, b->tblk, b->cid));
    c->pred_prec = c->prec;
    std::vector<int32_t> hs(K), hc(K);
    for (int k = 0; k < K; ++k) {
        hs[k] = (int32_t)b->roff[k];
        hc[k] = (int32_t)b->nk[k];
    }
    int rc = batch_force(b, 0, b->real_idx, nr, hs.data(), hc.data());
    if (rc == NB_OK) {
        k_batch_energy<<<K, BNT, 0, c->stream>>>(c->m, c->v, c->t, c->F, b->real_idx, d_roff, b->d_nk, c->np, b->esum);
        cudaMemcpyAsync(b->h_esum, b->esum, 3 * K * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        rc = bsync(b);
    }
    cudaFree(d_roff);
    if (rc != NB_OK) return rc;
    for (int k = 0; k < K; ++k) {
        if (b->h_esum[3 * k + 2] != 0.0) return berr(b, NB_ERR_NOT_SYNC, "cluster %d not synchronised", k);
        if (ekin) ekin[k] = b->h_esum[3 * k];
        if (epot) epot[k] = b->h_esum[3 * k + 1];
    }
    return NB_OK;
}

int nb_batch_get_state(nb_batch* b, double* x, double* v, double* t, double* dt)
{
    if (!b) return NB_ERR_ARG;
    nb_ctx* c = b->c;
    B_TRY(bsync(b));
    const size_t np = (size_t)c->np;
    std::vector<double> hx(3 * np), hv(3 * np), ht(np), hdt(np);
    B_CUDA(b, cudaMemcpy(hx.data(), c->x, 3 * np * 8, cudaMemcpyDeviceToHost));
    B_CUDA(b, cudaMemcpy(hv.data(), c->v, 3 * np * 8, cudaMemcpyDeviceToHost));
    B_CUDA(b, cudaMemcpy(ht.data(), c->t, np * 8, cudaMemcpyDeviceToHost));
    B_CUDA(b, cudaMemcpy(hdt.data(), c->dt, np * 8, cudaMemcpyDeviceToHost));
    for (int k = 0; k < b->K; ++k)
        for (int64_t i = 0; i < b->nk[k]; ++i) {
            const size_t r = (size_t)(b->roff[k] + i), s = (size_t)(b->off[k] + i);
            for (int q = 0; q < 3; ++q) {
                if (x) x[3 * r + q] = hx[q * np + s];
                if (v) v[3 * r + q] = hv[q * np + s];
            }
            if (t) t[r] = ht[s];
            if (dt) dt[r] = hdt[s];
        }
    return NB_OK;
}

}  // extern "C"
