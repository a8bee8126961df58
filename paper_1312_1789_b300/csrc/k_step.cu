// k_step.cu -- the kernels around the force: block scheduler (K5), predictor
// (K1), Hermite corrector + time step (K4), start-up and energy support.
//
// All of them read and write the FP64 structure-of-arrays state and are bound
// by HBM bandwidth or by the (slow on this part) FP64 pipe, not by the FP32
// pipe the force kernel saturates.
#include <cmath>

#include "nb_internal.cuh"

namespace nb {

// ===================================================================== K5
// Block scheduler (abstract: individual hierarchical block time-steps):
// t_blk = min_i (t_i + dt_i), active = {i : t_i + dt_i == t_blk} ascending.
// Two passes, no atomics, deterministic.  Chunk b = SCHED_NT threads x PER
// consecutive particles each (PER from sched_layout, a power of two).
//   1. chunk b publishes m_b = its minimum of t_i + dt_i and c_b = how many of
//      its particles reach m_b;
//   2. every chunk reads the table: t_blk = min_b m_b, its offset = sum of c_b'
//      over earlier chunks with m_b' == t_blk; a chunk with m_b == t_blk
//      writes its matches in index order (one block-wide exclusive scan).
// Times are compared as order-preserving integer keys of the (exact, dyadic)
// sums t_i + dt_i: the only FP64 operation is the sum itself (the FP64 pipe
// runs at 1/64 of the FP32 rate here).  A NaN sum raises NB_ERR_NAN and is
// left out.
constexpr int SCHED_NT = 256;
constexpr int SCHED_PER_MAX = 16;
// The predictor takes two consecutive particles per thread (16-byte loads,
// twice the bytes in flight) on stores large enough that the scheduler
// gives each thread SCHED_PER_MAX particles (n > 8 SCHED_NT SMs); below
// that the grid has too few CTAs to fill the SMs twice over and one particle
// per thread is faster (measured at N = 65536: 28 against 33 us per block
// for scheduler and predictor; at 2^20 the two-particle form moves the
// predictor from 51 % to 64 % of the HBM bandwidth).
__host__ __device__ constexpr bool pred_two(int per) { return per >= SCHED_PER_MAX; }
constexpr unsigned long long KEY_NONE = ~0ull;

// k(a) < k(b) <=> a < b for non-NaN doubles; NaN -> KEY_NONE
__device__ __forceinline__ unsigned long long time_key(double x)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    if ((u & 0x7FFFFFFFFFFFFFFFull) > 0x7FF0000000000000ull) return KEY_NONE;
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double key_time(unsigned long long k)
{
    if (k == KEY_NONE) return INFINITY;
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k));
}

__device__ __forceinline__ double warp_min(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int warp_isum(int v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// minimum key over the CTA; every thread gets it
__device__ __forceinline__ unsigned long long block_kmin(unsigned long long v, unsigned long long* ws)
{
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, v, o);
        v = y < v ? y : v;
    }
    __syncthreads();  // ws reuse
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long b = ws[0];
    for (int w = 1; w < SCHED_NT / 32; ++w) b = ws[w] < b ? ws[w] : b;
    return b;
}

// sum over the CTA; every thread gets it
__device__ __forceinline__ int block_isum(int v, int* ws)
{
    v = warp_isum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    int s = 0;
    for (int w = 0; w < SCHED_NT / 32; ++w) s += ws[w];
    return s;
}

// exclusive scan over the CTA; every thread gets its prefix and the total
__device__ __forceinline__ int block_exscan(int v, int* ws, int* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    __syncthreads();  // ws reuse
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    int base = 0, all = 0;
    for (int w = 0; w < SCHED_NT / 32; ++w) {
        if (w < warp) base += ws[w];
        all += ws[w];
    }
    *total = all;
    return base + incl - v;
}

// First pass: chunk b publishes its minimum of t + dt and how many of its
// particles reach it.  The last CTA to finish (a ticket in the device
// scalars) then reduces the chunk table in chunk order: the block time's key
// (the minimum), the number of matches, and each chunk's offset in the
// active list, so that the second pass reads them instead of the table.
// The order of that reduction does not depend on which CTA is last.
template <int PER>
__global__ void __launch_bounds__(SCHED_NT) k_sched_chunk(const double* __restrict__ t, const double* __restrict__ dt,
                                                          int64_t n, unsigned long long* __restrict__ cmin,
                                                          int32_t* __restrict__ ccnt, int32_t* __restrict__ coff,
                                                          DevScalars* sc)
{
    pdl_wait();
    pdl_release();
    __shared__ unsigned long long wk[SCHED_NT / 32];
    __shared__ int wi[SCHED_NT / 32];
    __shared__ bool last;
    const int64_t i0 = ((int64_t)blockIdx.x * SCHED_NT + threadIdx.x) * PER;
    unsigned long long key[PER];
    unsigned long long mn = KEY_NONE;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        key[k] = KEY_NONE;
        if (i0 + k < n) {
            key[k] = time_key(t[i0 + k] + dt[i0 + k]);
            bad |= key[k] == KEY_NONE;
            mn = key[k] < mn ? key[k] : mn;
        }
    }
    if (bad) raise_status(sc, NB_ERR_NAN);
    const unsigned long long m_b = block_kmin(mn, wk);
    int c = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) c += (key[k] == m_b && m_b != KEY_NONE) ? 1 : 0;
    c = block_isum(c, wi);
    if (threadIdx.x == 0) {
        cmin[blockIdx.x] = m_b;
        ccnt[blockIdx.x] = c;
        __threadfence();  // the table entry is visible before the ticket is taken
        last = atomicAdd(&sc->sched_ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int nch = (int)gridDim.x;
    unsigned long long tm = KEY_NONE;
    for (int k = threadIdx.x; k < nch; k += SCHED_NT) {
        const unsigned long long v = __ldcg(cmin + k);
        tm = v < tm ? v : tm;
    }
    const unsigned long long tbk = block_kmin(tm, wk);
    // chunks [k0, k1) per thread, in order
    const int seg = (nch + SCHED_NT - 1) / SCHED_NT;
    const int k0 = min((int)threadIdx.x * seg, nch), k1 = min(k0 + seg, nch);
    int mine = 0;
    for (int k = k0; k < k1; ++k) mine += (__ldcg(cmin + k) == tbk && tbk != KEY_NONE) ? __ldcg(ccnt + k) : 0;
    int total;
    int off = block_exscan(mine, wi, &total);
    for (int k = k0; k < k1; ++k) {
        coff[k] = off;
        off += (__ldcg(cmin + k) == tbk && tbk != KEY_NONE) ? __ldcg(ccnt + k) : 0;
    }
    if (threadIdx.x == 0) {
        sc->tb_key = tbk;
        sc->n_match = total;
        sc->sched_ticket = 0;  // ready for the next block
    }
}

// Second pass (every CTA): t_blk, the match count and this chunk's offset as
// the first pass's last CTA left them, then the chunk's matches in index
// order.  CTA 0 publishes t_blk and n_act (and, in a device-driven cycle,
// applies the launch-shape gate).  Returns t_blk.
template <int PER>
__device__ __forceinline__ double sched_compact_body(const double* __restrict__ t, const double* __restrict__ dt,
                                                     int64_t n, const unsigned long long* __restrict__ cmin,
                                                     const int32_t* __restrict__ coff, int nch,
                                                     int32_t* __restrict__ idx, DevScalars* sc,
                                                     const GateArgs* gate = nullptr)
{
    __shared__ int wi[SCHED_NT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long tbk = sc->tb_key;
    const double tb = key_time(tbk);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int total = sc->n_match;
        sc->t_blk = tb;
        sc->n_act = total;
        if (gate) cycle_gate_apply(sc, tb, total, *gate);
    }
    if (cmin[blockIdx.x] != tbk || tbk == KEY_NONE) return tb;  // CTA-uniform: no match in this chunk
    const int off = coff[blockIdx.x];
    const int64_t i0 = ((int64_t)blockIdx.x * SCHED_NT + threadIdx.x) * PER;
    unsigned flags = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k)
        if (i0 + k < n && time_key(t[i0 + k] + dt[i0 + k]) == tbk) flags |= 1u << k;
    // exclusive scan of the per-thread match counts over the CTA
    const int mine = __popc(flags);
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wi[warp] = incl;
    __syncthreads();
    int wbase = 0;
    for (int w = 0; w < warp; ++w) wbase += wi[w];
    int pos = off + wbase + incl - mine;
    while (flags) {
        const int k = __ffs(flags) - 1;
        flags &= flags - 1;
        idx[pos++] = (int32_t)(i0 + k);
    }
    return tb;
}

template <int PER>
__global__ void __launch_bounds__(SCHED_NT) k_sched_compact(const double* __restrict__ t,
                                                            const double* __restrict__ dt, int64_t n,
                                                            const unsigned long long* __restrict__ cmin,
                                                            const int32_t* __restrict__ coff, int nch,
                                                            int32_t* __restrict__ idx, DevScalars* sc)
{
    sched_compact_body<PER>(t, dt, n, cmin, coff, nch, idx, sc);
}

// Particles per scheduler thread: the smallest power of two that covers n
// with one chunk per SM, at most SCHED_PER_MAX (more chunks beyond that).
void sched_layout(int64_t n, int sm_count, int* per, int* nch)
{
    const int64_t lanes = (int64_t)SCHED_NT * (sm_count > 0 ? sm_count : 1);
    int p = 1;
    while (p < SCHED_PER_MAX && (int64_t)p * lanes < n) p *= 2;
    *per = p;
    *nch = (int)((n + (int64_t)SCHED_NT * p - 1) / ((int64_t)SCHED_NT * p));
}

// dispatch on the layout's PER
#define NB_SCHED_PER(per, F) \
    switch (per) {           \
    case 1: F(1); break;     \
    case 2: F(2); break;     \
    case 4: F(4); break;     \
    case 8: F(8); break;     \
    default: F(16); break;   \
    }

cudaError_t launch_sched(nb_ctx* c)
{
    int per, nch;
    sched_layout(c->n, c->sm_count, &per, &nch);
#define NB_S(P)                                                                                                      \
    k_sched_chunk<P><<<nch, SCHED_NT, 0, c->stream>>>(c->t, c->dt, c->n, c->chunk_min, c->chunk_cnt,               \
                                                      c->chunk_off, c->sc);                                          \
    k_sched_compact<P><<<nch, SCHED_NT, 0, c->stream>>>(c->t, c->dt, c->n, c->chunk_min, c->chunk_off, nch,         \
                                                        c->act_idx, c->sc)
    NB_SCHED_PER(per, NB_S)
#undef NB_S
    return cudaGetLastError();
}


// ===================================================================== K1
// Predictor: Taylor series of every particle from t_i to tp.
//   orders 4, 6: x to the crackle term (dt^5), v to dt^4; order 6 also a to dt^3
//   order 8: x to a^(5) (dt^7), v to dt^6, a to dt^5, jerk to dt^4
// Writes the j-particle store in the requested precision; padding records
// (i >= n) get m = 0 and eps2 = 1 so they contribute exactly zero.
//
// FP64 store: every term in FP64.  Mixed store: x = x0 + h (v0 + h T) in FP64
// (then split into hi + lo floats), with the Taylor tail T = a/2 + h j/6 + ...
// and the predicted v, a, jerk evaluated in FP32, the precision they are
// stored in: the FP64 pipe (1/64 of the FP32 rate here) does only the
// position.  The tail's FP32 rounding is a few float ulps of its terms,
// scaled by h^2 -- far below the pair separations that need the
// double-single position.
// IEEE format conversions in integer arithmetic: the FP64 pipe, which runs
// f64 <-> f32 conversions here, is 1/64 of the FP32 rate.
// double -> float rounded toward zero; a result below the normal float range
// flushes to zero, one above it gives inf, NaN stays NaN.
__device__ __forceinline__ float f64_to_f32_rz(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7FF);
    const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
    if (e == 0x7FF) return __uint_as_float(sgn | 0x7F800000u | (mant ? 0x400000u : 0u));
    const int ef = e - 1023 + 127;
    if (ef >= 255) return __uint_as_float(sgn | 0x7F800000u);
    if (ef <= 0) return __uint_as_float(sgn);
    return __uint_as_float(sgn | ((unsigned)ef << 23) | (unsigned)(mant >> 29));
}

// float -> double, exact for every normal float (a subnormal one flushes to
// zero)
__device__ __forceinline__ double f32_to_f64(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
    const int e = (int)((u >> 23) & 0xFF);
    const unsigned long long mant = u & 0x7FFFFFu;
    if (e == 0xFF) return __longlong_as_double((long long)(sgn | 0x7FF0000000000000ull | (mant << 29)));
    if (e == 0) return __longlong_as_double((long long)sgn);
    return __longlong_as_double((long long)(sgn | ((unsigned long long)(e - 127 + 1023) << 52) | (mant << 29)));
}

// The same two conversions by the cvt instruction (on the FP64 pipe), the
// reference that nb_selftest_convert checks the integer forms against: round
// toward zero with subnormal results and inputs flushed, and |x| >= 2^128 --
// which the rounding mode would clamp to the largest float -- taken to inf as
// above, so both give the same bits for every non-NaN input.
__device__ __forceinline__ float f64_to_f32_rz_cvt(double x)
{
    float r;
    asm("cvt.rz.ftz.f32.f64 %0, %1;" : "=f"(r) : "d"(x));
    if (fabsf(r) == 0x1.fffffep127f && ((__double2hiint(x) >> 20) & 0x7FF) >= 1023 + 128)
        r = copysignf(INFINITY, r);
    return r;
}

__device__ __forceinline__ double f32_to_f64_cvt(float f)
{
    double r;
    asm("cvt.ftz.f64.f32 %0, %1;" : "=d"(r) : "f"(f));
    return r;
}

// The state a particle's prediction reads: x, v, the derivatives it holds
// (a, j, s, c; order 8 also a^(4), a^(5)), t, m, eps^2.
template <int ORDER>
struct PredIn {
    static constexpr int ND = ORDER == 8 ? 6 : 4;
    double x[3], v[3], d[ND][3];
    double t, m, e;
};

template <int ORDER>
__device__ __forceinline__ void pred_load(PredIn<ORDER>& s, int64_t i, const double* __restrict__ m,
                                          const double* __restrict__ eps2, const double* __restrict__ x,
                                          const double* __restrict__ v, const double* __restrict__ d,
                                          const double* __restrict__ t, int64_t np)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        s.x[c] = x[c * np + i];
        s.v[c] = v[c * np + i];
#pragma unroll
        for (int k = 0; k < PredIn<ORDER>::ND; ++k) s.d[k][c] = d[(k * 3 + c) * np + i];
    }
    s.t = t[i];
    s.m = m[i];
    s.e = eps2[i];
}

// Two consecutive particles i, i + 1 (i even: the SoA rows are 16-byte
// aligned) with one 16-byte load per array: half the load instructions and
// twice the bytes in flight per thread of the one-particle form.
template <int ORDER>
__device__ __forceinline__ void pred_load2(PredIn<ORDER>& s0, PredIn<ORDER>& s1, int64_t i,
                                           const double* __restrict__ m, const double* __restrict__ eps2,
                                           const double* __restrict__ x, const double* __restrict__ v,
                                           const double* __restrict__ d, const double* __restrict__ t, int64_t np)
{
    auto ld2 = [](const double* p) { return *reinterpret_cast<const double2*>(p); };
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double2 xx = ld2(x + c * np + i), vv = ld2(v + c * np + i);
        s0.x[c] = xx.x, s1.x[c] = xx.y;
        s0.v[c] = vv.x, s1.v[c] = vv.y;
#pragma unroll
        for (int k = 0; k < PredIn<ORDER>::ND; ++k) {
            const double2 dd = ld2(d + (k * 3 + c) * np + i);
            s0.d[k][c] = dd.x, s1.d[k][c] = dd.y;
        }
    }
    const double2 tt = ld2(t + i), mm = ld2(m + i), ee = ld2(eps2 + i);
    s0.t = tt.x, s1.t = tt.y;
    s0.m = mm.x, s1.m = mm.y;
    s0.e = ee.x, s1.e = ee.y;
}

// Prediction of one particle from its loaded state to tp, written as record i
// of the j-particle store; real = false writes a padding record (m = 0,
// eps2 = 1).
template <int ORDER, bool MIXED>
__device__ __forceinline__ void pred_store(const PredIn<ORDER>& s, bool real, double tp, int64_t i,
                                           void* __restrict__ jstore)
{
    constexpr int RW = MIXED ? mixed_rw(ORDER) : fp64_rw(ORDER);
    double xp[3] = {0, 0, 0}, vp[3] = {0, 0, 0}, ap[3] = {0, 0, 0}, jp[3] = {0, 0, 0};
    float vf[3] = {0.f, 0.f, 0.f}, af[3] = {0.f, 0.f, 0.f}, jf[3] = {0.f, 0.f, 0.f};
    double mi = 0.0, ei = 1.0;
    if (real) {
        mi = s.m;
        ei = s.e;
        const double h = tp - s.t;
        const float hf = MIXED ? f64_to_f32_rz(h) : 0.0f;
        // Mixed: the FP32 tail needs every derivative within the float range
        // (interpolated high derivatives of a particle just out of a close
        // encounter can exceed it); such a particle takes the FP64 series.
        bool fp64_series = !MIXED;
        if (MIXED) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double x0 = s.x[c], v0 = s.v[c];
                const float a0 = f64_to_f32_rz(s.d[0][c]), j0 = f64_to_f32_rz(s.d[1][c]);
                const float s0 = f64_to_f32_rz(s.d[2][c]), c0 = f64_to_f32_rz(s.d[3][c]);
                float T;
                bool fin = isfinite(a0) && isfinite(j0) && isfinite(s0) && isfinite(c0);
                if (ORDER == 8) {
                    const float d4 = f64_to_f32_rz(s.d[4 % PredIn<ORDER>::ND][c]);
                    const float d5 = f64_to_f32_rz(s.d[5 % PredIn<ORDER>::ND][c]);
                    fin = fin && isfinite(d4) && isfinite(d5);
                    T = fmaf(hf, fmaf(hf, fmaf(hf, fmaf(hf, fmaf(hf, d5 * (1.f / 5040), d4 * (1.f / 720)),
                                                         c0 * (1.f / 120)), s0 * (1.f / 24)), j0 * (1.f / 6)),
                             a0 * 0.5f);
                    vf[c] = fmaf(hf, fmaf(hf, fmaf(hf, fmaf(hf, fmaf(hf, fmaf(hf, d5 * (1.f / 720), d4 * (1.f / 120)),
                                                                     c0 * (1.f / 24)), s0 * (1.f / 6)), j0 * 0.5f), a0),
                                 f64_to_f32_rz(v0));
                    af[c] = fmaf(hf, fmaf(hf, fmaf(hf, fmaf(hf, fmaf(hf, d5 * (1.f / 120), d4 * (1.f / 24)),
                                                           c0 * (1.f / 6)), s0 * 0.5f), j0), a0);
                    jf[c] = fmaf(hf, fmaf(hf, fmaf(hf, fmaf(hf, d5 * (1.f / 24), d4 * (1.f / 6)), c0 * 0.5f), s0), j0);
                } else {
                    T = fmaf(hf, fmaf(hf, fmaf(hf, c0 * (1.f / 120), s0 * (1.f / 24)), j0 * (1.f / 6)), a0 * 0.5f);
                    vf[c] = fmaf(hf, fmaf(hf, fmaf(hf, fmaf(hf, c0 * (1.f / 24), s0 * (1.f / 6)), j0 * 0.5f), a0),
                                 f64_to_f32_rz(v0));
                    af[c] = fmaf(hf, fmaf(hf, fmaf(hf, c0 * (1.f / 6), s0 * 0.5f), j0), a0);
                }
                fin = fin && isfinite(T) && isfinite(vf[c]) && isfinite(af[c]) && isfinite(jf[c]);
                fp64_series = fp64_series || !fin;
                xp[c] = fma(h, fma(h, f32_to_f64(T), v0), x0);
            }
        }
        if (fp64_series) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double x0 = s.x[c], v0 = s.v[c];
                const double a0 = s.d[0][c], j0 = s.d[1][c];
                const double s0 = s.d[2][c], c0 = s.d[3][c];
                if (ORDER == 8) {
                    const double d4 = s.d[4 % PredIn<ORDER>::ND][c], d5 = s.d[5 % PredIn<ORDER>::ND][c];
                    xp[c] = x0 + h * (v0 + h * (a0 * (1.0 / 2) + h * (j0 * (1.0 / 6) + h * (s0 * (1.0 / 24) +
                            h * (c0 * (1.0 / 120) + h * (d4 * (1.0 / 720) + h * d5 * (1.0 / 5040)))))));
                    vp[c] = v0 + h * (a0 + h * (j0 * (1.0 / 2) + h * (s0 * (1.0 / 6) + h * (c0 * (1.0 / 24) +
                            h * (d4 * (1.0 / 120) + h * d5 * (1.0 / 720))))));
                    ap[c] = a0 + h * (j0 + h * (s0 * (1.0 / 2) + h * (c0 * (1.0 / 6) + h * (d4 * (1.0 / 24) +
                            h * d5 * (1.0 / 120)))));
                    jp[c] = j0 + h * (s0 + h * (c0 * (1.0 / 2) + h * (d4 * (1.0 / 6) + h * d5 * (1.0 / 24))));
                } else {
                    xp[c] = x0 + h * (v0 + h * (a0 * (1.0 / 2) + h * (j0 * (1.0 / 6) + h * (s0 * (1.0 / 24) +
                            h * c0 * (1.0 / 120)))));
                    vp[c] = v0 + h * (a0 + h * (j0 * (1.0 / 2) + h * (s0 * (1.0 / 6) + h * c0 * (1.0 / 24))));
                    ap[c] = a0 + h * (j0 + h * (s0 * (1.0 / 2) + h * c0 * (1.0 / 6)));
                }
                vf[c] = (float)vp[c];
                af[c] = (float)ap[c];
                jf[c] = (float)jp[c];
            }
        }
    }
    if (MIXED) {
        float4* r = reinterpret_cast<float4*>(jstore) + (size_t)i * RW;
        float hx[3], lx[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            // hi = the leading 24 bits (the double with its low 29 mantissa bits
            // cleared, exact in float), lo = the rest (exact in double, then
            // truncated to float): |hi + lo - x| <= 2^-47 |x|
            const double dhi = __longlong_as_double(__double_as_longlong(xp[c]) & ~0x1FFFFFFFLL);
            hx[c] = f64_to_f32_rz(dhi);
            lx[c] = f64_to_f32_rz(xp[c] - dhi);
        }
        r[0] = make_float4(hx[0], hx[1], hx[2], f64_to_f32_rz(mi));
        r[1] = make_float4(lx[0], lx[1], lx[2], f64_to_f32_rz(ei));
        r[2] = make_float4(vf[0], vf[1], vf[2], 0.f);
        if (ORDER >= 6) r[3] = make_float4(af[0], af[1], af[2], 0.f);
        if (ORDER >= 8) r[4] = make_float4(jf[0], jf[1], jf[2], 0.f);
    } else {
        double2* r = reinterpret_cast<double2*>(jstore) + (size_t)i * RW;
        r[0] = make_double2(xp[0], xp[1]);
        r[1] = make_double2(xp[2], mi);
        r[2] = make_double2(vp[0], vp[1]);
        r[3] = make_double2(vp[2], ei);
        if (ORDER >= 6) {
            r[4] = make_double2(ap[0], ap[1]);
            r[5] = make_double2(ap[2], 0.0);
        }
        if (ORDER >= 8) {
            r[6] = make_double2(jp[0], jp[1]);
            r[7] = make_double2(jp[2], 0.0);
        }
    }
}

template <int ORDER, bool MIXED>
__device__ __forceinline__ void predict_one(const int64_t i, double tp, const double* __restrict__ m,
                                            const double* __restrict__ eps2, const double* __restrict__ x,
                                            const double* __restrict__ v, const double* __restrict__ d,
                                            const double* __restrict__ t, int64_t n, int64_t np,
                                            void* __restrict__ jstore, const double* __restrict__ tpc,
                                            const int32_t* __restrict__ cid)
{
    bool real = i < n;
    if (real && tpc) {
        // ensemble: each particle to its own cluster's block time; cid < 0 marks
        // padding between clusters, an infinite time an idle cluster
        const int k = cid[i];
        if (k < 0) real = false;
        else {
            tp = tpc[k];
            if (!(tp < INFINITY)) return;
        }
    }
    PredIn<ORDER> s;
    if (real) pred_load<ORDER>(s, i, m, eps2, x, v, d, t, np);
    pred_store<ORDER, MIXED>(s, real, tp, i, jstore);
}

// Particles i and i + 1 of one system (i even, i + 1 < np).
template <int ORDER, bool MIXED>
__device__ __forceinline__ void predict_two(const int64_t i, double tp, const double* __restrict__ m,
                                            const double* __restrict__ eps2, const double* __restrict__ x,
                                            const double* __restrict__ v, const double* __restrict__ d,
                                            const double* __restrict__ t, int64_t n, int64_t np,
                                            void* __restrict__ jstore)
{
    PredIn<ORDER> s0, s1;
    pred_load2<ORDER>(s0, s1, i, m, eps2, x, v, d, t, np);
    pred_store<ORDER, MIXED>(s0, i < n, tp, i, jstore);
    pred_store<ORDER, MIXED>(s1, i + 1 < n, tp, i + 1, jstore);
}

// TWO: one system (tpc == nullptr), two consecutive particles per thread;
// else one particle per thread (ensembles).
template <int ORDER, bool MIXED, bool TWO>
__global__ void __launch_bounds__(256) k_predict(const double* __restrict__ m, const double* __restrict__ eps2,
                                                 const double* __restrict__ x, const double* __restrict__ v,
                                                 const double* __restrict__ d, const double* __restrict__ t,
                                                 int64_t n, int64_t np, double tp, void* __restrict__ jstore,
                                                 const double* __restrict__ tpc, const int32_t* __restrict__ cid,
                                                 const DevScalars* dyn)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = TWO ? 2 * g : g;
    if (i >= np) return;
    if (dyn) {
        if (dyn->idle) return;
        tp = dyn->t_blk;
    }
    if (TWO) predict_two<ORDER, MIXED>(i, tp, m, eps2, x, v, d, t, n, np, jstore);
    else predict_one<ORDER, MIXED>(i, tp, m, eps2, x, v, d, t, n, np, jstore, tpc, cid);
}

// Second pass fused with the predictor.  The grid has one CTA per chunk or
// per 2 SCHED_NT records, whichever is more: the first nch CTAs compact their
// chunks, the others only read the block time the first pass published; then
// every CTA predicts 2 SCHED_NT records to t_blk, two consecutive ones per
// thread with 16-byte loads (the predictor is bound by memory traffic, so it
// gets far more threads than the scheduler's PER particles each).
// use_t_end: a device-driven cycle, which predicts nothing past sc->t_end and
// whose force launch shape CTA 0 sets with the gate.
template <int ORDER, bool MIXED, int PER>
__global__ void __launch_bounds__(SCHED_NT) k_sched_compact_predict(
    const double* __restrict__ t, const double* __restrict__ dt, int64_t n,
    const unsigned long long* __restrict__ cmin, const int32_t* __restrict__ coff, int nch,
    int32_t* __restrict__ idx, DevScalars* sc, int use_t_end, const double* __restrict__ m,
    const double* __restrict__ eps2, const double* __restrict__ x, const double* __restrict__ v,
    const double* __restrict__ d, int64_t np, void* __restrict__ jstore, GateArgs gate)
{
    pdl_wait();
    pdl_release();
    const double tb = (int)blockIdx.x < nch
                          ? sched_compact_body<PER>(t, dt, n, cmin, coff, nch, idx, sc, use_t_end ? &gate : nullptr)
                          : key_time(sc->tb_key);
    if (use_t_end && !(tb <= sc->t_end)) return;
    const int64_t g = (int64_t)blockIdx.x * SCHED_NT + threadIdx.x;
    if (pred_two(PER)) {
        if (2 * g < np) predict_two<ORDER, MIXED>(2 * g, tb, m, eps2, x, v, d, t, n, np, jstore);
    } else if (g < np) {
        predict_one<ORDER, MIXED>(g, tb, m, eps2, x, v, d, t, n, np, jstore, nullptr, nullptr);
    }
}

// CTAs of the fused second pass: every chunk, and SCHED_NT or 2 SCHED_NT
// records per CTA
static int sched_predict_grid(int nch, int64_t np, int per)
{
    const int64_t rec = pred_two(per) ? 2 * SCHED_NT : SCHED_NT;
    const int64_t g = (np + rec - 1) / rec;
    return g > nch ? (int)g : nch;
}

cudaError_t launch_sched_predict(nb_ctx* c, bool use_t_end, const int* shape_slots)
{
    int per, nch;
    sched_layout(c->n, c->sm_count, &per, &nch);
    GateArgs g{};
    if (use_t_end) {
        const int pi = c->prec == NB_MIXED ? 1 : 0;
        g.n = c->n;
        g.cap = (long long)c->partial_cap;
        g.ntiles = (int)(c->np / JT);
        g.nc = ncomp(c->order);
        g.mixed = c->prec == NB_MIXED;
        g.js_force = c->jsplit_force;
        g.slots = shape_slots ? make_int4(shape_slots[0], shape_slots[1], shape_slots[2], shape_slots[3])
                              : make_int4(1, 1, 1, 1);
        g.tab = c->d_tune + pi * TUNE_MAX;
        g.ntab = c->tune_n[pi];
    }
    const bool mixed = c->prec == NB_MIXED, pdl = c->pdl != 0;
    const int gsp = sched_predict_grid(nch, c->np, per);
    cudaError_t e = cudaSuccess;
#define NB_SP(O, MX, P)                                                                                             \
    e = launch_k(k_sched_compact_predict<O, MX, P>, dim3(gsp), dim3(SCHED_NT), 0, c->stream, pdl, c->t, c->dt,     \
                 c->n, c->chunk_min, c->chunk_off, nch, c->act_idx, c->sc, use_t_end ? 1 : 0, c->m, c->eps2, c->x, \
                 c->v, c->d, c->np, c->jstore, g)
#define NB_S(P)                                                                                                     \
    e = launch_k(k_sched_chunk<P>, dim3(nch), dim3(SCHED_NT), 0, c->stream, pdl, c->t, c->dt, c->n, c->chunk_min,  \
                 c->chunk_cnt, c->chunk_off, c->sc);                                                                \
    if (e != cudaSuccess) return e;                                                                                 \
    if (c->order == 4) {                                                                                            \
        if (mixed) NB_SP(4, true, P); else NB_SP(4, false, P);                                                      \
    } else if (c->order == 6) {                                                                                     \
        if (mixed) NB_SP(6, true, P); else NB_SP(6, false, P);                                                      \
    } else {                                                                                                        \
        if (mixed) NB_SP(8, true, P); else NB_SP(8, false, P);                                                      \
    }
    NB_SCHED_PER(per, NB_S)
#undef NB_S
#undef NB_SP
    return e;
}

// Prediction of a rank's share of the j particles (records [r0, r1)) and of
// the block's active particles outside it (list[0..nl)): what a j-restricted
// force reads.  Threads [0, r1 - r0) take the range, the next nl the list.
template <int ORDER, bool MIXED>
__global__ void __launch_bounds__(256) k_predict_ranged(const double* __restrict__ m,
                                                        const double* __restrict__ eps2,
                                                        const double* __restrict__ x, const double* __restrict__ v,
                                                        const double* __restrict__ d, const double* __restrict__ t,
                                                        int64_t n, int64_t np, double tp, void* __restrict__ jstore,
                                                        int64_t r0, int64_t r1, const int32_t* __restrict__ list,
                                                        int64_t nl)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i;
    if (g < r1 - r0) {
        i = r0 + g;
    } else if (g < r1 - r0 + nl) {
        i = list[g - (r1 - r0)];
        if ((uint64_t)i >= (uint64_t)n || (i >= r0 && i < r1)) return;  // in the range: predicted above
    } else {
        return;
    }
    predict_one<ORDER, MIXED>(i, tp, m, eps2, x, v, d, t, n, np, jstore, nullptr, nullptr);
}

cudaError_t launch_predict_ranged(nb_ctx* c, double t, int64_t r0, int64_t r1, const int32_t* list, int64_t nl)
{
    const int nt = 256;
    const int64_t work = (r1 - r0) + nl;
    if (work <= 0) return cudaSuccess;
    const int nb = (int)((work + nt - 1) / nt);
    const bool mixed = c->prec == NB_MIXED;
#define NB_PR(O, MX)                                                                                                 k_predict_ranged<O, MX><<<nb, nt, 0, c->stream>>>(c->m, c->eps2, c->x, c->v, c->d, c->t, c->n, c->np, t,                                                           c->jstore, r0, r1, list, nl)
    if (c->order == 4) {
        if (mixed) NB_PR(4, true); else NB_PR(4, false);
    } else if (c->order == 6) {
        if (mixed) NB_PR(6, true); else NB_PR(6, false);
    } else {
        if (mixed) NB_PR(8, true); else NB_PR(8, false);
    }
#undef NB_PR
    return cudaGetLastError();
}

cudaError_t launch_predict(nb_ctx* c, double t, const double* tpc, const int32_t* cid, const DevScalars* dyn)
{
    const int nt = 256;
    int per, nch;
    sched_layout(c->n, c->sm_count, &per, &nch);
    const bool two = tpc == nullptr && pred_two(per);  // one large system: two particles per thread
    const int64_t per_cta = two ? 2 * nt : nt;
    const int nb = (int)((c->np + per_cta - 1) / per_cta);
    const bool mixed = c->prec == NB_MIXED;
#define NB_PRED_K(O, MX)                                                                                      \
    if (two)                                                                                                  \
        k_predict<O, MX, true><<<nb, nt, 0, c->stream>>>(c->m, c->eps2, c->x, c->v, c->d, c->t, c->n, c->np, \
                                                         t, c->jstore, tpc, cid, dyn);                        \
    else                                                                                                      \
        k_predict<O, MX, false><<<nb, nt, 0, c->stream>>>(c->m, c->eps2, c->x, c->v, c->d, c->t, c->n,       \
                                                          c->np, t, c->jstore, tpc, cid, dyn);
#define NB_PRED(O)            \
    if (mixed) {              \
        NB_PRED_K(O, true)    \
    } else {                  \
        NB_PRED_K(O, false)   \
    }
    if (c->order == 4) {
        NB_PRED(4)
    } else if (c->order == 6) {
        NB_PRED(6)
    } else {
        NB_PRED(8)
    }
#undef NB_PRED
#undef NB_PRED_K
    return cudaGetLastError();
}

// ===================================================================== K4
// 2^j, the largest power of two that divides the dyadic t1 exactly: a normal
// t1 is mant * 2^(e - 1075) with an integer 53-bit mant, so j = e - 1075 +
// (trailing zeros of mant).  +inf for t1 == 0 (every step divides it).
__device__ __forceinline__ double pow2_dividing(double t1)
{
    const long long b = __double_as_longlong(t1);
    const int e = (int)((b >> 52) & 0x7FF);
    const long long mant = (b & 0xFFFFFFFFFFFFFLL) | (e ? (1LL << 52) : 0LL);
    if (mant == 0) return INFINITY;
    const int j = (e ? e : 1) - 1075 + (__ffsll(mant) - 1);
    if (j > 1023) return INFINITY;
    if (j < -1022) return 0.0;
    return __longlong_as_double((long long)(j + 1023) << 52);
}

// 1/h; exact bit arithmetic when h is a power of two (the usual case: an
// active particle's h is its own step), else a division (same result).
__device__ __forceinline__ double recip(double h)
{
    const long long b = __double_as_longlong(h);
    const int e = (int)((b >> 52) & 0x7FF);
    if ((b & 0xFFFFFFFFFFFFFLL) == 0 && e > 1 && e < 2045)
        return __longlong_as_double((b & (long long)0x8000000000000000ULL) | ((long long)(2046 - e) << 52));
    return 1.0 / h;
}

// Quantised block step: the largest power of two <= min(lim, dt_max) that
// divides t1 (all block times are dyadic, so divisibility is exact): the
// mantissa-cleared lim, capped by the largest power of two dividing t1.
__device__ double quantise_dt(double lim, double t1, double dt_max, double dt_min, DevScalars* sc)
{
    if (!(lim == lim)) {
        raise_status(sc, NB_ERR_NAN);
        return dt_max;
    }
    double dt;
    if (lim >= dt_max) {
        dt = dt_max;
    } else if (lim < dt_min) {
        raise_status(sc, NB_ERR_DT_UNDERFLOW);
        return dt_min;
    } else {
        // clear the mantissa: 2^floor(log2(lim)) for a positive normal double
        dt = __longlong_as_double(__double_as_longlong(lim) & 0xFFF0000000000000LL);
    }
    dt = fmin(dt, pow2_dividing(t1));
    if (dt < dt_min) {
        raise_status(sc, NB_ERR_DT_UNDERFLOW);
        return dt_min;
    }
    return dt;
}

__device__ __forceinline__ double norm3(const double* p) { return sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]); }

// Generalised Aarseth criterion from the norms n[k] = |a^(k)| at t1:
//   p = 4: sqrt(eta (|a||a2| + |a1|^2) / (|a1||a3| + |a2|^2))
//   p = 6, 8: eta ((sqrt(|a||a2|) + |a1|) / (sqrt(|a(p-3)||a(p-1)|) + |a(p-2)|))^(1/(p-3))
template <int ORDER>
__device__ double dt_criterion(double eta, const double* nrm)
{
    const double n0 = nrm[0], n1 = nrm[1], n2 = nrm[2];
    if (ORDER == 4) {
        const double n3 = nrm[3];
        const double num = n0 * n2 + n1 * n1, den = n1 * n3 + n2 * n2;
        if (!(den > 0.0)) return INFINITY;
        return sqrt(eta * num / den);
    }
    const double nlo = nrm[ORDER - 3], nmid = nrm[ORDER - 2], nhi = nrm[ORDER - 1];
    const double num = sqrt(n0 * n2) + n1, den = sqrt(nlo * nhi) + nmid;
    if (!(den > 0.0)) return INFINITY;
    return ORDER == 6 ? eta * cbrt(num / den) : eta * pow(num / den, 0.2);
}

// Noise floor of the interpolated derivatives.  The closed forms below take
// differences of force values whose relative precision is ea (acc), ej
// (jerk), es (snap), ec (crackle) -- already multiplied by the particle's
// conditioning kappa = sum_j m_j/R_ij^2 / |a| -- and a derivative k carries at most
// N_k = sum |coefficient| * eps * |input| / h^k of that rounding.  The
// criterion uses max(|a^(k)| - N_k, 0): what the inputs cannot resolve is
// treated as unknown (zero) rather than as signal.  With all eps = 0 the
// criterion is the plain one.  nL[r], nR[r] = |a^(r)| at t0 and t1.
template <int ORDER>
__device__ void noise_floor(const double* nL, const double* nR, double h, double ih, const double* e, double* N)
{
    const double A = e[0] * (nL[0] + nR[0]);
    if (ORDER == 4) {
        N[2] = 2.0 * (3.0 * A + h * e[1] * (nL[1] + 2.0 * nR[1])) * ih * ih;
        N[3] = 6.0 * (2.0 * A + h * e[1] * (nL[1] + nR[1])) * ih * ih * ih;
    } else if (ORDER == 6) {
        const double h2 = h * h, ih3 = ih * ih * ih;
        N[3] = 3.0 * (20.0 * A + h2 * e[2] * (nL[2] + 3.0 * nR[2]) + 4.0 * h * e[1] * (2.0 * nL[1] + 3.0 * nR[1])) * ih3;
        N[4] = 12.0 * (30.0 * A + h2 * e[2] * (2.0 * nL[2] + 3.0 * nR[2]) + 2.0 * h * e[1] * (7.0 * nL[1] + 8.0 * nR[1])) *
               ih3 * ih;
        N[5] = 60.0 * (12.0 * A + h2 * e[2] * (nL[2] + nR[2]) + 6.0 * h * e[1] * (nL[1] + nR[1])) * ih3 * ih * ih;
    } else {
        const double h2 = h * h, h3 = h2 * h, ih4 = (ih * ih) * (ih * ih);
        N[4] = 4.0 * (210.0 * A + h3 * e[3] * (nL[3] + 4.0 * nR[3]) + 15.0 * h2 * e[2] * (nL[2] + 2.0 * nR[2]) +
                      30.0 * h * e[1] * (3.0 * nL[1] + 4.0 * nR[1])) * ih4;
        N[5] = 60.0 * (168.0 * A + h3 * e[3] * (nL[3] + 2.0 * nR[3]) + 2.0 * h2 * e[2] * (7.0 * nL[2] + 10.0 * nR[2]) +
                       6.0 * h * e[1] * (13.0 * nL[1] + 15.0 * nR[1])) * ih4 * ih;
        N[6] = 120.0 * (420.0 * A + h3 * e[3] * (3.0 * nL[3] + 4.0 * nR[3]) + 3.0 * h2 * e[2] * (13.0 * nL[2] + 15.0 * nR[2]) +
                        12.0 * h * e[1] * (17.0 * nL[1] + 18.0 * nR[1])) * ih4 * ih * ih;
        N[7] = 840.0 * (120.0 * A + h3 * e[3] * (nL[3] + nR[3]) + 12.0 * h2 * e[2] * (nL[2] + nR[2]) +
                        60.0 * h * e[1] * (nL[1] + nR[1])) * ih4 * ih * ih * ih;
    }
}

// FP64 corrector of one particle: the Hermite interpolant through
// L[0..mm-1] (acc derivatives at t0, held) and H[0..mm-1] (new ones at t1)
// gives H[mm..2mm-1] in closed form (derived symbolically); then the
// corrected x1, v1 and the step limit lim (criterion, capped at 2h).
// Returns false if a value is not finite.
template <int ORDER>
__device__ __forceinline__ bool correct_fp64(const double (&L)[4][3], double (&H)[8][3], const double h,
                                             const double ih, const double (&x0)[3], const double (&v0)[3],
                                             const double bacc, const double eta, const NoiseEps& ne,
                                             double (&x1)[3], double (&v1)[3], double& lim)
{
    constexpr int MM = ORDER / 2;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double L0 = L[0][c], L1 = L[1][c], L2 = L[2][c], L3 = L[3][c];
        const double R0 = H[0][c], R1 = H[1][c];
        if (ORDER == 4) {
            H[2][c] = 2.0 * (3.0 * (L0 - R0) + h * (L1 + 2.0 * R1)) * ih * ih;
            H[3][c] = 6.0 * (2.0 * (L0 - R0) + h * (L1 + R1)) * ih * ih * ih;
        } else if (ORDER == 6) {
            const double R2 = H[2][c];
            const double h2 = h * h;
            H[3][c] = 3.0 * (20.0 * (R0 - L0) + h2 * (3.0 * R2 - L2) - 4.0 * h * (2.0 * L1 + 3.0 * R1)) * ih * ih * ih;
            H[4][c] = 12.0 * (30.0 * (R0 - L0) + h2 * (3.0 * R2 - 2.0 * L2) - 2.0 * h * (7.0 * L1 + 8.0 * R1)) *
                      (ih * ih) * (ih * ih);
            H[5][c] = 60.0 * (12.0 * (R0 - L0) + h2 * (R2 - L2) - 6.0 * h * (L1 + R1)) * (ih * ih) * (ih * ih) * ih;
        } else {
            const double R2 = H[2][c], R3 = H[3][c];
            const double h2 = h * h, h3 = h2 * h;
            const double ih2 = ih * ih, ih4 = ih2 * ih2;
            H[4][c] = 4.0 * (210.0 * (L0 - R0) + h3 * (L3 + 4.0 * R3) + 15.0 * h2 * (L2 - 2.0 * R2) +
                             30.0 * h * (3.0 * L1 + 4.0 * R1)) * ih4;
            H[5][c] = 60.0 * (168.0 * (L0 - R0) + h3 * (L3 + 2.0 * R3) + 2.0 * h2 * (7.0 * L2 - 10.0 * R2) +
                              6.0 * h * (13.0 * L1 + 15.0 * R1)) * ih4 * ih;
            H[6][c] = 120.0 * (420.0 * (L0 - R0) + h3 * (3.0 * L3 + 4.0 * R3) + 3.0 * h2 * (13.0 * L2 - 15.0 * R2) +
                               12.0 * h * (17.0 * L1 + 18.0 * R1)) * ih4 * ih2;
            H[7][c] = 840.0 * (120.0 * (L0 - R0) + h3 * (L3 + R3) + 12.0 * h2 * (L2 - R2) + 60.0 * h * (L1 + R1)) *
                      ih4 * ih2 * ih;
        }
    }

    // two-point Hermite corrector of order p for v' = a, then x' = v
    bool finite_state = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double vi = v0[c], xi = x0[c];
        double vn, xn;
        if (ORDER == 4) {
            vn = vi + h * 0.5 * (L[0][c] + H[0][c]) - h * h * (1.0 / 12) * (H[1][c] - L[1][c]);
            xn = xi + h * 0.5 * (vi + vn) - h * h * (1.0 / 12) * (H[0][c] - L[0][c]);
        } else if (ORDER == 6) {
            vn = vi + h * 0.5 * (L[0][c] + H[0][c]) - h * h * 0.1 * (H[1][c] - L[1][c]) +
                 h * h * h * (1.0 / 120) * (L[2][c] + H[2][c]);
            xn = xi + h * 0.5 * (vi + vn) - h * h * 0.1 * (H[0][c] - L[0][c]) +
                 h * h * h * (1.0 / 120) * (L[1][c] + H[1][c]);
        } else {
            vn = vi + h * 0.5 * (L[0][c] + H[0][c]) - h * h * (3.0 / 28) * (H[1][c] - L[1][c]) +
                 h * h * h * (1.0 / 84) * (L[2][c] + H[2][c]) - h * h * h * h * (1.0 / 1680) * (H[3][c] - L[3][c]);
            xn = xi + h * 0.5 * (vi + vn) - h * h * (3.0 / 28) * (H[0][c] - L[0][c]) +
                 h * h * h * (1.0 / 84) * (L[1][c] + H[1][c]) - h * h * h * h * (1.0 / 1680) * (H[2][c] - L[2][c]);
        }
        v1[c] = vn;
        x1[c] = xn;
        finite_state = finite_state && fabs(vn) < INFINITY && fabs(xn) < INFINITY;
    }

    // derivative norms at t1, the interpolated ones net of their noise floor
    double nrm[8], nL[4], nR[4], N[8];
#pragma unroll
    for (int k = 0; k < 2 * MM; ++k) {
        nrm[k] = norm3(H[k]);
        finite_state = finite_state && nrm[k] < INFINITY;  // false for inf and NaN
    }
    // all-zero channel precisions (the FP64 default): the floor is zero and
    // the plain criterion applies -- skip its norms and polynomials
    if (ne.e[0] != 0.0 || ne.e[1] != 0.0 || ne.e[2] != 0.0 || ne.e[3] != 0.0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            nL[k] = norm3(L[k]);
            nR[k] = k < MM ? nrm[k] : 0.0;
        }
        // rounding of a total scales with the terms it sums: kappa = B / |a| >= 1
        const double kappa = nR[0] > 0.0 ? fmax(1.0, bacc / nR[0]) : 1.0;
        const double ek[4] = {ne.e[0] * kappa, ne.e[1] * kappa, ne.e[2] * kappa, ne.e[3] * kappa};
        noise_floor<ORDER>(nL, nR, h, ih, ek, N);
#pragma unroll
        for (int k = MM; k < 2 * MM; ++k) nrm[k] = fmax(nrm[k] - N[k], 0.0);
    }
    lim = dt_criterion<ORDER>(eta, nrm);
    if (2.0 * h < lim) lim = 2.0 * h;
    return finite_state;
}

// |(x, y, z)| in FP32; a sum of squares outside the normal float range is
// redone on the vector scaled by a power of two.
__device__ __forceinline__ float norm3f(const float (&p)[3])
{
    const float s = fmaf(p[0], p[0], fmaf(p[1], p[1], p[2] * p[2]));
    if (s < 0x1p126f && (s > 0x1p-126f || s == 0.0f)) return sqrtf(s);
    const float m = fmaxf(fabsf(p[0]), fmaxf(fabsf(p[1]), fabsf(p[2])));
    if (!(m < INFINITY) || m == 0.0f) return m;  // inf / NaN propagate, 0 stays 0
    // 2^-e with 2^e <= m < 2^(e+1), e within the normal range
    const int e = (int)((__float_as_uint(m) >> 23) & 0xFF) - 127;
    const float sc = __uint_as_float((unsigned)(127 - max(-126, min(e, 126))) << 23);
    const float a = p[0] * sc, b = p[1] * sc, c = p[2] * sc;
    return sqrtf(fmaf(a, a, fmaf(b, b, c * c))) / sc;
}

// Mixed-precision corrector (the mixed path, whose forces carry FP32-level
// rounding): x1 and v1 keep their leading terms x0 + h/2 (v0 + v1) and
// v0 + h/2 (a0 + a1) in FP64 and take the higher-order terms in FP32; the
// interpolated derivatives, their noise floor and the step criterion run in
// FP32 on h-scaled quantities a^(k) h^k (all of the size of the acceleration,
// so that neither 1/h^k nor a high derivative's own range leaves the float
// range) -- the same closed forms as correct_fp64 with h^k moved across, and
// the criterion's ratio, which is h^(p-3) times the ratio of scaled norms.
// The FP64 pipe (1/64 of the FP32 rate here) then does ~45 operations per
// particle instead of ~500; the format conversions run on the integer pipe
// (with cvt on the FP64 pipe a full block of 2^20 took 235 instead of 201 us,
// and small blocks in graph replays were no faster).  Returns false, with nothing usable written, if a
// float value is not finite (a derivative beyond the float range); the
// caller then takes correct_fp64.
template <int ORDER>
__device__ __forceinline__ bool correct_mixed(const double (&L)[4][3], double (&H)[8][3], const double h,
                                              const double ih, const double (&x0)[3], const double (&v0)[3],
                                              const double bacc, const double eta, const NoiseEps& ne,
                                              double (&x1)[3], double (&v1)[3], double& lim)
{
    constexpr int MM = ORDER / 2;
    const float u = f64_to_f32_rz(h);
    if (!(u > 0.0f)) return false;  // h below the float range
    // scaled inputs: ls[k] = L[k] h^k, rs[k] = H[k] h^k (k < MM), d0 = a1 - a0
    float ls[4][3], rs[4][3], d0[3];
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        d0[c] = f64_to_f32_rz(H[0][c] - L[0][c]);
        float uk = 1.0f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            ls[k][c] = f64_to_f32_rz(L[k][c]) * uk;
            rs[k][c] = k < MM ? f64_to_f32_rz(H[k][c]) * uk : 0.0f;
            ok = ok && isfinite(ls[k][c]) && isfinite(rs[k][c]);
            uk *= u;
        }
        ok = ok && isfinite(d0[c]);
    }
    if (!ok) return false;
    // T[k] = a^(k)(t1) h^k for k = MM .. 2MM-1 (closed forms as in correct_fp64)
    float T[8][3], tv[3], tx[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float D = d0[c];
        const float l1 = ls[1][c], r1 = rs[1][c], l2 = ls[2][c], r2 = rs[2][c], l3 = ls[3][c], r3 = rs[3][c];
        if (ORDER == 4) {
            T[2][c] = 2.0f * (-3.0f * D + (l1 + 2.0f * r1));
            T[3][c] = 6.0f * (-2.0f * D + (l1 + r1));
            tv[c] = -(1.0f / 12) * (r1 - l1);             // x h
            tx[c] = -(1.0f / 12) * D;                     // x h^2
        } else if (ORDER == 6) {
            T[3][c] = 3.0f * (20.0f * D + (3.0f * r2 - l2) - 4.0f * (2.0f * l1 + 3.0f * r1));
            T[4][c] = 12.0f * (30.0f * D + (3.0f * r2 - 2.0f * l2) - 2.0f * (7.0f * l1 + 8.0f * r1));
            T[5][c] = 60.0f * (12.0f * D + (r2 - l2) - 6.0f * (l1 + r1));
            tv[c] = -0.1f * (r1 - l1) + (1.0f / 120) * (l2 + r2);
            tx[c] = -0.1f * D + (1.0f / 120) * (l1 + r1);
        } else {
            T[4][c] = 4.0f * (-210.0f * D + (l3 + 4.0f * r3) + 15.0f * (l2 - 2.0f * r2) + 30.0f * (3.0f * l1 + 4.0f * r1));
            T[5][c] = 60.0f * (-168.0f * D + (l3 + 2.0f * r3) + 2.0f * (7.0f * l2 - 10.0f * r2) +
                               6.0f * (13.0f * l1 + 15.0f * r1));
            T[6][c] = 120.0f * (-420.0f * D + (3.0f * l3 + 4.0f * r3) + 3.0f * (13.0f * l2 - 15.0f * r2) +
                                12.0f * (17.0f * l1 + 18.0f * r1));
            T[7][c] = 840.0f * (-120.0f * D + (l3 + r3) + 12.0f * (l2 - r2) + 60.0f * (l1 + r1));
            tv[c] = -(3.0f / 28) * (r1 - l1) + (1.0f / 84) * (l2 + r2) - (1.0f / 1680) * (r3 - l3);
            tx[c] = -(3.0f / 28) * D + (1.0f / 84) * (l1 + r1) - (1.0f / 1680) * (r2 - l2);
        }
        tv[c] *= u;
        tx[c] *= u * u;
        ok = ok && isfinite(tv[c]) && isfinite(tx[c]);
#pragma unroll
        for (int k = MM; k < 2 * MM; ++k) ok = ok && isfinite(T[k][c]);
    }
    if (!ok) return false;
    // scaled norms at t1: S[k] = |a^(k)| h^k, the interpolated ones net of
    // their (scaled) noise floor
    float S[8];
#pragma unroll
    for (int k = 0; k < 2 * MM; ++k) {
        float q[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) q[c] = k < MM ? rs[k][c] : T[k][c];
        S[k] = norm3f(q);
    }
    if (ne.e[0] != 0.0 || ne.e[1] != 0.0 || ne.e[2] != 0.0 || ne.e[3] != 0.0) {
        float nl[4], nr[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            nl[k] = norm3f(ls[k]);
            nr[k] = k < MM ? S[k] : 0.0f;
        }
        const float kappa = nr[0] > 0.0f ? fmaxf(1.0f, f64_to_f32_rz(bacc) / nr[0]) : 1.0f;
        float e[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) e[k] = f64_to_f32_rz(ne.e[k]) * kappa;
        const float A = e[0] * (nl[0] + nr[0]);
        float N[8];
        if (ORDER == 4) {
            N[2] = 2.0f * (3.0f * A + e[1] * (nl[1] + 2.0f * nr[1]));
            N[3] = 6.0f * (2.0f * A + e[1] * (nl[1] + nr[1]));
        } else if (ORDER == 6) {
            N[3] = 3.0f * (20.0f * A + e[2] * (nl[2] + 3.0f * nr[2]) + 4.0f * e[1] * (2.0f * nl[1] + 3.0f * nr[1]));
            N[4] = 12.0f * (30.0f * A + e[2] * (2.0f * nl[2] + 3.0f * nr[2]) + 2.0f * e[1] * (7.0f * nl[1] + 8.0f * nr[1]));
            N[5] = 60.0f * (12.0f * A + e[2] * (nl[2] + nr[2]) + 6.0f * e[1] * (nl[1] + nr[1]));
        } else {
            N[4] = 4.0f * (210.0f * A + e[3] * (nl[3] + 4.0f * nr[3]) + 15.0f * e[2] * (nl[2] + 2.0f * nr[2]) +
                           30.0f * e[1] * (3.0f * nl[1] + 4.0f * nr[1]));
            N[5] = 60.0f * (168.0f * A + e[3] * (nl[3] + 2.0f * nr[3]) + 2.0f * e[2] * (7.0f * nl[2] + 10.0f * nr[2]) +
                            6.0f * e[1] * (13.0f * nl[1] + 15.0f * nr[1]));
            N[6] = 120.0f * (420.0f * A + e[3] * (3.0f * nl[3] + 4.0f * nr[3]) + 3.0f * e[2] * (13.0f * nl[2] + 15.0f * nr[2]) +
                             12.0f * e[1] * (17.0f * nl[1] + 18.0f * nr[1]));
            N[7] = 840.0f * (120.0f * A + e[3] * (nl[3] + nr[3]) + 12.0f * e[2] * (nl[2] + nr[2]) +
                             60.0f * e[1] * (nl[1] + nr[1]));
        }
#pragma unroll
        for (int k = MM; k < 2 * MM; ++k) S[k] = fmaxf(S[k] - N[k], 0.0f);
    }
    // the criterion as a multiple f of h, capped at 2 (the step may at most double)
    float f;
    {
        const float etaf = f64_to_f32_rz(eta);
        if (ORDER == 4) {
            const float num = S[0] * S[2] + S[1] * S[1], den = S[1] * S[3] + S[2] * S[2];
            f = den > 0.0f ? sqrtf(etaf * (num / den)) : INFINITY;
        } else {
            const float num = sqrtf(S[0]) * sqrtf(S[2]) + S[1];
            const float den = sqrtf(S[ORDER - 3]) * sqrtf(S[ORDER - 1]) + S[ORDER - 2];
            const float r = num / den;
            f = den > 0.0f ? etaf * (ORDER == 6 ? cbrtf(r) : exp2f(0.2f * log2f(r))) : INFINITY;
        }
        if (!(f <= 2.0f)) f = f == f ? 2.0f : f;  // inf -> 2; NaN stays
    }
    if (!(f == f)) return false;
    lim = h * f32_to_f64(f);
    // H[k] = T[k] / h^k, and the corrected state
    double ihk = 1.0;
#pragma unroll
    for (int k = 1; k < 2 * MM; ++k) {
        ihk *= ih;
        if (k >= MM)
#pragma unroll
            for (int c = 0; c < 3; ++c) H[k][c] = f32_to_f64(T[k][c]) * ihk;
    }
    const double hh = 0.5 * h;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        v1[c] = fma(hh, L[0][c] + H[0][c], v0[c]) + f32_to_f64(tv[c]);
        x1[c] = fma(hh, v0[c] + v1[c], x0[c]) + f32_to_f64(tx[c]);
    }
    return true;
}

// Corrector, interpolation and new step of the force list's particle p
// (MIXED: the mixed-precision form, FP64 for the particles it cannot take);
// component k of its force is Fp[k * fs].
template <int ORDER, bool MIXED>
__device__ __forceinline__ void correct_one(const int p, const int32_t* __restrict__ fidx, double tf,
                                            const double* Fp, const size_t fs, int64_t n, int64_t np,
                                            double* __restrict__ x, double* __restrict__ v, double* __restrict__ d,
                                            double* __restrict__ t, double* __restrict__ dtv,
                                            double* __restrict__ pot, double eta, double dt_max, double dt_min,
                                            const NoiseEps& ne, DevScalars* sc, const double* __restrict__ tfc,
                                            const int32_t* __restrict__ cid)
{
    constexpr int MM = ORDER / 2;
    const int i = fidx[p];
    if ((unsigned)i >= (unsigned)n) {
        raise_status(sc, NB_ERR_ARG);
        return;
    }
    if (tfc) tf = tfc[cid[i]];  // ensemble: the particle's cluster block time
    const double h = tf - t[i];
    if (!(h > 0.0)) {
        raise_status(sc, NB_ERR_ARG);
        return;
    }
    double L[4][3], H[8][3], x0[3], v0[3];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) L[k][c] = d[(k * 3 + c) * np + i];
#pragma unroll
    for (int k = 0; k < MM; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) H[k][c] = Fp[(size_t)(3 * k + c) * fs];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        x0[c] = x[c * np + i];
        v0[c] = v[c * np + i];
    }
    const double potn = Fp[(size_t)(3 * MM) * fs];
    const double bacc = Fp[(size_t)(3 * MM + 1) * fs];  // sum_j m_j / R_ij^2

    const double ih = recip(h);
    double x1[3], v1[3], lim;
    bool finite_state;
    if (MIXED && correct_mixed<ORDER>(L, H, h, ih, x0, v0, bacc, eta, ne, x1, v1, lim)) {
        finite_state = true;
#pragma unroll
        for (int c = 0; c < 3; ++c) {  // exponent field not all ones
            finite_state = finite_state && (~__double_as_longlong(x1[c]) & 0x7FF0000000000000LL) != 0 &&
                           (~__double_as_longlong(v1[c]) & 0x7FF0000000000000LL) != 0;
        }
    } else {
        finite_state = correct_fp64<ORDER>(L, H, h, ih, x0, v0, bacc, eta, ne, x1, v1, lim);
    }
    // the floored criterion would read a non-finite derivative as zero
    if (!finite_state) raise_status(sc, NB_ERR_NAN);
    const double dtn = quantise_dt(lim, tf, dt_max, dt_min, sc);

#pragma unroll
    for (int c = 0; c < 3; ++c) {
        v[c * np + i] = v1[c];
        x[c * np + i] = x1[c];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) d[(k * 3 + c) * np + i] = (k < 2 * MM) ? H[k][c] : 0.0;
    t[i] = tf;
    dtv[i] = dtn;
    pot[i] = potn;
}

// Corrector, interpolation and new step for the particles of the last force.
// A device-driven cycle launches a fixed grid that strides over the block's
// active list (sized for the largest block, most of its CTAs would retire at
// once on the usual small ones).
template <int ORDER, bool MIXED>
__global__ void __launch_bounds__(128) k_correct(const int32_t* __restrict__ fidx, int fn, double tf,
                                                 const double* __restrict__ F, int64_t n, int64_t np,
                                                 double* __restrict__ x, double* __restrict__ v,
                                                 double* __restrict__ d, double* __restrict__ t,
                                                 double* __restrict__ dtv, double* __restrict__ pot, double eta,
                                                 double dt_max, double dt_min, NoiseEps ne, DevScalars* sc,
                                                 const double* __restrict__ tfc, const int32_t* __restrict__ cid,
                                                 const DevScalars* dyn, unsigned long long* hist)
{
    pdl_wait();
    pdl_release();
    if (dyn) {  // device-driven cycle: the block of the scheduler, unless idle
        if (dyn->idle) return;
        fn = (int)dyn->n_act;
        tf = dyn->t_blk;
    }
    if (hist && blockIdx.x == 0 && threadIdx.x == 0 && fn > 0) atomicAdd(&hist[31 - __clz(fn)], 1ull);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < fn; p += gridDim.x * blockDim.x)
        correct_one<ORDER, MIXED>(p, fidx, tf, F + p, (size_t)fn, n, np, x, v, d, t, dtv, pot, eta, dt_max, dt_min,
                                  ne, sc, tfc, cid);
}

cudaError_t launch_correct(nb_ctx* c, const double* tfc, const int32_t* cid, const DevScalars* dyn)
{
    const int nt = 128;
    const int64_t need = ((dyn ? c->n : c->f_n) + nt - 1) / nt;
    const int nb = (int)(dyn ? std::min<int64_t>(need, 4LL * c->sm_count) : need);
    const bool mixed = c->pred_prec == NB_MIXED;
    const bool pdl = c->pdl != 0;
    cudaError_t e;
#define NB_CORR(O, MX)                                                                                           \
    e = launch_k(k_correct<O, MX>, dim3(nb), dim3(nt), 0, c->stream, pdl, dyn ? c->act_idx : c->f_idx,         \
                 (int)c->f_n, c->f_t, c->F, c->n, c->np, c->x, c->v, c->d, c->t, c->dt, c->pot, c->eta,         \
                 c->dt_max, c->dt_min, c->noise[mixed ? 1 : 0], c->sc, tfc, cid, dyn, c->nact_hist)
    if (c->order == 4) {
        if (mixed) NB_CORR(4, true); else NB_CORR(4, false);
    } else if (c->order == 6) {
        if (mixed) NB_CORR(6, true); else NB_CORR(6, false);
    } else {
        if (mixed) NB_CORR(8, true); else NB_CORR(8, false);
    }
#undef NB_CORR
    return e;
}

// ============================================================== start-up
// Copy the start-up force (every particle active, list = identity) into the
// held derivatives: acc, jerk from the order-4 pass, snap from the order-6
// pass, crackle from the order-8 pass.
template <int PASS>
__global__ void k_startup_store(const double* __restrict__ F, int64_t n, int64_t np, double* __restrict__ d,
                                double* __restrict__ pot)
{
    constexpr int MM = PASS / 2;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int k = 0; k < MM; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) d[(k * 3 + c) * np + i] = F[(size_t)(3 * k + c) * n + i];
    pot[i] = F[(size_t)(3 * MM) * n + i];
}

cudaError_t launch_startup_store(nb_ctx* c, int order)
{
    const int nt = 256;
    const int nb = (int)((c->n + nt - 1) / nt);
    if (order == 4) k_startup_store<4><<<nb, nt, 0, c->stream>>>(c->F, c->n, c->np, c->d, c->pot);
    else if (order == 6) k_startup_store<6><<<nb, nt, 0, c->stream>>>(c->F, c->n, c->np, c->d, c->pot);
    else k_startup_store<8><<<nb, nt, 0, c->stream>>>(c->F, c->n, c->np, c->d, c->pot);
    return cudaGetLastError();
}

// Start-up step eta_s |a| / |jerk|, quantised at t = 0; t_i = 0.
__global__ void k_startup_dt(const double* __restrict__ d, int64_t n, int64_t np, double* __restrict__ t,
                             double* __restrict__ dtv, double eta_s, double dt_max, double dt_min, DevScalars* sc)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double a[3], j[3];
    for (int c = 0; c < 3; ++c) {
        a[c] = d[(0 * 3 + c) * np + i];
        j[c] = d[(1 * 3 + c) * np + i];
    }
    const double na = norm3(a), nj = norm3(j);
    const double lim = nj > 0.0 ? eta_s * na / nj : INFINITY;
    t[i] = 0.0;
    dtv[i] = quantise_dt(lim, 0.0, dt_max, dt_min, sc);
}

cudaError_t launch_startup_dt(nb_ctx* c)
{
    const int nt = 256;
    const int nb = (int)((c->n + nt - 1) / nt);
    k_startup_dt<<<nb, nt, 0, c->stream>>>(c->d, c->n, c->np, c->t, c->dt, c->eta_s, c->dt_max, c->dt_min, c->sc);
    return cudaGetLastError();
}

// ======================================================== shared step
// Every particle gets the step dtval; all must share t_0 = t[0], divisible by
// dtval (checked here, reported through the status word).
__global__ void k_set_dt(const double* __restrict__ t, double* __restrict__ dtv, int64_t n, double dtval,
                         DevScalars* sc)
{
    const double t0 = t[0];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (t[i] != t0) raise_status(sc, NB_ERR_NOT_SYNC);
        dtv[i] = dtval;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double q = t0 / dtval;
        if (q != floor(q)) raise_status(sc, NB_ERR_ARG);
    }
}

cudaError_t launch_set_dt(nb_ctx* c, double dt)
{
    int g = c->sm_count * 2;
    const int64_t need = (c->n + 255) / 256;
    if (need < g) g = (int)need;
    k_set_dt<<<g < 1 ? 1 : g, 256, 0, c->stream>>>(c->t, c->dt, c->n, dt, c->sc);
    return cudaGetLastError();
}

// ================================================================ energy
// Deterministic two-level sums: kinetic sum m v^2 / 2 and potential
// sum m_i pot_i / 2 (pot from an order-0 force pass, list = identity), and the
// time range min t_i, max t_i for the synchronisation check.
__global__ void __launch_bounds__(256) k_energy_part(const double* __restrict__ m, const double* __restrict__ v,
                                                     const double* __restrict__ F, const double* __restrict__ t,
                                                     int64_t n, int64_t np, double* __restrict__ red)
{
    __shared__ double sk[8], sp[8], smn[8], smx[8];
    double k = 0.0, w = 0.0, tmn = INFINITY, tmx = -INFINITY;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double vx = v[i], vy = v[np + i], vz = v[2 * np + i];
        k += 0.5 * m[i] * (vx * vx + vy * vy + vz * vz);
        if (F) w += 0.5 * m[i] * F[i];
        tmn = fmin(tmn, t[i]);
        tmx = fmax(tmx, t[i]);
    }
    k = warp_sum(k);
    w = warp_sum(w);
    tmn = warp_min(tmn);
    for (int o = 16; o > 0; o >>= 1) tmx = fmax(tmx, __shfl_xor_sync(0xffffffffu, tmx, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sk[warp] = k;
        sp[warp] = w;
        smn[warp] = tmn;
        smx[warp] = tmx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0, mn = INFINITY, mx = -INFINITY;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            a += sk[q];
            b += sp[q];
            mn = fmin(mn, smn[q]);
            mx = fmax(mx, smx[q]);
        }
        red[4 * blockIdx.x + 0] = a;
        red[4 * blockIdx.x + 1] = b;
        red[4 * blockIdx.x + 2] = mn;
        red[4 * blockIdx.x + 3] = mx;
    }
}

__global__ void k_energy_final(const double* __restrict__ red, int nb, double* __restrict__ out)
{
    if (threadIdx.x != 0) return;
    double a = 0, b = 0, mn = INFINITY, mx = -INFINITY;
    for (int q = 0; q < nb; ++q) {
        a += red[4 * q + 0];
        b += red[4 * q + 1];
        mn = fmin(mn, red[4 * q + 2]);
        mx = fmax(mx, red[4 * q + 3]);
    }
    out[0] = a;
    out[1] = b;
    out[2] = mn;
    out[3] = mx;
}

int energy_grid(const nb_ctx* c)
{
    int g = c->sm_count;
    const int64_t need = (c->n + 255) / 256;
    if (need < g) g = (int)need;
    return g < 1 ? 1 : g;
}

// with_pot = 0: only the time range and kinetic energy (F unused).
cudaError_t launch_energy_sums(nb_ctx* c, int with_pot)
{
    const int g = energy_grid(c);
    k_energy_part<<<g, 256, 0, c->stream>>>(c->m, c->v, with_pot ? c->F : nullptr, c->t, c->n, c->np, c->red);
    k_energy_final<<<1, 32, 0, c->stream>>>(c->red, g, c->red + 4 * g);
    return cudaGetLastError();
}

// ------------------------------------------------------------ state I/O
// The caller's state in particle order (x[n][3], v[n][3], d[n][6][3], t[n],
// dt[n]) sits in a staging buffer of 26 n doubles, segments in that order;
// these kernels move it to and from the structure-of-arrays state.
__global__ void k_state_check(const double* __restrict__ stage, int64_t n, DevScalars* sc)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* x = stage;
    const double* v = stage + 3 * n;
    const double* d = stage + 6 * n;
    const double* t = stage + 24 * n;
    const double* dt = stage + 25 * n;
    bool fin = isfinite(t[i]) && isfinite(dt[i]);
    for (int k = 0; k < 3; ++k) fin = fin && isfinite(x[3 * i + k]) && isfinite(v[3 * i + k]);
    for (int k = 0; k < 18; ++k) fin = fin && isfinite(d[18 * i + k]);
    if (!fin) raise_status(sc, NB_ERR_NAN);
    else if (!(dt[i] > 0.0)) raise_status(sc, NB_ERR_ARG);
}

__global__ void k_state_in(const double* __restrict__ stage, int64_t n, int64_t np, double* __restrict__ x,
                           double* __restrict__ v, double* __restrict__ d, double* __restrict__ t,
                           double* __restrict__ dt, const DevScalars* __restrict__ sc)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || sc->status != NB_OK) return;  // an invalid state leaves the old one in place
    for (int k = 0; k < 3; ++k) {
        x[k * np + i] = stage[3 * i + k];
        v[k * np + i] = stage[3 * n + 3 * i + k];
    }
    for (int k = 0; k < 18; ++k) d[k * np + i] = stage[6 * n + 18 * i + k];
    t[i] = stage[24 * n + i];
    dt[i] = stage[25 * n + i];
}

__global__ void k_state_out(double* __restrict__ stage, int64_t n, int64_t np, const double* __restrict__ x,
                            const double* __restrict__ v, const double* __restrict__ d,
                            const double* __restrict__ t, const double* __restrict__ dt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = 0; k < 3; ++k) {
        stage[3 * i + k] = x[k * np + i];
        stage[3 * n + 3 * i + k] = v[k * np + i];
    }
    for (int k = 0; k < 18; ++k) stage[6 * n + 18 * i + k] = d[k * np + i];
    stage[24 * n + i] = t[i];
    stage[25 * n + i] = dt[i];
}

cudaError_t launch_state_in(nb_ctx* c)
{
    const int g = (int)((c->n + 255) / 256);
    k_state_check<<<g, 256, 0, c->stream>>>(c->stage, c->n, c->sc);
    k_state_in<<<g, 256, 0, c->stream>>>(c->stage, c->n, c->np, c->x, c->v, c->d, c->t, c->dt, c->sc);
    return cudaGetLastError();
}

// Self-check of the integer conversions against cvt: n seeded
// inputs (splitmix64 of seed + k) -- every fourth any bit pattern, the others
// doubles with exponents across and at the edges of the float range -- and
// the widening of any float bit pattern; NaN inputs are skipped (NaN stays
// NaN in both, with payloads that may differ).  *bad += mismatching bits.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_convert_check(int64_t n, unsigned long long seed, unsigned long long* bad)
{
    unsigned long long nbad = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long z = splitmix64(seed + (unsigned long long)k);
        const unsigned long long keep = z & 0x800FFFFFFFFFFFFFull;  // sign and mantissa
        unsigned long long e;
        switch (k & 3) {
        case 0: e = (z >> 52) & 0x7FF; break;                                // any exponent
        case 1: e = 1023 - 160 + (z >> 53) % 321; break;                     // 2^-160 .. 2^160
        case 2: e = 1023 + 126 + (z >> 53) % 4; break;                       // 2^126 .. 2^129
        default: e = 1023 - 152 + (z >> 53) % 30; break;                     // 2^-152 .. 2^-123
        }
        const double x = __longlong_as_double((long long)(keep | (e << 52)));
        if (x == x && __float_as_uint(f64_to_f32_rz(x)) != __float_as_uint(f64_to_f32_rz_cvt(x))) ++nbad;
        const float f = __uint_as_float((unsigned)(z >> 16));
        if (f == f && __double_as_longlong(f32_to_f64(f)) != __double_as_longlong(f32_to_f64_cvt(f))) ++nbad;
    }
    if (nbad) atomicAdd(bad, nbad);
}

cudaError_t launch_convert_check(nb_ctx* c, int64_t n, unsigned long long seed, unsigned long long* bad)
{
    k_convert_check<<<4 * c->sm_count, 256, 0, c->stream>>>(n, seed, bad);
    return cudaGetLastError();
}

cudaError_t launch_state_out(nb_ctx* c)
{
    const int g = (int)((c->n + 255) / 256);
    k_state_out<<<g, 256, 0, c->stream>>>(c->stage, c->n, c->np, c->x, c->v, c->d, c->t, c->dt);
    return cudaGetLastError();
}

}  // namespace nb
