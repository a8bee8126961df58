// force_kernels.cuh -- direct-summation force kernel (K2) and its j-split reduction (K3).
//
// For each active particle i and every particle j of the predicted store the
// kernel sums the Plummer-softened Newtonian acceleration and its time
// derivatives ("Codes description": the GPUs compute the gravitational forces
// between particles; abstract: 4th/6th/8th-order Hermite).  With
// r = x_j - x_i, v = v_j - v_i, a = a_j - a_i, k = jerk_j - jerk_i,
// R^2 = r.r + eps_ij^2, q = m_j / R^3, alpha = r.v / R^2,
// w = (v.v + r.a) / R^2, u = (3 v.a + r.k) / R^2, the pair terms are
//   A = q r
//   J = q (v - 3 alpha r)
//   S = q (a - 6 alpha v + (15 alpha^2 - 3 w) r)
//   C = q (k - 9 alpha a + (45 alpha^2 - 9 w) v + (-105 alpha^3 + 45 alpha w - 3 u) r)
// which are dA/dt, d2A/dt2, d3A/dt3 rearranged so that every term is q times a
// combination of the four difference vectors; the potential sum is m_j / R.
//
// Layout: one CTA holds FORCE_NT i-particles in registers (one per thread) and
// streams a contiguous range of j tiles of JT records each through a ring of
// NSTAGE shared-memory buffers filled by one-dimensional TMA bulk copies
// (cp.async.bulk + mbarrier).  blockIdx.y splits the j range; each split writes
// partial sums [split][component][i] which K3 adds in fixed split order, so
// results are bitwise reproducible for a given launch shape.
//
// Mixed precision: positions are double-single (hi + lo floats); the difference
// (x_hi_j - x_hi_i) + (x_lo_j - x_lo_i) keeps ~44 bits for close pairs, the
// rest of the chain runs in FP32 (one MUFU rsqrt per pair), each tile's FP32
// sums are folded into a double-single accumulator with an error-free TwoSum,
// and the accumulator is widened to FP64 once per CTA.  No FP64 or conversion
// instruction runs in the j loop.
//
// FP64: the same structure in double, tile sums added to double accumulators
// (blocked summation).
#pragma once

#include "nb_internal.cuh"

namespace nb {

// Inverse distance of a pair: the hardware reciprocal square root (MUFU)
// with subnormal inputs flushed to zero.  rsqrtf without the flush adds a
// compare and two multiplies per pair to rescale subnormal inputs; R^2 is
// never subnormal here (at least eps^2 for softened pairs, and a subnormal
// unsoftened R^2 would put the pair force beyond the float range anyway).
// Measured: 5 % more interactions/s at N = 2^20, identical results.
__device__ __forceinline__ float rsqrt_ftz(float r2)
{
    float ri;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(ri) : "f"(r2));
    return ri;
}

// self-term guard: with per-particle softening a pair can have R^2 = 0 (an
// unsoftened particle meeting itself); its contribution is zero by definition.
template <bool PAIR>
__device__ __forceinline__ float guard_rinv(float r2)
{
    float ri = rsqrt_ftz(r2);
    if (PAIR) ri = (r2 > 0.0f) ? ri : 0.0f;
    return ri;
}

template <bool PAIR>
__device__ __forceinline__ double guard_rinv_d(double r2)
{
    double ri = rsqrt(r2);
    if (PAIR) ri = (r2 > 0.0) ? ri : 0.0;
    return ri;
}

// Per-particle softening: a warp whose i-particles all carry the system's
// largest eps^2 takes eps_i^2 as the pair value (no per-pair max or R^2 = 0
// guard); the others take the per-pair form, and lane 0 counts them.
__device__ __forceinline__ void count_pair_warp(DevScalars* sc, bool pair_form)
{
    if (pair_form && (threadIdx.x & 31) == 0) atomicAdd(&sc->pair_warps, 1ull);
}

// Wait for the copies still in flight after a timeout (bounded again), then
// the caller returns.  Called by thread 0 only.
static __device__ void drain_after_timeout(uint64_t* bars, int k, int nt, int ns = NSTAGE)
{
    for (int kk = k; kk < nt && kk < k + ns; ++kk) mbar_wait_bounded(&bars[kk % ns], (kk / ns) & 1);
}

// -------------------------------------------------------------------- K3
// F[c][p] = the sum of the j-split partials of component c of active particle
// p; the potential sum is negated (PC = index of the potential component).
// The summation order depends on (jsplit, n_act) alone, so every launcher
// (per-launch, device-driven, static) gives the same bits:
//   by warp   : lane l adds splits l, l+32, ... in turn, then the 32 lane
//               sums meet in a butterfly (every lane ends with the same bits,
//               as a + b == b + a exactly);
//   sequential: one thread per (component, particle) adds the splits in turn.
// The warp form serves many splits over few particles, where a thread per
// particle would leave the GPU idle behind one long chain of loads.
constexpr int RED_WARP_MIN_SPLIT = 9;
constexpr int RED_WARP_MAX_NACT = 4096;
constexpr int RED_NT = 256;
__host__ __device__ __forceinline__ bool reduce_by_warp(int jsplit, int n_act)
{
    return jsplit >= RED_WARP_MIN_SPLIT && n_act < RED_WARP_MAX_NACT;
}
// per-launch grid of k_force_reduce for NC components
__host__ __forceinline__ int reduce_grid(int jsplit, int n_act, int nc)
{
    return reduce_by_warp(jsplit, n_act) ? (n_act * nc + RED_NT / 32 - 1) / (RED_NT / 32)
                                         : (n_act * nc + RED_NT - 1) / RED_NT;
}

// q = c * n_act + p
template <int NC, int PC>
__device__ __forceinline__ void reduce_seq(const double* __restrict__ partial, int jsplit, int n_act, int q,
                                           double* __restrict__ F)
{
    const int c = q / n_act;
    const double* src = partial + q;
    const size_t stride = (size_t)NC * n_act;
    double s = 0.0;
#pragma unroll 8
    for (int sp = 0; sp < jsplit; ++sp) s += src[(size_t)sp * stride];
    F[q] = c == PC ? -s : s;
}

// q = p * NC + c; called by a whole warp
template <int NC, int PC>
__device__ __forceinline__ void reduce_warp(const double* __restrict__ partial, int jsplit, int n_act, int q,
                                            int lane, double* __restrict__ F)
{
    const int p = q / NC, c = q - p * NC;
    double s = 0.0;
    // unrolled so that the loads of several splits are in flight at once
    // (the adds keep their order: the same bits)
#pragma unroll 8
    for (int sp = lane; sp < jsplit; sp += 32) s += partial[((size_t)sp * NC + c) * n_act + p];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) F[(size_t)c * n_act + p] = c == PC ? -s : s;
}

// With one j-split the CTA holds the complete sums of its i-particles and
// writes the result straight to F (potential negated); otherwise it writes
// its partial row for the split reduction.  F == nullptr: partials always.
struct TileSum {
    double* F;  // [ncomp][ncol] result
    int jsplit;
};

template <int NC, int PC>
__device__ __forceinline__ void store_result(double* __restrict__ partial, int split, int ncol, int p, int c,
                                             double val, const TileSum& ts)
{
    if (ts.F && ts.jsplit == 1) ts.F[(size_t)c * ncol + p] = c == PC ? -val : val;
    else partial[((size_t)split * NC + c) * ncol + p] = val;
}

// i-particle data of the mixed kernel, as read from its own record.
struct IMixed {
    float4 i0, i1, i2, i3, i4;  // (x_hi, m) (x_lo, eps2) (v) (a) (jerk)
};

// One pair (i <- j): accumulates the pair terms into acc.  is_self masks the
// i-particle's own record by zeroing the inverse distance (every term
// carries it).
template <int ORDER, bool PAIR, bool SELF>
__device__ __forceinline__ void pair_mixed(const float4 w0, const float4 w1, const float4 w2, const float4 w3,
                                           const float4 w4, const IMixed& I, const float ei2, const bool is_self,
                                           float (&acc)[ncomp(ORDER)])
{
    constexpr int NC = ncomp(ORDER);
    const float dx = (w0.x - I.i0.x) + (w1.x - I.i1.x);
    const float dy = (w0.y - I.i0.y) + (w1.y - I.i1.y);
    const float dz = (w0.z - I.i0.z) + (w1.z - I.i1.z);
    // PAIR: eps_ij^2 = max(eps_i^2, eps_j^2); otherwise ei2 is the constant pair value
    const float e2 = PAIR ? fmaxf(w1.w, ei2) : ei2;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, e2)));
    float rinv = guard_rinv<PAIR>(r2);
    if (SELF) rinv = is_self ? 0.0f : rinv;
    const float mr = w0.w * rinv;
    if (ORDER == 0) {
        acc[0] += mr;
        return;
    }
    const float rinv2 = rinv * rinv;
    const float q = mr * rinv2;
    const float r3 = -3.0f * rinv2;
    const float dvx = w2.x - I.i2.x, dvy = w2.y - I.i2.y, dvz = w2.z - I.i2.z;
    acc[0] = fmaf(q, dx, acc[0]);
    acc[1] = fmaf(q, dy, acc[1]);
    acc[2] = fmaf(q, dz, acc[2]);
    // a3 = -3 alpha, the jerk coefficient
    const float a3 = fmaf(dx, dvx, fmaf(dy, dvy, dz * dvz)) * r3;
    acc[3] = fmaf(q, fmaf(a3, dx, dvx), acc[3]);
    acc[4] = fmaf(q, fmaf(a3, dy, dvy), acc[4]);
    acc[5] = fmaf(q, fmaf(a3, dz, dvz), acc[5]);
    if (ORDER >= 6) {
        const float dax = w3.x - I.i3.x, day = w3.y - I.i3.y, daz = w3.z - I.i3.z;
        // ww3 = -3 w; snap coefficients c2 = -6 alpha, c3 = 15 alpha^2 - 3 w
        const float ww3 = fmaf(dvx, dvx, fmaf(dvy, dvy, fmaf(dvz, dvz, fmaf(dx, dax, fmaf(dy, day, dz * daz))))) * r3;
        const float c2 = a3 + a3;
        const float c3 = fmaf((5.0f / 3.0f) * a3, a3, ww3);
        acc[6] = fmaf(q, fmaf(c3, dx, fmaf(c2, dvx, dax)), acc[6]);
        acc[7] = fmaf(q, fmaf(c3, dy, fmaf(c2, dvy, day)), acc[7]);
        acc[8] = fmaf(q, fmaf(c3, dz, fmaf(c2, dvz, daz)), acc[8]);
        if (ORDER >= 8) {
            const float dkx = w4.x - I.i4.x, dky = w4.y - I.i4.y, dkz = w4.z - I.i4.z;
            // u3 = -3 u; crackle: c4 = -9 alpha, c5 = 45 alpha^2 - 9 w = 3 c3,
            // c6 = -105 alpha^3 + 45 alpha w - 3 u
            const float u3 =
                fmaf(3.0f, fmaf(dvx, dax, fmaf(dvy, day, dvz * daz)), fmaf(dx, dkx, fmaf(dy, dky, dz * dkz))) * r3;
            const float c4 = 3.0f * a3;
            const float c5 = 3.0f * c3;  // 5 a3^2 + 3 ww3
            const float c6 = fmaf(a3, fmaf((35.0f / 9.0f) * a3, a3, 5.0f * ww3), u3);
            acc[9] = fmaf(q, fmaf(c6, dx, fmaf(c5, dvx, fmaf(c4, dax, dkx))), acc[9]);
            acc[10] = fmaf(q, fmaf(c6, dy, fmaf(c5, dvy, fmaf(c4, day, dky))), acc[10]);
            acc[11] = fmaf(q, fmaf(c6, dz, fmaf(c5, dvz, fmaf(c4, daz, dkz))), acc[11]);
        }
    }
    acc[NC - 2] += mr;
    acc[NC - 1] = fmaf(mr, rinv, acc[NC - 1]);
}

// i side of packed FP32x2 arithmetic: two i-particles (one per lane) or one
// particle in both.  The values are held negated (n*) so that every
// difference is an add.
struct IMixed2 {
    float2 nxh[3], nxl[3], nv[3], na[3], nk[3];
    float2 e2;  // eps_i^2 (per-particle softening) or the uniform pair value
};

__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }

// The j side of a packed pair: one record broadcast to both lanes, or one
// record per lane.
struct JMixed2 {
    float2 xh[3], xl[3], v[3], a[3], k[3];
    float2 m, e2;  // m_j, eps_j^2
};

template <int ORDER>
__device__ __forceinline__ JMixed2 j_bcast(const float4 w0, const float4 w1, const float4 w2, const float4 w3,
                                           const float4 w4)
{
    JMixed2 J;
    J.xh[0] = bc2(w0.x), J.xh[1] = bc2(w0.y), J.xh[2] = bc2(w0.z), J.m = bc2(w0.w);
    J.xl[0] = bc2(w1.x), J.xl[1] = bc2(w1.y), J.xl[2] = bc2(w1.z), J.e2 = bc2(w1.w);
    J.v[0] = bc2(w2.x), J.v[1] = bc2(w2.y), J.v[2] = bc2(w2.z);
    J.a[0] = bc2(w3.x), J.a[1] = bc2(w3.y), J.a[2] = bc2(w3.z);
    J.k[0] = bc2(w4.x), J.k[1] = bc2(w4.y), J.k[2] = bc2(w4.z);
    return J;
}

// records r (lane x) and s (lane y), RW float4 each
template <int ORDER, int RW>
__device__ __forceinline__ JMixed2 j_lanes(const float4* __restrict__ r, const float4* __restrict__ s)
{
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 r0 = r[0], r1 = r[1], r2 = ORDER >= 4 ? r[2] : z, r3 = ORDER >= 6 ? r[3] : z,
                 r4 = ORDER >= 8 ? r[4] : z;
    const float4 s0 = s[0], s1 = s[1], s2 = ORDER >= 4 ? s[2] : z, s3 = ORDER >= 6 ? s[3] : z,
                 s4 = ORDER >= 8 ? s[4] : z;
    JMixed2 J;
    J.xh[0] = make_float2(r0.x, s0.x), J.xh[1] = make_float2(r0.y, s0.y), J.xh[2] = make_float2(r0.z, s0.z);
    J.m = make_float2(r0.w, s0.w);
    J.xl[0] = make_float2(r1.x, s1.x), J.xl[1] = make_float2(r1.y, s1.y), J.xl[2] = make_float2(r1.z, s1.z);
    J.e2 = make_float2(r1.w, s1.w);
    J.v[0] = make_float2(r2.x, s2.x), J.v[1] = make_float2(r2.y, s2.y), J.v[2] = make_float2(r2.z, s2.z);
    J.a[0] = make_float2(r3.x, s3.x), J.a[1] = make_float2(r3.y, s3.y), J.a[2] = make_float2(r3.z, s3.z);
    J.k[0] = make_float2(r4.x, s4.x), J.k[1] = make_float2(r4.y, s4.y), J.k[2] = make_float2(r4.z, s4.z);
    return J;
}

// The packed pair chain: lane x and lane y each take one (i, j) pair.  Same
// pair terms and operation order as pair_mixed.  SELF: self_x / self_y mask
// a lane whose pair is a particle with itself.
template <int ORDER, bool PAIR, bool SELF>
__device__ __forceinline__ void pair_mixed_x2j(const JMixed2& J, const IMixed2& I, float2 (&acc)[ncomp(ORDER)],
                                               const bool self_x, const bool self_y)
{
    constexpr int NC = ncomp(ORDER);
    const float2 dx = __fadd2_rn(__fadd2_rn(J.xh[0], I.nxh[0]), __fadd2_rn(J.xl[0], I.nxl[0]));
    const float2 dy = __fadd2_rn(__fadd2_rn(J.xh[1], I.nxh[1]), __fadd2_rn(J.xl[1], I.nxl[1]));
    const float2 dz = __fadd2_rn(__fadd2_rn(J.xh[2], I.nxh[2]), __fadd2_rn(J.xl[2], I.nxl[2]));
    const float2 e2 = PAIR ? make_float2(fmaxf(J.e2.x, I.e2.x), fmaxf(J.e2.y, I.e2.y)) : I.e2;
    const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
    float2 rinv = make_float2(guard_rinv<PAIR>(r2.x), guard_rinv<PAIR>(r2.y));
    if (SELF) {  // every term carries rinv
        if (self_x) rinv.x = 0.0f;
        if (self_y) rinv.y = 0.0f;
    }
    const float2 mr = __fmul2_rn(J.m, rinv);
    if (ORDER == 0) {
        acc[0] = __fadd2_rn(acc[0], mr);
        return;
    }
    const float2 rinv2 = __fmul2_rn(rinv, rinv);
    const float2 q = __fmul2_rn(mr, rinv2);
    const float2 r3 = __fmul2_rn(bc2(-3.0f), rinv2);
    const float2 dvx = __fadd2_rn(J.v[0], I.nv[0]), dvy = __fadd2_rn(J.v[1], I.nv[1]),
                 dvz = __fadd2_rn(J.v[2], I.nv[2]);
    acc[0] = __ffma2_rn(q, dx, acc[0]);
    acc[1] = __ffma2_rn(q, dy, acc[1]);
    acc[2] = __ffma2_rn(q, dz, acc[2]);
    const float2 a3 = __fmul2_rn(__ffma2_rn(dx, dvx, __ffma2_rn(dy, dvy, __fmul2_rn(dz, dvz))), r3);
    acc[3] = __ffma2_rn(q, __ffma2_rn(a3, dx, dvx), acc[3]);
    acc[4] = __ffma2_rn(q, __ffma2_rn(a3, dy, dvy), acc[4]);
    acc[5] = __ffma2_rn(q, __ffma2_rn(a3, dz, dvz), acc[5]);
    if (ORDER >= 6) {
        const float2 dax = __fadd2_rn(J.a[0], I.na[0]), day = __fadd2_rn(J.a[1], I.na[1]),
                     daz = __fadd2_rn(J.a[2], I.na[2]);
        const float2 ww3 = __fmul2_rn(
            __ffma2_rn(dvx, dvx,
                       __ffma2_rn(dvy, dvy,
                                  __ffma2_rn(dvz, dvz, __ffma2_rn(dx, dax, __ffma2_rn(dy, day, __fmul2_rn(dz, daz)))))),
            r3);
        const float2 c2 = __fadd2_rn(a3, a3);
        const float2 c3 = __ffma2_rn(__fmul2_rn(bc2(5.0f / 3.0f), a3), a3, ww3);
        acc[6] = __ffma2_rn(q, __ffma2_rn(c3, dx, __ffma2_rn(c2, dvx, dax)), acc[6]);
        acc[7] = __ffma2_rn(q, __ffma2_rn(c3, dy, __ffma2_rn(c2, dvy, day)), acc[7]);
        acc[8] = __ffma2_rn(q, __ffma2_rn(c3, dz, __ffma2_rn(c2, dvz, daz)), acc[8]);
        if (ORDER >= 8) {
            const float2 dkx = __fadd2_rn(J.k[0], I.nk[0]), dky = __fadd2_rn(J.k[1], I.nk[1]),
                         dkz = __fadd2_rn(J.k[2], I.nk[2]);
            const float2 u3 = __fmul2_rn(
                __ffma2_rn(bc2(3.0f), __ffma2_rn(dvx, dax, __ffma2_rn(dvy, day, __fmul2_rn(dvz, daz))),
                           __ffma2_rn(dx, dkx, __ffma2_rn(dy, dky, __fmul2_rn(dz, dkz)))),
                r3);
            const float2 c4 = __fmul2_rn(bc2(3.0f), a3);
            const float2 c5 = __fmul2_rn(bc2(3.0f), c3);  // 5 a3^2 + 3 ww3
            const float2 c6 =
                __ffma2_rn(a3, __ffma2_rn(__fmul2_rn(bc2(35.0f / 9.0f), a3), a3, __fmul2_rn(bc2(5.0f), ww3)), u3);
            acc[9] = __ffma2_rn(q, __ffma2_rn(c6, dx, __ffma2_rn(c5, dvx, __ffma2_rn(c4, dax, dkx))), acc[9]);
            acc[10] = __ffma2_rn(q, __ffma2_rn(c6, dy, __ffma2_rn(c5, dvy, __ffma2_rn(c4, day, dky))), acc[10]);
            acc[11] = __ffma2_rn(q, __ffma2_rn(c6, dz, __ffma2_rn(c5, dvz, __ffma2_rn(c4, daz, dkz))), acc[11]);
        }
    }
    acc[NC - 2] = __fadd2_rn(acc[NC - 2], mr);
    acc[NC - 1] = __ffma2_rn(mr, rinv, acc[NC - 1]);
}

// Two i-particles in the two lanes (FFMA2 and kin on sm_100+), the j record
// broadcast to both: one instruction does the work of two.  srel: the
// lanes' own record in the tile (if any).
template <int ORDER, bool PAIR, bool SELF = false>
__device__ __forceinline__ void pair_mixed_x2(const float4 w0, const float4 w1, const float4 w2, const float4 w3,
                                              const float4 w4, const IMixed2& I, float2 (&acc)[ncomp(ORDER)],
                                              const int2 srel = make_int2(-1, -1), const int jj = 0)
{
    pair_mixed_x2j<ORDER, PAIR, SELF>(j_bcast<ORDER>(w0, w1, w2, w3, w4), I, acc, SELF && jj == srel.x,
                                      SELF && jj == srel.y);
}

// One j tile for NP lane-pairs (2 NP i-particles) of a thread: every record
// is read once from shared memory and applied to each pair.
// j-loop unroll of the packed tile: 4 records in flight at orders 4 and 6
// (+1-6 % measured), none at order 8 (its larger body unrolled by 2 is 1.5 %
// slower at 4 CTAs per SM).
template <int ORDER>
__host__ __device__ constexpr int xn_unroll()
{
    return ORDER >= 8 ? 1 : 4;
}
template <int ORDER, int RW, bool PAIR, bool SELF, int NP>
__device__ __forceinline__ void tile_mixed_xn(const float4* __restrict__ b, const IMixed2 (&I)[NP],
                                              const int2 (&srel)[NP], float2 (&acc)[NP][ncomp(ORDER)])
{
#pragma unroll xn_unroll<ORDER>()
    for (int jj = 0; jj < JT; ++jj) {
        const float4 w0 = b[jj * RW + 0];
        const float4 w1 = b[jj * RW + 1];
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 w2 = ORDER >= 4 ? b[jj * RW + 2] : z;
        const float4 w3 = ORDER >= 6 ? b[jj * RW + 3] : z;
        const float4 w4 = ORDER >= 8 ? b[jj * RW + 4] : z;
#pragma unroll
        for (int p = 0; p < NP; ++p) pair_mixed_x2<ORDER, PAIR, SELF>(w0, w1, w2, w3, w4, I[p], acc[p], srel[p], jj);
    }
}

__device__ __forceinline__ IMixed2 pack_pair(const IMixed& a, const IMixed& z, float ea, float ez)
{
    IMixed2 r;
    r.nxh[0] = make_float2(-a.i0.x, -z.i0.x);
    r.nxh[1] = make_float2(-a.i0.y, -z.i0.y);
    r.nxh[2] = make_float2(-a.i0.z, -z.i0.z);
    r.nxl[0] = make_float2(-a.i1.x, -z.i1.x);
    r.nxl[1] = make_float2(-a.i1.y, -z.i1.y);
    r.nxl[2] = make_float2(-a.i1.z, -z.i1.z);
    r.nv[0] = make_float2(-a.i2.x, -z.i2.x);
    r.nv[1] = make_float2(-a.i2.y, -z.i2.y);
    r.nv[2] = make_float2(-a.i2.z, -z.i2.z);
    r.na[0] = make_float2(-a.i3.x, -z.i3.x);
    r.na[1] = make_float2(-a.i3.y, -z.i3.y);
    r.na[2] = make_float2(-a.i3.z, -z.i3.z);
    r.nk[0] = make_float2(-a.i4.x, -z.i4.x);
    r.nk[1] = make_float2(-a.i4.y, -z.i4.y);
    r.nk[2] = make_float2(-a.i4.z, -z.i4.z);
    r.e2 = make_float2(ea, ez);
    return r;
}

// Resident CTAs per SM that the persistent kernels holding several mixed
// variants are compiled for: 4 at orders <= 6, 3 at order 8 (where the
// 4-particle variant's chain needs more than the 128 registers of 4 CTAs).
__host__ __device__ constexpr int dyn_min_ctas(int order) { return order >= 8 ? 3 : 4; }
// The per-launch two-per-thread kernel is compiled for the 4 CTAs per SM
// that its shared memory admits (at order 8 with the 2-stage ring), so that
// ptxas may use the registers occupancy leaves free: 116 instead of 96 at
// order 6 (3 % faster); at order 8, 3.2 % faster than ptxas's own target.
__host__ __device__ constexpr int xs_min_ctas(int order) { return 4; }

// Stages of the two-per-thread variant's ring: 2 at order 8, where 3 stages of
// 80-byte records and the sums of 13 components (57 KB per CTA) left room
// for 3 CTAs per SM and 2 stages (47 KB) admit 4; NSTAGE otherwise.
__host__ __device__ constexpr int xs_nstage(int order) { return order >= 8 ? 2 : NSTAGE; }

// Dynamic shared memory of the force variants that keep their double-single
// sums in shared memory (NP lane-pairs per thread): the TMA ring, then
// (hi, lo) float2 [NC][2 NP][FORCE_NT].
__host__ __device__ constexpr size_t xs_smem(int order, int rw, int np)
{
    return (size_t)xs_nstage(order) * JT * rw * 16 + (size_t)ncomp(order) * 2 * np * FORCE_NT * 8;
}

// One j tile for IPT i-particles: every record is read once from shared
// memory and applied to each i-particle of the thread.  SELF: the tile may
// hold one of the thread's own particles (at self_rel[q]).
template <int ORDER, int RW, bool PAIR, bool SELF, int IPT>
__device__ __forceinline__ void tile_mixed(const float4* __restrict__ b, const IMixed (&I)[IPT], const float (&ei2)[IPT],
                                           const int (&self_rel)[IPT], float (&acc)[IPT][ncomp(ORDER)])
{
#pragma unroll(IPT == 1 ? 2 : 1)
    for (int jj = 0; jj < JT; ++jj) {
        const float4 w0 = b[jj * RW + 0];
        const float4 w1 = b[jj * RW + 1];
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 w2 = ORDER >= 4 ? b[jj * RW + 2] : z;
        const float4 w3 = ORDER >= 6 ? b[jj * RW + 3] : z;
        const float4 w4 = ORDER >= 8 ? b[jj * RW + 4] : z;
#pragma unroll
        for (int q = 0; q < IPT; ++q)
            pair_mixed<ORDER, PAIR, SELF>(w0, w1, w2, w3, w4, I[q], ei2[q], SELF && jj == self_rel[q], acc[q]);
    }
}

// ----------------------------------------------------------------- mixed
// One CTA's work: the i-particles idx[p] for p = pbase + q * FORCE_NT < plim
// (q < IPT; thread t holds positions t and t + FORCE_NT of the i-tile) against
// the j tiles [t0, t0 + nt), partial sums to row `split`, column p of a
// [split][component][ncol] array.
template <int ORDER, int RW, bool PAIR, int IPT>
__device__ __forceinline__ void force_block_mixed(const float4* __restrict__ js, const int32_t* __restrict__ idx,
                                                  const int pbase0, const int plim, const int n, const int t0,
                                                  const int nt, const int split, const int ncol, const float eps2u,
                                                  const float eps2max, double* __restrict__ partial, DevScalars* sc,
                                                  const TileSum ts = TileSum{})
{
    constexpr int NC = ncomp(ORDER);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float4* buf = reinterpret_cast<float4*>(smem_raw);
    __shared__ __align__(8) uint64_t bars[NSTAGE];

    const int tid = threadIdx.x;
    const int pbase = pbase0 + tid;
    constexpr uint32_t TILE_BYTES = JT * RW * 16;

    if (tid == 0) {
        for (int k = 0; k < NSTAGE; ++k) mbar_init(&bars[k], 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int k = 0; k < NSTAGE && k < nt; ++k) {
            mbar_expect_tx(&bars[k], TILE_BYTES);
            bulk_g2s(buf + k * JT * RW, js + (size_t)(t0 + k) * JT * RW, TILE_BYTES, &bars[k]);
        }
    }

    // i-particles from the same store (identical predicted values on both sides)
    IMixed I[IPT];
    float ei2[IPT];
    int gi[IPT];
    bool dom_lane = true;
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        const int p = pbase + q * FORCE_NT;
        gi[q] = idx[p < plim ? p : plim - 1];
        if ((unsigned)gi[q] >= (unsigned)n) {
            raise_status(sc, NB_ERR_ARG);
            gi[q] = 0;
        }
        const float4* ri = js + (size_t)gi[q] * RW;
        I[q].i0 = ri[0];
        I[q].i1 = ri[1];
        I[q].i2 = ri[2];
        I[q].i3 = ORDER >= 6 ? ri[3] : make_float4(0.f, 0.f, 0.f, 0.f);
        I[q].i4 = ORDER >= 8 ? ri[4] : make_float4(0.f, 0.f, 0.f, 0.f);
        ei2[q] = PAIR ? I[q].i1.w : eps2u;
        dom_lane = dom_lane && ei2[q] >= eps2max && ei2[q] > 0.0f;
    }
    // A warp whose every i-particle is softened at least as much as any
    // particle pairs with the constant eps_i^2: the per-pair max and the
    // R^2 = 0 guard drop out (same results, fewer instructions).
    const bool dom = PAIR && __all_sync(0xffffffffu, dom_lane);
    count_pair_warp(sc, PAIR && !dom);

    float hi[IPT][NC], lo[IPT][NC];
#pragma unroll
    for (int q = 0; q < IPT; ++q)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            hi[q][c] = 0.f;
            lo[q][c] = 0.f;
        }

    for (int k = 0; k < nt; ++k) {
        const int st = k % NSTAGE;
        const bool ok = mbar_wait_bounded(&bars[st], (k / NSTAGE) & 1);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                raise_status(sc, NB_ERR_TIMEOUT);
                drain_after_timeout(bars, k, nt);
            }
            return;
        }
        const float4* b = buf + st * JT * RW;
        float acc[IPT][NC];
#pragma unroll
        for (int q = 0; q < IPT; ++q)
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[q][c] = 0.f;
        // the tile holding one of a lane's own particles takes the masked variant
        int self_rel[IPT];
        bool mine = false;
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            self_rel[q] = gi[q] - (t0 + k) * JT;
            mine = mine || (unsigned)self_rel[q] < (unsigned)JT;
        }
        const bool self_here = __any_sync(0xffffffffu, mine);
        // ei2 holds eps_i^2 (per-particle softening) or the uniform eps^2; on the
        // uniform and dominant paths it is the pair value itself
        if (!PAIR || dom) {
            if (self_here) tile_mixed<ORDER, RW, false, true, IPT>(b, I, ei2, self_rel, acc);
            else tile_mixed<ORDER, RW, false, false, IPT>(b, I, ei2, self_rel, acc);
        } else {
            if (self_here) tile_mixed<ORDER, RW, true, true, IPT>(b, I, ei2, self_rel, acc);
            else tile_mixed<ORDER, RW, true, false, IPT>(b, I, ei2, self_rel, acc);
        }
#pragma unroll
        for (int q = 0; q < IPT; ++q)
#pragma unroll
            for (int c = 0; c < NC; ++c) ds_add(hi[q][c], lo[q][c], acc[q][c]);

        __syncthreads();  // every thread is done with stage st
        if (tid == 0 && k + NSTAGE < nt) {
            mbar_expect_tx(&bars[st], TILE_BYTES);
            bulk_g2s(buf + st * JT * RW, js + (size_t)(t0 + k + NSTAGE) * JT * RW, TILE_BYTES, &bars[st]);
        }
    }

#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        const int p = pbase + q * FORCE_NT;
        if (p < plim) {
#pragma unroll
            for (int c = 0; c < NC; ++c)
                store_result<NC, pot_comp(ORDER)>(partial, split, ncol, p, c, (double)hi[q][c] + (double)lo[q][c], ts);
        }
    }
}

// Packed form with 2 NP i-particles per thread (positions t + q FORCE_NT,
// q < 2 NP, paired as lanes (2p, 2p+1)): every tile in packed FP32x2
// arithmetic, the self tile with per-lane masking; the double-single sums
// live in shared memory behind the ring (folded once per tile), so that the
// registers hold only the i-data and one tile's FP32 sums.
template <int ORDER, int RW, bool PAIR, int NP>
__device__ __forceinline__ void force_block_mixed_xs(const float4* __restrict__ js, const int32_t* __restrict__ idx,
                                                     const int pbase0, const int plim, const int n, const int t0,
                                                     const int nt, const int split, const int ncol,
                                                     const float eps2u, const float eps2max,
                                                     double* __restrict__ partial, DevScalars* sc,
                                                     const TileSum ts = TileSum{})
{
    constexpr int NC = ncomp(ORDER);
    constexpr int NQ = 2 * NP;
    constexpr int XS = xs_nstage(ORDER);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float4* buf = reinterpret_cast<float4*>(smem_raw);
    float2* dsum = reinterpret_cast<float2*>(smem_raw + (size_t)XS * JT * RW * 16);
    __shared__ __align__(8) uint64_t bars[XS];

    const int tid = threadIdx.x;
    const int pbase = pbase0 + tid;
    constexpr uint32_t TILE_BYTES = JT * RW * 16;

    if (tid == 0) {
        for (int k = 0; k < XS; ++k) mbar_init(&bars[k], 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int k = 0; k < XS && k < nt; ++k) {
            mbar_expect_tx(&bars[k], TILE_BYTES);
            bulk_g2s(buf + k * JT * RW, js + (size_t)(t0 + k) * JT * RW, TILE_BYTES, &bars[k]);
        }
    }

    IMixed2 I2[NP];
    int gi[NQ];
    bool dom_lane = true;
#pragma unroll
    for (int pp = 0; pp < NP; ++pp) {
        IMixed I[2];
        float e[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int q = 2 * pp + h;
            const int p = pbase + q * FORCE_NT;
            gi[q] = idx[p < plim ? p : plim - 1];
            if ((unsigned)gi[q] >= (unsigned)n) {
                raise_status(sc, NB_ERR_ARG);
                gi[q] = 0;
            }
            const float4* ri = js + (size_t)gi[q] * RW;
            I[h].i0 = ri[0];
            I[h].i1 = ri[1];
            I[h].i2 = ri[2];
            I[h].i3 = ORDER >= 6 ? ri[3] : make_float4(0.f, 0.f, 0.f, 0.f);
            I[h].i4 = ORDER >= 8 ? ri[4] : make_float4(0.f, 0.f, 0.f, 0.f);
            e[h] = PAIR ? I[h].i1.w : eps2u;
            dom_lane = dom_lane && e[h] >= eps2max && e[h] > 0.0f;
        }
        I2[pp] = pack_pair(I[0], I[1], e[0], e[1]);
    }
    const bool dom = PAIR && __all_sync(0xffffffffu, dom_lane);
    count_pair_warp(sc, PAIR && !dom);
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int q = 0; q < NQ; ++q) dsum[(c * NQ + q) * FORCE_NT + tid] = make_float2(0.f, 0.f);

    for (int k = 0; k < nt; ++k) {
        const int st = k % XS;
        const bool ok = mbar_wait_bounded(&bars[st], (k / XS) & 1);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                raise_status(sc, NB_ERR_TIMEOUT);
                drain_after_timeout(bars, k, nt, XS);
            }
            return;
        }
        const float4* b = buf + st * JT * RW;
        float2 acc[NP][NC];
#pragma unroll
        for (int pp = 0; pp < NP; ++pp)
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[pp][c] = make_float2(0.f, 0.f);
        int2 srel[NP];
        bool mine = false;
#pragma unroll
        for (int pp = 0; pp < NP; ++pp) {
            srel[pp] = make_int2(gi[2 * pp] - (t0 + k) * JT, gi[2 * pp + 1] - (t0 + k) * JT);
            mine = mine || (unsigned)srel[pp].x < (unsigned)JT || (unsigned)srel[pp].y < (unsigned)JT;
        }
        const bool self_here = __any_sync(0xffffffffu, mine);
        if (!PAIR || dom) {
            if (self_here) tile_mixed_xn<ORDER, RW, false, true, NP>(b, I2, srel, acc);
            else tile_mixed_xn<ORDER, RW, false, false, NP>(b, I2, srel, acc);
        } else {
            if (self_here) tile_mixed_xn<ORDER, RW, true, true, NP>(b, I2, srel, acc);
            else tile_mixed_xn<ORDER, RW, true, false, NP>(b, I2, srel, acc);
        }
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int pp = 0; pp < NP; ++pp) {
                float2* s0 = &dsum[(c * NQ + 2 * pp) * FORCE_NT + tid];
                float2* s1 = &dsum[(c * NQ + 2 * pp + 1) * FORCE_NT + tid];
                float2 h0 = *s0, h1 = *s1;
                ds_add(h0.x, h0.y, acc[pp][c].x);
                ds_add(h1.x, h1.y, acc[pp][c].y);
                *s0 = h0;
                *s1 = h1;
            }

        __syncthreads();  // every thread is done with stage st
        if (tid == 0 && k + XS < nt) {
            mbar_expect_tx(&bars[st], TILE_BYTES);
            bulk_g2s(buf + st * JT * RW, js + (size_t)(t0 + k + XS) * JT * RW, TILE_BYTES, &bars[st]);
        }
    }

#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int p = pbase + q * FORCE_NT;
        if (p < plim) {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const float2 h = dsum[(c * NQ + q) * FORCE_NT + tid];
                store_result<NC, pot_comp(ORDER)>(partial, split, ncol, p, c, (double)h.x + (double)h.y, ts);
            }
        }
    }
}

template <int ORDER, int RW, bool PAIR, int NP>
__global__ void __launch_bounds__(FORCE_NT, xs_min_ctas(ORDER)) k_force_mixed_xs(const float4* __restrict__ js,
                                                             const int32_t* __restrict__ idx, int n_act, int n,
                                                             int ntiles, int jt0, int jsplit, float eps2u, float eps2max,
                                                             double* __restrict__ partial, DevScalars* sc, double* F)
{
    const int split = blockIdx.y;
    const int t0 = jt0 + (int)((long long)split * ntiles / jsplit);
    const int t1 = jt0 + (int)((long long)(split + 1) * ntiles / jsplit);
    force_block_mixed_xs<ORDER, RW, PAIR, NP>(js, idx, blockIdx.x * (FORCE_NT * 2 * NP), n_act, n, t0, t1 - t0,
                                              split, n_act, eps2u, eps2max, partial, sc, TileSum{F, jsplit});
}

// j-parallel form for small active sets: NI = FORCE_NT / JP i-particles per
// CTA; thread (il, jl) = (tid % NI, tid / NI) takes i-particle il and the
// records jl, jl + JP, ... of every j tile, two at a time in the two lanes of
// packed FP32x2 arithmetic (records jl + 2 JP m in lane x, jl + 2 JP m + JP in
// lane y; the i-particle in both).  Each thread folds its two FP32 lane sums
// into one double-single sum every 2 JP tiles (JT records per lane sum, as in
// the two-per-thread form); at the end the JP sums of an i-particle are added
// in jl order through the (then idle) ring buffer, so the result depends on
// the launch shape only.
template <int JP>
__host__ __device__ constexpr int jx_unroll()
{
    return JT / (2 * JP) >= 4 ? 2 : JT / (2 * JP);
}
template <int ORDER, int RW, bool PAIR, bool SELF, int JP>
__device__ __forceinline__ void tile_mixed_jx(const float4* __restrict__ b, const IMixed2& I, const int jl,
                                              const int self_rel, float2 (&acc)[ncomp(ORDER)])
{
    static_assert(JT % (2 * JP) == 0, "a tile holds whole lane pairs");
#pragma unroll jx_unroll<JP>()
    for (int m = 0; m < JT / (2 * JP); ++m) {
        const int ja = jl + 2 * JP * m, jb = ja + JP;
        pair_mixed_x2j<ORDER, PAIR, SELF>(j_lanes<ORDER, RW>(b + ja * RW, b + jb * RW), I, acc,
                                          SELF && ja == self_rel, SELF && jb == self_rel);
    }
}

template <int ORDER, int RW, bool PAIR, int JP>
__device__ __forceinline__ void force_block_mixed_jp(const float4* __restrict__ js, const int32_t* __restrict__ idx,
                                                     const int pbase0, const int plim, const int n, const int t0,
                                                     const int nt, const int split, const int ncol,
                                                     const float eps2u, const float eps2max,
                                                     double* __restrict__ partial, DevScalars* sc,
                                                     const TileSum ts = TileSum{})
{
    constexpr int NC = ncomp(ORDER);
    constexpr int NI = FORCE_NT / JP;
    constexpr int FOLD = 2 * JP;
    static_assert(NSTAGE * JT * RW * 16 >= NC * FORCE_NT * 8, "ring too small for the lane reduction");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float4* buf = reinterpret_cast<float4*>(smem_raw);
    __shared__ __align__(8) uint64_t bars[NSTAGE];

    const int tid = threadIdx.x, il = tid % NI, jl = tid / NI;
    constexpr uint32_t TILE_BYTES = JT * RW * 16;

    if (tid == 0) {
        for (int k = 0; k < NSTAGE; ++k) mbar_init(&bars[k], 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int k = 0; k < NSTAGE && k < nt; ++k) {
            mbar_expect_tx(&bars[k], TILE_BYTES);
            bulk_g2s(buf + k * JT * RW, js + (size_t)(t0 + k) * JT * RW, TILE_BYTES, &bars[k]);
        }
    }

    const int p = pbase0 + il;
    int gi = idx[p < plim ? p : plim - 1];
    if ((unsigned)gi >= (unsigned)n) {
        raise_status(sc, NB_ERR_ARG);
        gi = 0;
    }
    IMixed I;
    {
        const float4* ri = js + (size_t)gi * RW;
        I.i0 = ri[0];
        I.i1 = ri[1];
        I.i2 = ri[2];
        I.i3 = ORDER >= 6 ? ri[3] : make_float4(0.f, 0.f, 0.f, 0.f);
        I.i4 = ORDER >= 8 ? ri[4] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float ei2 = PAIR ? I.i1.w : eps2u;
    const bool dom = PAIR && __all_sync(0xffffffffu, ei2 >= eps2max && ei2 > 0.0f);
    count_pair_warp(sc, PAIR && !dom);
    const IMixed2 I2 = pack_pair(I, I, ei2, ei2);

    float hi[NC], lo[NC];
    float2 acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        hi[c] = lo[c] = 0.f;
        acc[c] = make_float2(0.f, 0.f);
    }

    for (int k = 0; k < nt; ++k) {
        const int st = k % NSTAGE;
        const bool ok = mbar_wait_bounded(&bars[st], (k / NSTAGE) & 1);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                raise_status(sc, NB_ERR_TIMEOUT);
                drain_after_timeout(bars, k, nt);
            }
            return;
        }
        const float4* b = buf + st * JT * RW;
        const int self_rel = gi - (t0 + k) * JT;
        const bool self_here = __any_sync(0xffffffffu, (unsigned)self_rel < (unsigned)JT);
        if (!PAIR || dom) {
            if (self_here) tile_mixed_jx<ORDER, RW, false, true, JP>(b, I2, jl, self_rel, acc);
            else tile_mixed_jx<ORDER, RW, false, false, JP>(b, I2, jl, self_rel, acc);
        } else {
            if (self_here) tile_mixed_jx<ORDER, RW, true, true, JP>(b, I2, jl, self_rel, acc);
            else tile_mixed_jx<ORDER, RW, true, false, JP>(b, I2, jl, self_rel, acc);
        }
        if ((k + 1) % FOLD == 0 || k + 1 == nt) {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                ds_add(hi[c], lo[c], acc[c].x);
                ds_add(hi[c], lo[c], acc[c].y);
                acc[c] = make_float2(0.f, 0.f);
            }
        }
        __syncthreads();  // every thread is done with stage st
        if (tid == 0 && k + NSTAGE < nt) {
            mbar_expect_tx(&bars[st], TILE_BYTES);
            bulk_g2s(buf + st * JT * RW, js + (size_t)(t0 + k + NSTAGE) * JT * RW, TILE_BYTES, &bars[st]);
        }
    }
    // every copy has landed and been consumed: the ring holds the lane sums
    float2* lane = reinterpret_cast<float2*>(smem_raw);
#pragma unroll
    for (int c = 0; c < NC; ++c) lane[c * FORCE_NT + tid] = make_float2(hi[c], lo[c]);
    __syncthreads();
    for (int o = tid; o < NI * NC; o += FORCE_NT) {
        const int oi = o % NI, c = o / NI;
        float h = 0.f, l = 0.f;
        for (int q = 0; q < JP; ++q) {
            const float2 v = lane[c * FORCE_NT + q * NI + oi];
            ds_add_ds(h, l, v.x, v.y);
        }
        const int pp = pbase0 + oi;
        if (pp < plim) store_result<NC, pot_comp(ORDER)>(partial, split, ncol, pp, c, (double)h + (double)l, ts);
    }
}

// One system, j-parallel form: blockIdx.x = i-tile of FORCE_NT / JP active
// particles, blockIdx.y = j-split of the whole store.  Compiled for the
// resident CTAs of the persistent kernels (dyn_min_ctas): at order 8, 3 CTAs
// give the chain 156-161 registers without spills (4 CTAs: 128 registers and
// spills, 3 % slower on 64-200 active particles of the cusp).
template <int ORDER, int RW, bool PAIR, int JP>
__global__ void __launch_bounds__(FORCE_NT, dyn_min_ctas(ORDER)) k_force_mixed_jp(const float4* __restrict__ js,
                                                             const int32_t* __restrict__ idx, int n_act, int n,
                                                             int ntiles, int jt0, int jsplit, float eps2u, float eps2max,
                                                             double* __restrict__ partial, DevScalars* sc, double* F)
{
    const int split = blockIdx.y;
    const int t0 = jt0 + (int)((long long)split * ntiles / jsplit);
    const int t1 = jt0 + (int)((long long)(split + 1) * ntiles / jsplit);
    force_block_mixed_jp<ORDER, RW, PAIR, JP>(js, idx, blockIdx.x * (FORCE_NT / JP), n_act, n, t0, t1 - t0, split,
                                              n_act, eps2u, eps2max, partial, sc,
                                              TileSum{F, jsplit});
}

// One system: blockIdx.x = i-tile of FORCE_NT * IPT active particles,
// blockIdx.y = j-split of the whole store.
template <int ORDER, int RW, bool PAIR, int IPT>
__global__ void __launch_bounds__(FORCE_NT) k_force_mixed(const float4* __restrict__ js, const int32_t* __restrict__ idx,
                                                          int n_act, int n, int ntiles, int jt0, int jsplit, float eps2u,
                                                          float eps2max, double* __restrict__ partial, DevScalars* sc,
                                                          double* F)
{
    const int split = blockIdx.y;
    const int t0 = jt0 + (int)((long long)split * ntiles / jsplit);
    const int t1 = jt0 + (int)((long long)(split + 1) * ntiles / jsplit);
    force_block_mixed<ORDER, RW, PAIR, IPT>(js, idx, blockIdx.x * (FORCE_NT * IPT), n_act, n, t0, t1 - t0, split, n_act,
                                            eps2u, eps2max, partial, sc, TileSum{F, jsplit});
}

// records jl, jl + JP, ... of the tile (JP = 1: every record)
template <int ORDER, int RW, bool PAIR, bool SELF, int JP = 1>
__device__ __forceinline__ void tile_fp64(const double2* __restrict__ b, const double2 i0, const double2 i1,
                                          const double2 i2, const double2 i3, const double2 i4, const double2 i5,
                                          const double2 i6, const double2 i7, const double ei2, const double eps2u,
                                          const int self_rel, double (&acc)[ncomp(ORDER)], const int jl = 0)
{
    constexpr int NC = ncomp(ORDER);
    for (int jj = jl; jj < JT; jj += JP) {
        const double2 w0 = b[jj * RW + 0], w1 = b[jj * RW + 1];
        const double dx = w0.x - i0.x, dy = w0.y - i0.y, dz = w1.x - i1.x;
        const double2 w3 = b[jj * RW + 3];
        const double e2 = PAIR ? fmax(w3.y, ei2) : eps2u;
        const double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, e2)));
        double rinv = guard_rinv_d<PAIR>(r2);
        if (SELF) rinv = (jj == self_rel) ? 0.0 : rinv;
        const double mr = w1.y * rinv;
        if (ORDER == 0) {
            acc[0] += mr;
            continue;
        }
        const double rinv2 = rinv * rinv;
        const double q = mr * rinv2;
        const double2 w2 = b[jj * RW + 2];
        const double dvx = w2.x - i2.x, dvy = w2.y - i2.y, dvz = w3.x - i3.x;
        acc[0] = fma(q, dx, acc[0]);
        acc[1] = fma(q, dy, acc[1]);
        acc[2] = fma(q, dz, acc[2]);
        const double al = fma(dx, dvx, fma(dy, dvy, dz * dvz)) * rinv2;
        const double c1 = -3.0 * al;
        acc[3] = fma(q, fma(c1, dx, dvx), acc[3]);
        acc[4] = fma(q, fma(c1, dy, dvy), acc[4]);
        acc[5] = fma(q, fma(c1, dz, dvz), acc[5]);
        if (ORDER >= 6) {
            const double2 w4 = b[jj * RW + 4], w5 = b[jj * RW + 5];
            const double dax = w4.x - i4.x, day = w4.y - i4.y, daz = w5.x - i5.x;
            const double w = fma(dvx, dvx, fma(dvy, dvy, fma(dvz, dvz, fma(dx, dax, fma(dy, day, dz * daz))))) * rinv2;
            const double c2 = -6.0 * al;
            const double c3 = fma(15.0 * al, al, -3.0 * w);
            acc[6] = fma(q, fma(c3, dx, fma(c2, dvx, dax)), acc[6]);
            acc[7] = fma(q, fma(c3, dy, fma(c2, dvy, day)), acc[7]);
            acc[8] = fma(q, fma(c3, dz, fma(c2, dvz, daz)), acc[8]);
            if (ORDER >= 8) {
                const double2 w6 = b[jj * RW + 6], w7 = b[jj * RW + 7];
                const double dkx = w6.x - i6.x, dky = w6.y - i6.y, dkz = w7.x - i7.x;
                const double u =
                    fma(3.0, fma(dvx, dax, fma(dvy, day, dvz * daz)), fma(dx, dkx, fma(dy, dky, dz * dkz))) * rinv2;
                const double c4 = -9.0 * al;
                const double c5 = fma(45.0 * al, al, -9.0 * w);
                const double c6 = fma(al, fma(-105.0 * al, al, 45.0 * w), -3.0 * u);
                acc[9] = fma(q, fma(c6, dx, fma(c5, dvx, fma(c4, dax, dkx))), acc[9]);
                acc[10] = fma(q, fma(c6, dy, fma(c5, dvy, fma(c4, day, dky))), acc[10]);
                acc[11] = fma(q, fma(c6, dz, fma(c5, dvz, fma(c4, daz, dkz))), acc[11]);
            }
        }
        acc[NC - 2] += mr;
        acc[NC - 1] = fma(mr, rinv, acc[NC - 1]);
    }
}

// ------------------------------------------------------------------ FP64
// FP64 record in 16-byte words (double2): w0 = (x.x, x.y), w1 = (x.z, m),
// w2 = (v.x, v.y), w3 = (v.z, eps2), w4 = (a.x, a.y), w5 = (a.z, 0),
// w6 = (jerk.x, jerk.y), w7 = (jerk.z, 0).
// One CTA's work (one i-particle per thread), as force_block_mixed.
// JP > 1: the j-parallel form (NI = FORCE_NT / JP i-particles per CTA,
// thread (tid % NI, tid / NI) takes every JP-th record of a tile; the JP
// lane sums of a particle are added in lane order through the idle ring).
template <int ORDER, int RW, bool PAIR, int JP = 1>
__device__ __forceinline__ void force_block_fp64(const double2* __restrict__ js, const int32_t* __restrict__ idx,
                                                 const int pbase0, const int plim, const int n, const int t0,
                                                 const int nt, const int split, const int ncol, const double eps2u,
                                                 double* __restrict__ partial, DevScalars* sc,
                                                 const TileSum ts = TileSum{})
{
    constexpr int NC = ncomp(ORDER);
    constexpr int NI = FORCE_NT / JP;
    static_assert(JP == 1 || NSTAGE * JT * RW * 16 >= NC * FORCE_NT * 8, "ring too small for the lane reduction");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    double2* buf = reinterpret_cast<double2*>(smem_raw);
    __shared__ __align__(8) uint64_t bars[NSTAGE];

    const int tid = threadIdx.x, il = tid % NI, jl = tid / NI;
    const int p = pbase0 + il;
    constexpr uint32_t TILE_BYTES = JT * RW * 16;

    if (tid == 0) {
        for (int k = 0; k < NSTAGE; ++k) mbar_init(&bars[k], 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int k = 0; k < NSTAGE && k < nt; ++k) {
            mbar_expect_tx(&bars[k], TILE_BYTES);
            bulk_g2s(buf + k * JT * RW, js + (size_t)(t0 + k) * JT * RW, TILE_BYTES, &bars[k]);
        }
    }

    int gi = idx[p < plim ? p : plim - 1];
    if ((unsigned)gi >= (unsigned)n) {
        raise_status(sc, NB_ERR_ARG);
        gi = 0;
    }
    const double2* ri = js + (size_t)gi * RW;
    const double2 i0 = ri[0], i1 = ri[1], i2 = ri[2], i3 = ri[3];
    double2 i4 = make_double2(0.0, 0.0), i5 = i4, i6 = i4, i7 = i4;
    if (ORDER >= 6) {
        i4 = ri[4];
        i5 = ri[5];
    }
    if (ORDER >= 8) {
        i6 = ri[6];
        i7 = ri[7];
    }
    const double ei2 = PAIR ? i3.y : eps2u;

    double sum[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) sum[c] = 0.0;

    for (int k = 0; k < nt; ++k) {
        const int st = k % NSTAGE;
        const bool ok = mbar_wait_bounded(&bars[st], (k / NSTAGE) & 1);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                raise_status(sc, NB_ERR_TIMEOUT);
                drain_after_timeout(bars, k, nt);
            }
            return;
        }
        const double2* b = buf + st * JT * RW;
        double acc[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = 0.0;
        const int self_rel = gi - (t0 + k) * JT;
        if (__any_sync(0xffffffffu, (unsigned)self_rel < (unsigned)JT))
            tile_fp64<ORDER, RW, PAIR, true, JP>(b, i0, i1, i2, i3, i4, i5, i6, i7, ei2, eps2u, self_rel, acc, jl);
        else
            tile_fp64<ORDER, RW, PAIR, false, JP>(b, i0, i1, i2, i3, i4, i5, i6, i7, ei2, eps2u, -1, acc, jl);
#pragma unroll
        for (int c = 0; c < NC; ++c) sum[c] += acc[c];

        __syncthreads();
        if (tid == 0 && k + NSTAGE < nt) {
            mbar_expect_tx(&bars[st], TILE_BYTES);
            bulk_g2s(buf + st * JT * RW, js + (size_t)(t0 + k + NSTAGE) * JT * RW, TILE_BYTES, &bars[st]);
        }
    }

    if (JP == 1) {
        if (p < plim) {
#pragma unroll
            for (int c = 0; c < NC; ++c) store_result<NC, pot_comp(ORDER)>(partial, split, ncol, p, c, sum[c], ts);
        }
        return;
    }
    // every copy has landed and been consumed: the ring holds the lane sums
    double* lane = reinterpret_cast<double*>(smem_raw);
#pragma unroll
    for (int c = 0; c < NC; ++c) lane[c * FORCE_NT + tid] = sum[c];
    __syncthreads();
    for (int o = tid; o < NI * NC; o += FORCE_NT) {
        const int oi = o % NI, c = o / NI;
        double s = 0.0;
        for (int q = 0; q < JP; ++q) s += lane[c * FORCE_NT + q * NI + oi];
        const int pp = pbase0 + oi;
        if (pp < plim) store_result<NC, pot_comp(ORDER)>(partial, split, ncol, pp, c, s, ts);
    }
}

// F: result of a one-split launch (nullptr: partials only)
template <int ORDER, int RW, bool PAIR, int JP = 1>
__global__ void __launch_bounds__(FORCE_NT) k_force_fp64(const double2* __restrict__ js, const int32_t* __restrict__ idx,
                                                         int n_act, int n, int ntiles, int jt0, int jsplit, double eps2u,
                                                         double* __restrict__ partial, DevScalars* sc, double* F)
{
    const int split = blockIdx.y;
    const int t0 = jt0 + (int)((long long)split * ntiles / jsplit);
    const int t1 = jt0 + (int)((long long)(split + 1) * ntiles / jsplit);
    force_block_fp64<ORDER, RW, PAIR, JP>(js, idx, blockIdx.x * (FORCE_NT / JP), n_act, n, t0, t1 - t0, split, n_act,
                                          eps2u, partial, sc, TileSum{F, jsplit});
}

// ------------------------------------------------------- device-driven cycle
// Launch shape from the scheduler's n_act, chosen on the device with the
// host's rule (makespan ceil(it*js/slots)/js, ties within 0.5% to fewer splits,
// capped by the partial-sum buffer); an active set past t_end makes the
// cycle idle.

// Persistent force: a fixed grid walks the (i-tile, split) items of the
// device-chosen shape.  SMALL: the variants of up to FORCE_NT i-particles per
// CTA (4, 32, FORCE_NT), compiled for dyn_min_ctas resident CTAs; otherwise
// the two-per-thread variant (2 FORCE_NT), whose block is an out-of-line
// call (xs_item), compiled for the CTAs of its per-launch kernel.  The kernel not matching the chosen variant returns at
// once.
// The two-per-thread block as a call of its own: compiled apart from a
// persistent caller's item loop it keeps the code of its per-launch kernel
// (inlined into the loop it ran 12-20 % slower at order 8, 5 % at order 6).
template <int ORDER, int RW, bool PAIR>
__device__ __noinline__ void xs_item(const float4* __restrict__ js, const int32_t* __restrict__ idx, int pbase0,
                                     int plim, int n, int t0, int nt, int split, int ncol, float eps2u, float eps2max,
                                     double* __restrict__ partial, DevScalars* sc, TileSum ts)
{
    force_block_mixed_xs<ORDER, RW, PAIR, 1>(js, idx, pbase0, plim, n, t0, nt, split, ncol, eps2u, eps2max, partial,
                                             sc, ts);
}

template <int ORDER, int RW, bool PAIR, bool SMALL>
__global__ void __launch_bounds__(FORCE_NT, SMALL ? dyn_min_ctas(ORDER) : xs_min_ctas(ORDER))
    k_force_mixed_dyn(const float4* __restrict__ js, const int32_t* __restrict__ idx, int n, int ntiles, float eps2u,
                      float eps2max, double* __restrict__ partial, DevScalars* sc, double* F)
{
    pdl_wait();
    pdl_release();
    if (sc->idle) return;
    const int ni = sc->ni;
    if (SMALL != (ni <= FORCE_NT)) return;
    const int n_act = (int)sc->n_act, it = sc->itiles, jsplit = sc->jsplit;
    for (int w = blockIdx.x; w < it * jsplit; w += gridDim.x) {
        const int itile = w % it, split = w / it;
        const int t0 = (int)((long long)split * ntiles / jsplit);
        const int t1 = (int)((long long)(split + 1) * ntiles / jsplit);
        const TileSum tsum{F, jsplit};
        if (!SMALL)
            xs_item<ORDER, RW, PAIR>(js, idx, itile * ni, n_act, n, t0, t1 - t0, split, n_act, eps2u, eps2max, partial,
                                     sc, tsum);
        else if (ni == FORCE_NT)
            force_block_mixed<ORDER, RW, PAIR, 1>(js, idx, itile * ni, n_act, n, t0, t1 - t0, split, n_act, eps2u,
                                                  eps2max, partial, sc, tsum);
        else if (ni == FORCE_NT / 4)
            force_block_mixed_jp<ORDER, RW, PAIR, 4>(js, idx, itile * ni, n_act, n, t0, t1 - t0, split, n_act,
                                                     eps2u, eps2max, partial, sc, tsum);
        else
            force_block_mixed_jp<ORDER, RW, PAIR, 32>(js, idx, itile * ni, n_act, n, t0, t1 - t0, split, n_act,
                                                      eps2u, eps2max, partial, sc, tsum);
        // every thread is done before the next item re-arms the ring; a
        // status raised by any CTA ends the walk
        if (__syncthreads_or(threadIdx.x == 0 && *(volatile int*)&sc->status != 0)) return;
    }
}

template <int ORDER, int RW, bool PAIR>
__global__ void __launch_bounds__(FORCE_NT) k_force_fp64_dyn(const double2* __restrict__ js,
                                                             const int32_t* __restrict__ idx, int n, int ntiles,
                                                             double eps2u, double* __restrict__ partial,
                                                             DevScalars* sc, double* F)
{
    pdl_wait();
    pdl_release();
    if (sc->idle) return;
    const int n_act = (int)sc->n_act, it = sc->itiles, jsplit = sc->jsplit;
    for (int w = blockIdx.x; w < it * jsplit; w += gridDim.x) {
        const int itile = w % it, split = w / it;
        const int t0 = (int)((long long)split * ntiles / jsplit);
        const int t1 = (int)((long long)(split + 1) * ntiles / jsplit);
        const int ni = sc->ni;
        if (ni == FORCE_NT)
            force_block_fp64<ORDER, RW, PAIR, 1>(js, idx, itile * ni, n_act, n, t0, t1 - t0, split, n_act, eps2u,
                                                 partial, sc, TileSum{F, jsplit});
        else if (ni == FORCE_NT / 4)
            force_block_fp64<ORDER, RW, PAIR, 4>(js, idx, itile * ni, n_act, n, t0, t1 - t0, split, n_act, eps2u,
                                                 partial, sc, TileSum{F, jsplit});
        else
            force_block_fp64<ORDER, RW, PAIR, 32>(js, idx, itile * ni, n_act, n, t0, t1 - t0, split, n_act, eps2u,
                                                  partial, sc, TileSum{F, jsplit});
        if (__syncthreads_or(threadIdx.x == 0 && *(volatile int*)&sc->status != 0)) return;
    }
}

// Device-driven form: a fixed grid strides over the block the scheduler
// chose; nothing to do after a one-split launch (the force wrote F).
template <int NC, int PC>
__global__ void __launch_bounds__(RED_NT) k_force_reduce_dyn(const double* __restrict__ partial,
                                                             const DevScalars* __restrict__ sc,
                                                             double* __restrict__ F)
{
    pdl_wait();
    pdl_release();
    if (sc->idle || sc->jsplit == 1) return;
    const int n_act = (int)sc->n_act, jsplit = sc->jsplit;
    const int g = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    if (reduce_by_warp(jsplit, n_act)) {
        for (int q = g >> 5; q < n_act * NC; q += stride >> 5)
            reduce_warp<NC, PC>(partial, jsplit, n_act, q, threadIdx.x & 31, F);
    } else {
        for (int q = g; q < n_act * NC; q += stride) reduce_seq<NC, PC>(partial, jsplit, n_act, q, F);
    }
}

template <int NC, int PC>
__global__ void __launch_bounds__(RED_NT) k_force_reduce(const double* __restrict__ partial, int jsplit, int n_act,
                                                         double* __restrict__ F)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (reduce_by_warp(jsplit, n_act)) {
        const int q = g >> 5;  // warp-uniform
        if (q < n_act * NC) reduce_warp<NC, PC>(partial, jsplit, n_act, q, threadIdx.x & 31, F);
    } else if (g < n_act * NC) {
        reduce_seq<NC, PC>(partial, jsplit, n_act, g, F);
    }
}


}  // namespace nb
