// k_force.cu -- launchers of the force kernel (K2) and its j-split reduction (K3);
// the kernels are in force_kernels.cuh.
#include "force_kernels.cuh"

namespace nb {

// ---------------------------------------------------------------- launch
template <typename KernelT>
static int occupancy_of(KernelT kern, size_t smem)
{
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, FORCE_NT, smem) != cudaSuccess) occ = 1;
    return occ < 1 ? 1 : occ;
}

template <int ORDER, int RW, bool PAIR, int IPT>
static cudaError_t run_mixed_ipt(nb_ctx* c, const int32_t* idx, int n_act, int jsplit, int itiles, int* occ_out)
{
    auto kern = k_force_mixed<ORDER, RW, PAIR, IPT>;
    const size_t smem = (size_t)NSTAGE * JT * RW * 16;
    static bool configured = false;
    static int occ = 1;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        occ = occupancy_of(kern, smem);
        configured = true;
    }
    if (occ_out) {
        *occ_out = occ;
        return cudaSuccess;
    }
    dim3 grid(itiles, jsplit);
    kern<<<grid, FORCE_NT, smem, c->stream>>>(reinterpret_cast<const float4*>(c->jstore), idx, n_act, (int)c->n,
                                              c->ltn, c->lt0, jsplit, (float)(c->eps * c->eps),
                                              eps2_threshold(c->eps2_max), c->partial, c->sc, c->F);
    return cudaGetLastError();
}

template <int ORDER, int RW, bool PAIR, int JP>
static cudaError_t run_mixed_jp(nb_ctx* c, const int32_t* idx, int n_act, int jsplit, int itiles, int* occ_out)
{
    auto kern = k_force_mixed_jp<ORDER, RW, PAIR, JP>;
    const size_t smem = (size_t)NSTAGE * JT * RW * 16;
    static bool configured = false;
    static int occ = 1;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        occ = occupancy_of(kern, smem);
        configured = true;
    }
    if (occ_out) {
        *occ_out = occ;
        return cudaSuccess;
    }
    dim3 grid(itiles, jsplit);
    kern<<<grid, FORCE_NT, smem, c->stream>>>(reinterpret_cast<const float4*>(c->jstore), idx, n_act, (int)c->n,
                                              c->ltn, c->lt0, jsplit, (float)(c->eps * c->eps),
                                              eps2_threshold(c->eps2_max), c->partial, c->sc, c->F);
    return cudaGetLastError();
}

template <int ORDER, int RW, bool PAIR, int NP>
static cudaError_t run_mixed_xs(nb_ctx* c, const int32_t* idx, int n_act, int jsplit, int itiles, int* occ_out)
{
    auto kern = k_force_mixed_xs<ORDER, RW, PAIR, NP>;
    const size_t smem = xs_smem(ORDER, RW, NP);
    static bool configured = false;
    static int occ = 1;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        occ = occupancy_of(kern, smem);
        configured = true;
    }
    if (occ_out) {
        *occ_out = occ;
        return cudaSuccess;
    }
    dim3 grid(itiles, jsplit);
    kern<<<grid, FORCE_NT, smem, c->stream>>>(reinterpret_cast<const float4*>(c->jstore), idx, n_act, (int)c->n,
                                              c->ltn, c->lt0, jsplit, (float)(c->eps * c->eps),
                                              eps2_threshold(c->eps2_max), c->partial, c->sc, c->F);
    return cudaGetLastError();
}

// Mixed path: the variant with ni i-particles per CTA (mixed_ni).
template <int ORDER, int RW, bool PAIR>
static cudaError_t run_mixed(nb_ctx* c, const int32_t* idx, int n_act, int jsplit, int itiles, int* occ_out, int ni)
{
    switch (ni) {
    case 2 * FORCE_NT: return run_mixed_xs<ORDER, RW, PAIR, 1>(c, idx, n_act, jsplit, itiles, occ_out);
    case FORCE_NT: return run_mixed_ipt<ORDER, RW, PAIR, 1>(c, idx, n_act, jsplit, itiles, occ_out);
    case FORCE_NT / 4: return run_mixed_jp<ORDER, RW, PAIR, 4>(c, idx, n_act, jsplit, itiles, occ_out);
    case FORCE_NT / 32: return run_mixed_jp<ORDER, RW, PAIR, 32>(c, idx, n_act, jsplit, itiles, occ_out);
    default: return cudaErrorInvalidValue;
    }
}

// FP64 path: bound by the FP64 pipe; one i-particle per thread (JP = 1) or
// the j-parallel forms for small active sets.
template <int ORDER, int RW, bool PAIR, int JP>
static cudaError_t run_fp64_jp(nb_ctx* c, const int32_t* idx, int n_act, int jsplit, int itiles, int* occ_out)
{
    auto kern = k_force_fp64<ORDER, RW, PAIR, JP>;
    const size_t smem = (size_t)NSTAGE * JT * RW * 16;
    static bool configured = false;
    static int occ = 1;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        occ = occupancy_of(kern, smem);
        configured = true;
    }
    if (occ_out) {
        *occ_out = occ;
        return cudaSuccess;
    }
    dim3 grid(itiles, jsplit);
    kern<<<grid, FORCE_NT, smem, c->stream>>>(reinterpret_cast<const double2*>(c->jstore), idx, n_act, (int)c->n,
                                              c->ltn, c->lt0, jsplit, c->eps * c->eps, c->partial, c->sc,
                                              c->F);
    return cudaGetLastError();
}

template <int ORDER, int RW, bool PAIR>
static cudaError_t run_fp64(nb_ctx* c, const int32_t* idx, int n_act, int jsplit, int itiles, int* occ_out, int ni)
{
    switch (ni) {
    case FORCE_NT: return run_fp64_jp<ORDER, RW, PAIR, 1>(c, idx, n_act, jsplit, itiles, occ_out);
    case FORCE_NT / 4: return run_fp64_jp<ORDER, RW, PAIR, 4>(c, idx, n_act, jsplit, itiles, occ_out);
    case FORCE_NT / 32: return run_fp64_jp<ORDER, RW, PAIR, 32>(c, idx, n_act, jsplit, itiles, occ_out);
    default: return cudaErrorInvalidValue;
    }
}

// Dispatch on (computed order, stored record layout, softening mode, precision).
// occ_out != nullptr only queries the kernel's occupancy.
static cudaError_t dispatch(nb_ctx* c, int order, const int32_t* idx, int n_act, int jsplit, int itiles,
                            int* occ_out, int ni)
{
    const bool pair = c->pair_eps || !(c->eps > 0.0);
    const int so = c->order;  // stored layout
#define NB_CASE(PRECFN, RW, O)                                                                  \
    if (order == O) return pair ? PRECFN<O, RW, true>(c, idx, n_act, jsplit, itiles, occ_out, ni) \
                                : PRECFN<O, RW, false>(c, idx, n_act, jsplit, itiles, occ_out, ni);
#define NB_DISPATCH(PRECFN, RWFN)       \
    if (so == 4) {                      \
        NB_CASE(PRECFN, RWFN(4), 0)     \
        NB_CASE(PRECFN, RWFN(4), 4)     \
    } else if (so == 6) {               \
        NB_CASE(PRECFN, RWFN(6), 0)     \
        NB_CASE(PRECFN, RWFN(6), 4)     \
        NB_CASE(PRECFN, RWFN(6), 6)     \
    } else if (so == 8) {               \
        NB_CASE(PRECFN, RWFN(8), 0)     \
        NB_CASE(PRECFN, RWFN(8), 4)     \
        NB_CASE(PRECFN, RWFN(8), 6)     \
        NB_CASE(PRECFN, RWFN(8), 8)     \
    }
    const int prec = c->pred_prec >= 0 ? c->pred_prec : c->prec;
    if (prec == NB_MIXED) {
        NB_DISPATCH(run_mixed, mixed_rw)
    } else {
        NB_DISPATCH(run_fp64, fp64_rw)
    }
#undef NB_DISPATCH
#undef NB_CASE
    return cudaErrorInvalidValue;
}

int force_occupancy(nb_ctx* c, int order, int ni)
{
    int occ = 1;
    if (dispatch(c, order, nullptr, 0, 1, 1, &occ, ni) != cudaSuccess) return 1;
    return occ;
}

int force_ni(const nb_ctx* c, int64_t n_act)
{
    const int prec = c->pred_prec >= 0 ? c->pred_prec : c->prec;
    return prec == NB_MIXED ? mixed_ni(n_act) : fp64_ni(n_act);
}

cudaError_t launch_force(nb_ctx* c, int order, const int32_t* idx, int64_t n_act, int jsplit, int itiles, int ni)
{
    return dispatch(c, order, idx, (int)n_act, jsplit, itiles, nullptr, ni);
}

cudaError_t launch_force_reduce(nb_ctx* c, int order, const int32_t* idx, int64_t n_act, int jsplit)
{
    (void)idx;
    const int na = (int)n_act;
#define NB_RED(O)                                                                                              \
    k_force_reduce<ncomp(O), pot_comp(O)><<<reduce_grid(jsplit, na, ncomp(O)), RED_NT, 0, c->stream>>>(c->partial, \
                                                                                                      jsplit, na, c->F)
    switch (order) {
    case 0: NB_RED(0); break;
    case 4: NB_RED(4); break;
    case 6: NB_RED(6); break;
    case 8: NB_RED(8); break;
    default: return cudaErrorInvalidValue;
    }
#undef NB_RED
    return cudaGetLastError();
}

cudaError_t launch_parts_reduce(nb_ctx* c, int order, const double* parts, int64_t n_act, int n_parts)
{
    const int na = (int)n_act;
#define NB_RED(O)                                                                                               \
    k_force_reduce<ncomp(O), -1><<<reduce_grid(n_parts, na, ncomp(O)), RED_NT, 0, c->stream>>>(parts, n_parts, na, \
                                                                                             c->F)
    switch (order) {
    case 4: NB_RED(4); break;
    case 6: NB_RED(6); break;
    case 8: NB_RED(8); break;
    default: return cudaErrorInvalidValue;
    }
#undef NB_RED
    return cudaGetLastError();
}

// ------------------------------------------------------- device-driven cycle
template <typename K>
static int dyn_slots(nb_ctx* c, K kern, size_t smem)
{
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return c->sm_count * occupancy_of(kern, smem);
}

// Launch (or, query_only, size) the persistent force kernels of the context's
// order in the given precision: on the mixed path one for the variants of up
// to FORCE_NT i-particles per CTA (grid[0]) and one for two per thread
// (grid[1]); FP64 one kernel (both entries).
template <int O>
static cudaError_t force_dyn_o(nb_ctx* c, int* grid, bool query_only, bool mixed)
{
    const bool pair = c->pair_eps || !(c->eps > 0.0);
    const int ntiles = (int)(c->np / JT);
    if (mixed) {
        constexpr int RW = mixed_rw(O);
        const size_t smem = (size_t)NSTAGE * JT * RW * 16, smem_big = xs_smem(O, RW, 1);
        auto k1 = pair ? k_force_mixed_dyn<O, RW, true, true> : k_force_mixed_dyn<O, RW, false, true>;
        auto k2 = pair ? k_force_mixed_dyn<O, RW, true, false> : k_force_mixed_dyn<O, RW, false, false>;
        static int occ[2][2] = {{0, 0}, {0, 0}};  // [pair][big]
        int* o = occ[pair ? 1 : 0];
        if (!o[0]) o[0] = dyn_slots(c, k1, smem) / c->sm_count;
        if (!o[1]) o[1] = dyn_slots(c, k2, smem_big) / c->sm_count;
        if (query_only) {
            grid[0] = c->sm_count * o[0];
            grid[1] = c->sm_count * o[1];
            return cudaSuccess;
        }
        const float e2 = (float)(c->eps * c->eps), e2max = eps2_threshold(c->eps2_max);
        const float4* js = reinterpret_cast<const float4*>(c->jstore);
        cudaError_t e = launch_k(k1, dim3(grid[0]), dim3(FORCE_NT), smem, c->stream, c->pdl != 0, js, c->act_idx,
                                 (int)c->n, ntiles, e2, e2max, c->partial, c->sc, c->F);
        if (e != cudaSuccess) return e;
        return launch_k(k2, dim3(grid[1]), dim3(FORCE_NT), smem_big, c->stream, c->pdl != 0, js, c->act_idx,
                        (int)c->n, ntiles, e2, e2max, c->partial, c->sc, c->F);
    } else {
        constexpr int RW = fp64_rw(O);
        const size_t smem = (size_t)NSTAGE * JT * RW * 16;
        auto k = pair ? k_force_fp64_dyn<O, RW, true> : k_force_fp64_dyn<O, RW, false>;
        static int occ[2] = {0, 0};
        int& o = occ[pair ? 1 : 0];
        if (!o) o = dyn_slots(c, k, smem) / c->sm_count;
        if (query_only) {
            grid[0] = grid[1] = c->sm_count * o;
            return cudaSuccess;
        }
        return launch_k(k, dim3(grid[0]), dim3(FORCE_NT), smem, c->stream, c->pdl != 0,
                        reinterpret_cast<const double2*>(c->jstore), c->act_idx, (int)c->n, ntiles,
                        c->eps * c->eps, c->partial, c->sc, c->F);
    }
    return cudaGetLastError();
}

cudaError_t launch_force_dyn(nb_ctx* c, int* grid, bool query_only)
{
    const bool mixed = c->prec == NB_MIXED;
    if (c->order == 4) return force_dyn_o<4>(c, grid, query_only, mixed);
    if (c->order == 6) return force_dyn_o<6>(c, grid, query_only, mixed);
    return force_dyn_o<8>(c, grid, query_only, mixed);
}

// Resident CTAs the split rule plans for.  At the context's own order, those
// of the persistent kernel that runs the variant: a block then gets the same
// shape in host-driven and device-driven cycles, and a device-driven cycle
// never runs more waves than were planned (a per-launch kernel with more
// resident CTAs just finishes its waves sooner).  At other orders (start-up
// passes, energy) the per-launch kernel's.
int shape_slots(nb_ctx* c, int order, int ni, bool mixed)
{
    if (order != c->order) return c->sm_count * force_occupancy(c, order, ni);
    int g[2] = {0, 0};
    if (order == 4) force_dyn_o<4>(c, g, true, mixed);
    else if (order == 6) force_dyn_o<6>(c, g, true, mixed);
    else force_dyn_o<8>(c, g, true, mixed);
    const int s = g[mixed && ni > FORCE_NT ? 1 : 0];
    return s > 0 ? s : c->sm_count;
}

cudaError_t launch_force_reduce_dyn(nb_ctx* c)
{
    const int nb = c->sm_count * 8;
    const DevScalars* sc = c->sc;
    auto k = c->order == 4   ? k_force_reduce_dyn<ncomp(4), pot_comp(4)>
             : c->order == 6 ? k_force_reduce_dyn<ncomp(6), pot_comp(6)>
                             : k_force_reduce_dyn<ncomp(8), pot_comp(8)>;
    return launch_k(k, dim3(nb), dim3(RED_NT), 0, c->stream, c->pdl != 0, (const double*)c->partial, sc, c->F);
}

// Self-test of the bounded wait every kernel uses: one CTA waits on an
// mbarrier that expects one arrival nobody makes, with the given limit; the
// wait runs out, the kernel raises NB_ERR_TIMEOUT and returns.
__global__ void k_wait_probe(long long limit_cycles, DevScalars* sc)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0, limit_cycles);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) raise_status(sc, NB_ERR_TIMEOUT);
}

cudaError_t launch_wait_probe(nb_ctx* c, long long limit_cycles)
{
    k_wait_probe<<<1, 32, 0, c->stream>>>(limit_cycles, c->sc);
    return cudaGetLastError();
}

}  // namespace nb
