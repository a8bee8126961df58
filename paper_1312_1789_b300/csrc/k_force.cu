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
                                              (int)(c->np / JT), jsplit, (float)(c->eps * c->eps),
                                              (float)c->eps2_max, c->partial, c->sc);
    return cudaGetLastError();
}

// Mixed path: one or two i-particles per thread.
template <int ORDER, int RW, bool PAIR>
static cudaError_t run_mixed(nb_ctx* c, const int32_t* idx, int n_act, int jsplit, int itiles, int* occ_out, int ipt)
{
    if (ipt == 2) return run_mixed_ipt<ORDER, RW, PAIR, 2>(c, idx, n_act, jsplit, itiles, occ_out);
    return run_mixed_ipt<ORDER, RW, PAIR, 1>(c, idx, n_act, jsplit, itiles, occ_out);
}

// FP64 path: bound by the FP64 pipe, one i-particle per thread.
template <int ORDER, int RW, bool PAIR>
static cudaError_t run_fp64(nb_ctx* c, const int32_t* idx, int n_act, int jsplit, int itiles, int* occ_out, int)
{
    auto kern = k_force_fp64<ORDER, RW, PAIR>;
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
                                              (int)(c->np / JT), jsplit, c->eps * c->eps, c->partial, c->sc);
    return cudaGetLastError();
}

// Dispatch on (computed order, stored record layout, softening mode, precision).
// occ_out != nullptr only queries the kernel's occupancy.
static cudaError_t dispatch(nb_ctx* c, int order, const int32_t* idx, int n_act, int jsplit, int itiles,
                            int* occ_out, int ipt)
{
    const bool pair = c->pair_eps || !(c->eps > 0.0);
    const int so = c->order;  // stored layout
#define NB_CASE(PRECFN, RW, O)                                                                  \
    if (order == O) return pair ? PRECFN<O, RW, true>(c, idx, n_act, jsplit, itiles, occ_out, ipt) \
                                : PRECFN<O, RW, false>(c, idx, n_act, jsplit, itiles, occ_out, ipt);
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

int force_occupancy(nb_ctx* c, int order, int ipt)
{
    int occ = 1;
    if (dispatch(c, order, nullptr, 0, 1, 1, &occ, ipt) != cudaSuccess) return 1;
    return occ;
}

int force_ipt(const nb_ctx* c, int64_t n_act)
{
    const int prec = c->pred_prec >= 0 ? c->pred_prec : c->prec;
    return (prec == NB_MIXED && n_act >= IPT2_MIN_NACT) ? 2 : 1;
}

cudaError_t launch_force(nb_ctx* c, int order, const int32_t* idx, int64_t n_act, int jsplit, int itiles, int ipt)
{
    return dispatch(c, order, idx, (int)n_act, jsplit, itiles, nullptr, ipt);
}

cudaError_t launch_force_reduce(nb_ctx* c, int order, const int32_t* idx, int64_t n_act, int jsplit)
{
    const int nt = 256;
    const int nb = (int)((n_act + nt - 1) / nt);
    const int na = (int)n_act, n = (int)c->n;
    switch (order) {
    case 0: k_force_reduce<ncomp(0), pot_comp(0)><<<nb, nt, 0, c->stream>>>(c->partial, jsplit, na, idx, c->m, c->eps2, n, c->F); break;
    case 4: k_force_reduce<ncomp(4), pot_comp(4)><<<nb, nt, 0, c->stream>>>(c->partial, jsplit, na, idx, c->m, c->eps2, n, c->F); break;
    case 6: k_force_reduce<ncomp(6), pot_comp(6)><<<nb, nt, 0, c->stream>>>(c->partial, jsplit, na, idx, c->m, c->eps2, n, c->F); break;
    case 8: k_force_reduce<ncomp(8), pot_comp(8)><<<nb, nt, 0, c->stream>>>(c->partial, jsplit, na, idx, c->m, c->eps2, n, c->F); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace nb
