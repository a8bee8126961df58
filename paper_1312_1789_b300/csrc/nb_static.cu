// nb_static.cu -- a force evaluation that never allocates device memory.
//
// Some callers cannot call cudaMalloc at the moment they need a force: code
// running inside another framework's memory pool or arena that forbids
// allocations outside its own allocator, code that must not allocate once a
// real-time loop has started, or a caller embedded where any allocation could
// stall or fail.  nb_force_static serves them: the caller passes every input
// and output in its own device memory, and the scratch the force kernel needs
// beyond them (the packed j-particle records, the j-split partial sums and a
// status word) lives in one fixed array compiled into the library.
//
// The array is a file-scope __device__ variable: every GPU on which this part
// of the library is loaded holds it (NB_STATIC_SCRATCH_BYTES, about 10.5 MB)
// until the process exits.  All calls on a device share it, and it keeps the
// last call's contents, so calls that overlap on the GPU (different streams,
// or different host threads) race on it; callers must order their calls.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "force_kernels.cuh"

namespace {

using namespace nb;

constexpr int64_t STATIC_MAX_N = NB_STATIC_MAX_N;           // particles (a multiple of JT)
constexpr size_t REC_MAX_BYTES = 8 * 16;                     // largest record: FP64, order 8
constexpr size_t REC_REGION = (size_t)STATIC_MAX_N * REC_MAX_BYTES;
constexpr size_t PARTIAL_DOUBLES = (size_t)1 << 20;          // j-split partial sums
constexpr size_t PARTIAL_REGION = PARTIAL_DOUBLES * sizeof(double);
constexpr size_t SCALAR_REGION = 256;
constexpr size_t SCRATCH_BYTES = REC_REGION + PARTIAL_REGION + SCALAR_REGION;
static_assert(SCRATCH_BYTES == NB_STATIC_SCRATCH_BYTES, "scratch size must match nb.h");
static_assert(sizeof(DevScalars) <= SCALAR_REGION, "the device scalars must fit their scratch region");
static_assert(STATIC_MAX_N % JT == 0, "the scratch capacity must be whole j tiles");

static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

// Device address of g_scratch per device, taken once with that device current.
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_addr[MAX_DEVICES] = {nullptr};

// The message is formatted in the caller's own buffer and stored as the
// calling thread's nb_last_error(NULL) text, so concurrent callers do not
// overwrite each other's message.
int fail(int code, const char* fmt, ...)
{
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    nb::set_global_error(buf);
    return code;
}

int scratch_address(int dev, unsigned char** out)
{
    if (dev < 0 || dev >= MAX_DEVICES) return fail(NB_ERR_ARG, "device %d beyond the supported %d", dev, MAX_DEVICES);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail(NB_ERR_CUDA, "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        }
        g_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_addr[dev]);
    return NB_OK;
}

// Pack caller arrays ([n][3] row-major) into j-particle records, the layout
// the predictor writes (here with no time advance); padding records get m = 0
// and eps2 = 1 so they contribute exact zeros.
template <int ORDER, bool MIXED>
__global__ void k_pack(const double* __restrict__ m, const double* __restrict__ eps2, const double* __restrict__ x,
                       const double* __restrict__ v, const double* __restrict__ a, const double* __restrict__ jk,
                       int n, int np, void* __restrict__ rec)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    constexpr int RW = MIXED ? mixed_rw(ORDER) : fp64_rw(ORDER);
    double xx[3] = {0, 0, 0}, vv[3] = {0, 0, 0}, aa[3] = {0, 0, 0}, kk[3] = {0, 0, 0};
    double mi = 0.0, ei = 1.0;
    if (i < n) {
        mi = m[i];
        ei = eps2[i];
        for (int c = 0; c < 3; ++c) {
            xx[c] = x[3 * i + c];
            vv[c] = v[3 * i + c];
            if (ORDER >= 6) aa[c] = a[3 * i + c];
            if (ORDER >= 8) kk[c] = jk[3 * i + c];
        }
    }
    if (MIXED) {
        float4* r = reinterpret_cast<float4*>(rec) + (size_t)i * RW;
        float hx[3], lx[3];
        for (int c = 0; c < 3; ++c) {
            hx[c] = __double2float_rn(xx[c]);
            lx[c] = __double2float_rn(xx[c] - (double)hx[c]);
        }
        r[0] = make_float4(hx[0], hx[1], hx[2], (float)mi);
        r[1] = make_float4(lx[0], lx[1], lx[2], (float)ei);
        r[2] = make_float4((float)vv[0], (float)vv[1], (float)vv[2], 0.f);
        if (ORDER >= 6) r[3] = make_float4((float)aa[0], (float)aa[1], (float)aa[2], 0.f);
        if (ORDER >= 8) r[4] = make_float4((float)kk[0], (float)kk[1], (float)kk[2], 0.f);
    } else {
        double2* r = reinterpret_cast<double2*>(rec) + (size_t)i * RW;
        r[0] = make_double2(xx[0], xx[1]);
        r[1] = make_double2(xx[2], mi);
        r[2] = make_double2(vv[0], vv[1]);
        r[3] = make_double2(vv[2], ei);
        if (ORDER >= 6) {
            r[4] = make_double2(aa[0], aa[1]);
            r[5] = make_double2(aa[2], 0.0);
        }
        if (ORDER >= 8) {
            r[6] = make_double2(kk[0], kk[1]);
            r[7] = make_double2(kk[2], 0.0);
        }
    }
}

template <typename K>
int slots_of(K kern, size_t smem, int sm_count)
{
    int occ = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, FORCE_NT, smem) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    return occ * sm_count;
}

// Same makespan rule as the context path, capped by the fixed partial region.
int choose_split(int it, int ntiles, int nc, int n_act, int slots)
{
    return makespan_split(it, ntiles, slots, (long long)(PARTIAL_DOUBLES / ((size_t)nc * (size_t)n_act)));
}

template <int ORDER, bool MIXED>
int run_static(const double* m, const double* eps2, const double* x, const double* v, const double* a,
               const double* jk, int n, const int32_t* idx, int n_act, double* out, cudaStream_t st,
               unsigned char* scratch, int sm_count)
{
    constexpr int RW = MIXED ? mixed_rw(ORDER) : fp64_rw(ORDER);
    constexpr int NC = ncomp(ORDER);
    const int np = (n + JT - 1) / JT * JT;
    unsigned char* rec = scratch;
    double* partial = reinterpret_cast<double*>(scratch + REC_REGION);
    DevScalars* sc = reinterpret_cast<DevScalars*>(scratch + REC_REGION + PARTIAL_REGION);
    // the status word starts every call at NB_OK
    if (cudaMemsetAsync(sc, 0, sizeof(DevScalars), st) != cudaSuccess) return NB_ERR_CUDA;
    k_pack<ORDER, MIXED><<<(np + 255) / 256, 256, 0, st>>>(m, eps2, x, v, a, jk, n, np, rec);
    const size_t smem = (size_t)NSTAGE * JT * RW * 16;
    const int it = (n_act + FORCE_NT - 1) / FORCE_NT;
    int js;
    if (MIXED) {
        auto kern = k_force_mixed<ORDER, RW, true, 1>;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return NB_ERR_CUDA;
        js = choose_split(it, np / JT, NC, n_act, slots_of(kern, smem, sm_count));
        kern<<<dim3(it, js), FORCE_NT, smem, st>>>(reinterpret_cast<const float4*>(rec), idx, n_act, n, np / JT, 0, js,
                                                   0.0f, INFINITY, partial, sc, nullptr);
    } else {
        auto kern = k_force_fp64<ORDER, RW, true>;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return NB_ERR_CUDA;
        js = choose_split(it, np / JT, NC, n_act, slots_of(kern, smem, sm_count));
        kern<<<dim3(it, js), FORCE_NT, smem, st>>>(reinterpret_cast<const double2*>(rec), idx, n_act, n, np / JT, 0, js,
                                                   0.0, partial, sc, nullptr);
    }
    k_force_reduce<NC, pot_comp(ORDER)><<<reduce_grid(js, n_act, NC), RED_NT, 0, st>>>(partial, js, n_act, out);
    if (cudaGetLastError() != cudaSuccess) return NB_ERR_CUDA;
    // wait for the work so that device-side argument errors are reported here
    DevScalars h;
    if (cudaMemcpyAsync(&h, sc, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess) return NB_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return NB_ERR_CUDA;
    return h.status;
}

}  // namespace

extern "C" int nb_force_static(int order, int precision, int64_t n, const double* m, const double* eps2,
                               const double* x, const double* v, const double* a, const double* jerk,
                               const int32_t* idx, int64_t n_act, double* out, void* stream)
{
    if (!(order == 4 || order == 6 || order == 8) || (precision != NB_FP64 && precision != NB_MIXED))
        return fail(NB_ERR_ARG, "order must be 4, 6 or 8 and precision NB_FP64 or NB_MIXED");
    if (n < 1 || n > STATIC_MAX_N)
        return fail(NB_ERR_ARG, "n = %lld outside [1, %lld]: the fixed scratch holds at most %lld particles",
                    (long long)n, (long long)STATIC_MAX_N, (long long)STATIC_MAX_N);
    if (n_act < 1 || n_act > n) return fail(NB_ERR_ARG, "n_act = %lld outside [1, n]", (long long)n_act);
    if (!m || !eps2 || !x || !v || !idx || !out || (order >= 6 && !a) || (order >= 8 && !jerk))
        return fail(NB_ERR_ARG, "a required pointer is NULL");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(NB_ERR_CUDA, "no usable CUDA device");
    }
    unsigned char* scratch = nullptr;
    int rc = scratch_address(dev, &scratch);
    if (rc != NB_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nn = (int)n, na = (int)n_act;
    if (precision == NB_MIXED) {
        if (order == 4) rc = run_static<4, true>(m, eps2, x, v, a, jerk, nn, idx, na, out, st, scratch, sms);
        else if (order == 6) rc = run_static<6, true>(m, eps2, x, v, a, jerk, nn, idx, na, out, st, scratch, sms);
        else rc = run_static<8, true>(m, eps2, x, v, a, jerk, nn, idx, na, out, st, scratch, sms);
    } else {
        if (order == 4) rc = run_static<4, false>(m, eps2, x, v, a, jerk, nn, idx, na, out, st, scratch, sms);
        else if (order == 6) rc = run_static<6, false>(m, eps2, x, v, a, jerk, nn, idx, na, out, st, scratch, sms);
        else rc = run_static<8, false>(m, eps2, x, v, a, jerk, nn, idx, na, out, st, scratch, sms);
    }
    if (rc == NB_ERR_CUDA) return fail(rc, "a CUDA call or launch failed");
    if (rc != NB_OK) return fail(rc, "a device kernel reported error %d (index out of range?)", rc);
    return NB_OK;
}
