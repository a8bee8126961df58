// peak_probe.cu -- FMA-throughput microbenchmark: the measured FP32 / FP64
// CUDA-core peak that roofline fractions can be set against (beside the
// nominal SMs x lanes x 2 x clock figure).
//
// Every thread runs CHAINS independent multiply-add chains of ITERS steps
// (enough independent work to keep the pipe full at any occupancy); the
// result is stored so the chains are not removed.  Flops = 2 x chains x
// steps x threads.
#include "nb_internal.cuh"

namespace nb {
namespace {

#define PK_CUDA(call)                    \
    do {                                 \
        if ((call) != cudaSuccess) {     \
            cudaGetLastError();          \
            return NB_ERR_CUDA;          \
        }                                \
    } while (0)

constexpr int CHAINS = 8;
constexpr int ITERS = 4096;
constexpr int PNT = 256;

template <typename T>
__global__ void __launch_bounds__(PNT) k_fma_chains(T a, T b, T* out)
{
    T acc[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) acc[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int it = 0; it < ITERS; ++it) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) acc[c] = acc[c] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += acc[c];
    out[blockIdx.x * PNT + threadIdx.x] = s;
}

template <typename T>
int run(nb_ctx* c, int ctas_per_sm, double* tflops)
{
    const int grid = c->sm_count * ctas_per_sm;
    T* out = nullptr;
    PK_CUDA(cudaMalloc(&out, sizeof(T) * (size_t)grid * PNT));
    cudaEvent_t e0, e1;
    PK_CUDA(cudaEventCreate(&e0));
    PK_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int r = 0; r < 4; ++r) {  // r = 0: warm-up
        PK_CUDA(cudaEventRecord(e0, c->stream));
        k_fma_chains<T><<<grid, PNT, 0, c->stream>>>((T)0.999, (T)1e-4, out);
        PK_CUDA(cudaEventRecord(e1, c->stream));
        PK_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        PK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (r > 0 && ms < best) best = ms;
    }
    c->n_launch += 4;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    const double flops = 2.0 * CHAINS * ITERS * (double)grid * PNT;
    *tflops = flops / (best * 1e-3) / 1e12;
    return NB_OK;
}

}  // namespace
}  // namespace nb

extern "C" int nb_fma_peak(nb_ctx* c, int fp64, double* tflops)
{
    if (!c || !tflops) return NB_ERR_ARG;
    return fp64 ? nb::run<double>(c, 8, tflops) : nb::run<float>(c, 8, tflops);
}
