// nl_peak.cu -- measured arithmetic peaks of the device, the denominators of the library's
// ALU roofline fractions (the paper has no counterpart: it reports MATLAB wall times only).
//
// Each kernel runs eight independent fused multiply-add chains per thread (x <- x a + b) for
// `iters` steps on every SM (4 blocks of 256 threads per SM), so the FMA pipe is never waiting
// on a dependency; a final data-dependent store keeps the chains alive.  An FMA counts as two
// flops; a paired f32x2 FMA as four.  Times are CUDA events on the caller's stream around
// each launch, after one warm-up launch; the best of five launches is returned.
#include <algorithm>

#include "nl_internal.cuh"

namespace {

constexpr int PEAK_THREADS = 256;
constexpr int PEAK_BLOCKS_PER_SM = 4;
constexpr int PEAK_CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(PEAK_THREADS) k_peak_fma(T *out, int iters, T a, T b)
{
    T x[PEAK_CHAINS];
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
#pragma unroll 8
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) s += x[c];
    if (s == (T)-12345.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // never taken
}

__global__ void __launch_bounds__(PEAK_THREADS) k_peak_fma_f32x2(float *out, int iters, float a,
                                                                 float b)
{
    unsigned long long x[PEAK_CHAINS], av, bv;
    asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) {
        const float lo = (threadIdx.x + c) * 1e-3f, hi = (threadIdx.x + 2 * c) * 1e-3f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[c]) : "f"(lo), "f"(hi));
    }
#pragma unroll 8
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS; ++c)
            asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(av), "l"(bv));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
        s += lo + hi;
    }
    if (s == -12345.f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;     // never taken
}

}  // namespace

// Runs `launch` once untimed and five times timed; returns the best time in ms.
template <typename F>
static nl_status time_best(F launch, cudaStream_t st, float *best_ms)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    NL_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return nl_cuda_fail(cudaGetLastError(), "cudaEventCreate");
    }
    float best = 1e30f;
    cudaError_t ce = cudaSuccess;
    launch();
    for (int r = 0; r < 5 && ce == cudaSuccess; ++r) {
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        ce = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
        if (ce == cudaSuccess) best = std::min(best, ms);
    }
    if (ce == cudaSuccess) ce = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ce != cudaSuccess) return nl_cuda_fail(ce, "nl_measure_peaks");
    *best_ms = best;
    return NL_OK;
}

extern "C" nl_status nl_measure_peaks(double *fp32_tflops, double *fp32x2_tflops,
                                      double *fp64_tflops, void *stream)
{
    if (!fp32_tflops || !fp32x2_tflops || !fp64_tflops) {
        nl_set_error("nl_measure_peaks: null output");
        return NL_EINVAL;
    }
    int dev = 0, sms = 0;
    NL_CUDA_TRY(cudaGetDevice(&dev));
    NL_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t st = nl_stream(stream);
    const int blocks = sms * PEAK_BLOCKS_PER_SM;
    const double threads = (double)blocks * PEAK_THREADS;
    void *sink = nullptr;
    NL_CUDA_TRY(cudaMalloc(&sink, (size_t)blocks * PEAK_THREADS * sizeof(double)));
    const int it32 = 16384, it64 = 512;
    float ms = 0.f;
    nl_status s = time_best([&] {
        k_peak_fma<float><<<blocks, PEAK_THREADS, 0, st>>>((float *)sink, it32, 0.9999999f, 1e-7f);
    }, st, &ms);
    if (s == NL_OK) {
        *fp32_tflops = 2.0 * PEAK_CHAINS * it32 * threads / (ms * 1e-3) / 1e12;
        s = time_best([&] {
            k_peak_fma_f32x2<<<blocks, PEAK_THREADS, 0, st>>>((float *)sink, it32 / 2, 0.9999999f,
                                                               1e-7f);
        }, st, &ms);
    }
    if (s == NL_OK) {
        *fp32x2_tflops = 4.0 * PEAK_CHAINS * (it32 / 2) * threads / (ms * 1e-3) / 1e12;
        s = time_best([&] {
            k_peak_fma<double><<<blocks, PEAK_THREADS, 0, st>>>((double *)sink, it64,
                                                                0.9999999999, 1e-12);
        }, st, &ms);
    }
    if (s == NL_OK) *fp64_tflops = 2.0 * PEAK_CHAINS * it64 * threads / (ms * 1e-3) / 1e12;
    cudaFree(sink);
    return s;
}
