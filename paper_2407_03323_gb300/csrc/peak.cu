// mot_fma_peak: the device's sustained FMA rate in FP64 or FP32, the denominator of the
// roofline of the FP64 history kernels (bound by FP64 arithmetic on this GPU, whose
// FP64 rate is a small fraction of its FP32 rate).  The paper has no counterpart.
//
// Every thread runs kChains independent accumulator chains a = a * m + c over `iters`
// iterations (independent chains hide the FMA latency; the chain values stay bounded
// because |m| < 1), so the kernel issues only FMAs; one CTA of 256 threads per SM slot
// reported by the occupancy calculator, times the SM count, keeps every FMA pipe busy.
#include "mot_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename R>
__global__ void __launch_bounds__(kThreads) k_fma(int iters, R m, R c, R* __restrict__ sink) {
    R a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (R)(threadIdx.x + k) * (R)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], m, c);
    }
    R s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == (R)-12345.0) sink[threadIdx.x] = s;   // never true; keeps the chains live
}

template <typename R>
void run(int iters, float* ms, double* flops) {
    int dev = 0, nsm = 0, per_sm = 0;
    MOT_CUDA_TRY(cudaGetDevice(&dev));
    MOT_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    MOT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma<R>, kThreads, 0));
    const int blocks = nsm * (per_sm > 0 ? per_sm : 1);
    R* sink = nullptr;
    MOT_CUDA_TRY(cudaMalloc(&sink, sizeof(R) * kThreads));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    try {
        MOT_CUDA_TRY(cudaEventCreate(&e0));
        MOT_CUDA_TRY(cudaEventCreate(&e1));
        const R m = (R)0.999, c = (R)1e-4;
        k_fma<R><<<blocks, kThreads>>>(iters / 8 + 1, m, c, sink);   // warm-up
        MOT_LAUNCH_CHECK();
        MOT_CUDA_TRY(cudaEventRecord(e0));
        k_fma<R><<<blocks, kThreads>>>(iters, m, c, sink);
        MOT_LAUNCH_CHECK();
        MOT_CUDA_TRY(cudaEventRecord(e1));
        MOT_CUDA_TRY(cudaEventSynchronize(e1));
        MOT_CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
        *flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
    } catch (...) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(sink);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
}

}  // namespace

extern "C" mot_status mot_fma_peak(int fp64, int iters, float* ms, double* flops) {
    if (!ms || !flops || iters < 1) return MOT_ERR_ARG;
    try {
        if (fp64) run<double>(iters, ms, flops);
        else run<float>(iters, ms, flops);
    } catch (const MotError& e) {
        return e.st;
    }
    return MOT_OK;
}
