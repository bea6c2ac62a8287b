// nm_measure_peak: the arithmetic ceiling of this GPU for the roofline of the ALU-bound kernels (the FP64
// path).  A grid of independent fused multiply-add chains, enough warps and chains per thread to keep
// every pipe busy, timed with CUDA events on a private stream.
#include "mesh.cuh"

namespace {

constexpr int kChains = 8;     // independent chains per thread
constexpr int kThreads = 256;

__device__ float g_sink_f;
__device__ double g_sink_d;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(int iters, T seed)
{
    T a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + (T)(threadIdx.x + c);
    const T m = (T)0.999999, s = (T)1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = a[c] * m + s;
    }
    T r = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) r += a[c];
    if (r == (T)-1) {  // never true (the chains stay near 0.1): keeps them live
        if (sizeof(T) == 8) g_sink_d = (double)r;
        else g_sink_f = (float)r;
    }
}

template <typename T>
int measure(int reps, double *out)
{
    int dev = 0, sms = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int per_sm = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<T>, kThreads, 0));
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    const int iters = sizeof(T) == 8 ? 1 << 12 : 1 << 16;
    cudaStream_t st;
    CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    k_fma_chains<T><<<blocks, kThreads, 0, st>>>(iters, (T)1);  // warm-up
    CUDA_TRY(cudaEventRecord(e0, st));
    for (int r = 0; r < reps; ++r) k_fma_chains<T><<<blocks, kThreads, 0, st>>>(iters, (T)1);
    CUDA_TRY(cudaEventRecord(e1, st));
    CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    CHECK_LAUNCH();
    const double flops = 2.0 * kChains * (double)iters * kThreads * blocks * reps;
    *out = flops / (ms * 1e-3);
    return NM_OK;
}

}  // namespace

extern "C" int nm_measure_peak(int kind, int reps, double *flops_per_s)
{
    clear_error();
    if (!flops_per_s || reps < 1) return fail(NM_ERR_ARG, "flops_per_s must be non-NULL and reps >= 1");
    if (kind == 0) return measure<float>(reps, flops_per_s);
    if (kind == 1) return measure<double>(reps, flops_per_s);
    return fail(NM_ERR_ARG, "kind must be 0 (FP32) or 1 (FP64)");
}
