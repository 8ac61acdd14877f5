// FMA throughput of this GPU in FP32 and FP64: the denominators of the
// arithmetic rooflines (quadrature and ACA assembly, the complex128 product).
// Every thread runs 8 independent chains of fused multiply-adds for a fixed
// number of steps; the clocks and power settings are left as they are.
#include "common.cuh"

namespace bem {
namespace {

constexpr int PK_CHAINS = 8;
constexpr int PK_UNROLL = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T* out, int iters, T m, T c) {
    T a[PK_CHAINS];
#pragma unroll
    for (int u = 0; u < PK_CHAINS; ++u) a[u] = (T)(threadIdx.x + u) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PK_UNROLL; ++k)
#pragma unroll
            for (int u = 0; u < PK_CHAINS; ++u) a[u] = fma(a[u], m, c);
    }
    T s = 0;
#pragma unroll
    for (int u = 0; u < PK_CHAINS; ++u) s += a[u];
    if (s == (T)-1.25) out[blockIdx.x] = s;  // never taken for these inputs; keeps the chains live
}

template <typename T>
cudaError_t run_peak(int iters, int reps, cudaStream_t st, double* tflops) {
    int dev = 0, nsm = 0;
    BEM_CUDA_TRY(cudaGetDevice(&dev));
    BEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = 8 * nsm, threads = 256;
    T* out = nullptr;
    BEM_CUDA_TRY(cudaMalloc(&out, sizeof(T) * blocks));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    double best = 0;
    for (int r = 0; r <= reps && err == cudaSuccess; ++r) {  // launch 0 warms up
        err = cudaEventRecord(e0, st);
        if (err != cudaSuccess) break;
        k_fma_peak<T><<<blocks, threads, 0, st>>>(out, iters, (T)0.999999, (T)1e-6);
        err = cudaGetLastError();
        if (err == cudaSuccess) err = cudaEventRecord(e1, st);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err == cudaSuccess && r > 0 && ms > 0) {
            const double flop = 2.0 * PK_CHAINS * PK_UNROLL * (double)iters * blocks * threads;
            best = std::max(best, flop / (ms * 1e-3) / 1e12);
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (err == cudaSuccess) *tflops = best;
    return err;
}

}  // namespace
}  // namespace bem

extern "C" bem_status bem_measure_fma_peak(int fp64, void* stream, double* tflops) {
    if (!tflops) return BEM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    // about 0.4 ms (FP32) and 1 ms (FP64) per launch on a GB300
    const cudaError_t e = fp64 ? bem::run_peak<double>(16, 5, st, tflops) : bem::run_peak<float>(512, 5, st, tflops);
    if (e == cudaErrorMemoryAllocation) return BEM_ENOMEM;
    return e == cudaSuccess ? BEM_OK : BEM_ECUDA;
}
