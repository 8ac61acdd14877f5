// Test harness: one tensor-core tile through the library's tcgen05 primitives
// (csrc/tc.cuh), D (128 x N) = A (128 x K) B^T (B: N x K), FP32 accumulation.
//   mode 0: A in tensor memory (written with tcgen05.st), B in shared memory,
//           one TF32 product of the inputs as given;
//   mode 1: A and B in shared memory, one TF32 product;
//   mode 2: A in tensor memory, three-term TF32 split of A and B in the kernel
//           (hi*hi + hi*lo + lo*hi), the arithmetic of the many-vector product.
// Shared-memory operands are K-major without swizzle: element (r, k) of an R-row
// operand at float index ((k / 4) * R + r) * 4 + k % 4, so LBO = 16 R bytes and
// SBO = 128 bytes.  One CTA of 128 threads; every wait is bounded.
#include <cuda_runtime.h>

#include <cstdio>

#include "../../paper_2310_15644_gb300/csrc/tc.cuh"

namespace {

constexpr int kSmemBytes = 128 * 1024;  // generous: every descriptor-addressed read stays inside

__global__ void __launch_bounds__(128, 1) k_tile(const float* __restrict__ A, const float* __restrict__ B,
                                                 float* __restrict__ D, int N, int K, int mode, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    float* sBh = reinterpret_cast<float*>(smem);
    float* sBl = sBh + N * K;
    float* sA = sBl + N * K;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sA + 128 * K);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(tslot, 256);
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::fence_mbar_init();
    }
    for (int e = tid; e < N * K; e += blockDim.x) {
        const int n = e / K, k = e % K;
        const int s = ((k >> 2) * N + n) * 4 + (k & 3);
        const float v = B[e];
        if (mode == 2) {
            uint32_t h, l;
            tc::tf32_split(v, h, l);
            sBh[s] = __uint_as_float(h);
            sBl[s] = __uint_as_float(l);
        } else {
            sBh[s] = v;
        }
    }
    if (mode == 1)
        for (int e = tid; e < 128 * K; e += blockDim.x) {
            const int m = e / K, k = e % K;
            sA[((k >> 2) * 128 + m) * 4 + (k & 3)] = A[e];
        }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tb = *tslot;
    const uint32_t colA = 128, colAl = 128 + K;  // D in columns [0, N), A hi / lo after it
    if (mode != 1) {
        const int m = 32 * warp + lane;  // this thread's lane = row of A
        for (int k0 = 0; k0 < K; k0 += 8) {
            uint32_t h[8], l[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float v = A[m * K + k0 + j];
                if (mode == 2) {
                    tc::tf32_split(v, h[j], l[j]);
                } else {
                    h[j] = __float_as_uint(v);
                    l[j] = 0u;
                }
            }
            tc::tmem_st8(tc::taddr(tb, 32 * warp, colA + k0), h);
            tc::tmem_st8(tc::taddr(tb, 32 * warp, colAl + k0), l);
        }
        tc::tmem_st_wait();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
        tc::fence_after_sync();
        const uint32_t id = tc::idesc_tf32(128, N);
        uint32_t acc = 0;
        for (int s = 0; s < K / 8; ++s) {
            const uint64_t bh = tc::sdesc(tc::smem_u32(sBh + s * 8 * N), 16 * N, 128);
            if (mode == 1) {
                const uint64_t ad = tc::sdesc(tc::smem_u32(sA + s * 8 * 128), 16 * 128, 128);
                tc::mma_tf32_ss(tb, ad, bh, id, acc);
                acc = 1;
            } else {
                tc::mma_tf32_ts(tb, tb + colA + 8 * s, bh, id, acc);
                acc = 1;
                if (mode == 2) {
                    const uint64_t bl = tc::sdesc(tc::smem_u32(sBl + s * 8 * N), 16 * N, 128);
                    tc::mma_tf32_ts(tb, tb + colA + 8 * s, bl, id, 1);
                    tc::mma_tf32_ts(tb, tb + colAl + 8 * s, bh, id, 1);
                }
            }
        }
        tc::mma_commit(bar);
    }
    const bool ok = tc::mbar_wait(bar, 0, 1u << 24);
    if (!ok && lane == 0) atomicExch(err, 1);
    tc::fence_after_sync();
    if (ok) {
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tc::taddr(tb, 32 * warp, c0), v);
            for (int j = 0; j < 16; ++j) D[(32 * warp + lane) * N + c0 + j] = v[j];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tb, 256);
        tc::tmem_relinquish();
    }
}

}  // namespace

// Host entry: returns 0 on success, 1 if the completion wait ran out, 2 on a CUDA
// error, 3 on unsupported sizes (N in {16, 32, ..., 128}, K in {8, 16, 24, 32}).
extern "C" int tc_tile(const float* A, const float* B, float* D, int N, int K, int mode) {
    if (N < 16 || N > 128 || N % 16 || K < 8 || K > 32 || K % 8 || mode < 0 || mode > 2) return 3;
    float *dA = nullptr, *dB = nullptr, *dD = nullptr;
    int* derr = nullptr;
    int herr = 0;
    cudaError_t e = cudaMalloc(&dA, sizeof(float) * 128 * K);
    if (e == cudaSuccess) e = cudaMalloc(&dB, sizeof(float) * N * K);
    if (e == cudaSuccess) e = cudaMalloc(&dD, sizeof(float) * 128 * N);
    if (e == cudaSuccess) e = cudaMalloc(&derr, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(dA, A, sizeof(float) * 128 * K, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dB, B, sizeof(float) * N * K, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(derr, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(dD, 0, sizeof(float) * 128 * N);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e == cudaSuccess) {
        k_tile<<<1, 128, kSmemBytes>>>(dA, dB, dD, N, K, mode, derr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(D, dD, sizeof(float) * 128 * N, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dD);
    cudaFree(derr);
    if (e != cudaSuccess) {
        fprintf(stderr, "tc_tile: %s\n", cudaGetErrorString(e));
        return 2;
    }
    return herr ? 1 : 0;
}
