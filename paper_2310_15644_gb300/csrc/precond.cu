// Near-field block-Jacobi preconditioner of the GMRES inner solve.
//
// For every leaf cluster tau the 2m x 2m self block of the PMCHWT matrix,
// [[A_tt, B_tt], [-B_tt, C_tt]], is read from the stored dense item (the self
// block is always a near block) and inverted exactly (Gauss-Jordan with partial
// pivoting, FP32 complex in shared memory, one CTA per leaf); applying the
// preconditioner multiplies every leaf's J and M coefficients by its inverse.
// This is a preconditioner of the discretised operator (not part of the paper,
// whose Eq. 11 inverts the compressed matrix directly); it leaves the solution
// unchanged and only reduces the number of Krylov iterations.
#include "common.cuh"

namespace bem {

#define BJ_THREADS 256

__global__ void __launch_bounds__(BJ_THREADS)
    k_bj_build(const int* __restrict__ leaf_r0, const int* __restrict__ leaf_m, const int64_t* __restrict__ item_off,
               const c64* __restrict__ near, int64_t op_stride, const int64_t* __restrict__ inv_off,
               c64* __restrict__ inv, int* __restrict__ flag) {
    extern __shared__ c64 M[];  // N x N row-major, N = 2m
    __shared__ int s_piv[2 * BEM_MAX_LEAF];
    __shared__ c64 colk[2 * BEM_MAX_LEAF];
    __shared__ float sv[BJ_THREADS / 32];
    __shared__ int si[BJ_THREADS / 32];
    const int leaf = blockIdx.x;
    const int m = leaf_m[leaf], N = 2 * m;
    const c64* A = near + item_off[leaf];
    const c64* Bm = A + op_stride;
    const c64* C = Bm + op_stride;
    const int tid = threadIdx.x;
    // item layout: element (i, j) at 2 ((j / 2) m + i) + j mod 2
    for (int e = tid; e < m * m; e += blockDim.x) {
        const int i = e % m, j = e / m;
        const int64_t o = 2 * ((int64_t)(j >> 1) * m + i) + (j & 1);
        const c64 a = A[o], b = Bm[o], cc = C[o];
        M[i * N + j] = a;
        M[i * N + m + j] = b;
        M[(m + i) * N + j] = mk<float>(-b.re, -b.im);
        M[(m + i) * N + m + j] = cc;
    }
    __syncthreads();
    for (int k = 0; k < N; ++k) {
        // pivot: largest |M[i][k]|, i >= k (smallest index on ties)
        float bv = -1.0f;
        int bi = N;
        for (int i = k + tid; i < N; i += blockDim.x) {
            const float v = cabs2(M[i * N + k]);
            if (v > bv) {
                bv = v;
                bi = i;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float v2 = __shfl_xor_sync(0xffffffffu, bv, o);
            const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
            if (v2 > bv || (v2 == bv && i2 < bi)) {
                bv = v2;
                bi = i2;
            }
        }
        if ((tid & 31) == 0) {
            sv[tid >> 5] = bv;
            si[tid >> 5] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            float b = sv[0];
            int p = si[0];
            for (int w = 1; w < BJ_THREADS / 32; ++w)
                if (sv[w] > b || (sv[w] == b && si[w] < p)) {
                    b = sv[w];
                    p = si[w];
                }
            if (!(b > 0.0f)) {
                *flag = 1;  // singular self block: the row is left as it is
                p = k;
            }
            s_piv[k] = p;
        }
        __syncthreads();
        const int p = s_piv[k];
        if (p != k)
            for (int j = tid; j < N; j += blockDim.x) {
                const c64 t = M[k * N + j];
                M[k * N + j] = M[p * N + j];
                M[p * N + j] = t;
            }
        __syncthreads();
        const c64 piv = M[k * N + k];
        const c64 d = (cabs2(piv) > 0.0f) ? cdiv(mk<float>(1.0f, 0.0f), piv) : mk<float>(0.0f, 0.0f);
        __syncthreads();
        if (tid == 0) M[k * N + k] = mk<float>(1.0f, 0.0f);
        __syncthreads();
        for (int j = tid; j < N; j += blockDim.x) M[k * N + j] = d * M[k * N + j];
        for (int i = tid; i < N; i += blockDim.x) colk[i] = M[i * N + k];  // read before column k changes
        __syncthreads();
        for (int e = tid; e < N * N; e += blockDim.x) {
            const int i = e / N, j = e % N;
            if (i == k) continue;
            const c64 f = colk[i];
            const c64 rk = M[k * N + j];
            if (j == k)
                M[i * N + j] = mk<float>(0.0f, 0.0f) - f * rk;
            else
                M[i * N + j] = M[i * N + j] - f * rk;
        }
        __syncthreads();
    }
    // undo the row exchanges as column exchanges, in reverse order
    for (int k = N - 1; k >= 0; --k) {
        const int p = s_piv[k];
        if (p != k)
            for (int i = tid; i < N; i += blockDim.x) {
                const c64 t = M[i * N + k];
                M[i * N + k] = M[i * N + p];
                M[i * N + p] = t;
            }
        __syncthreads();
    }
    // store column-major: element (k, l) at l N + k
    c64* out = inv + inv_off[leaf];
    for (int e = tid; e < N * N; e += blockDim.x) {
        const int l = e / N, k = e % N;
        out[e] = M[k * N + l];
    }
}

// z = P^-1 x (ADJ: P^-H x) in the caller's edge order; one CTA per leaf
template <bool ADJ>
__global__ void __launch_bounds__(2 * BEM_MAX_LEAF)
    k_bj_apply(const int* __restrict__ leaf_r0, const int* __restrict__ leaf_m, const int64_t* __restrict__ perm,
               const int64_t* __restrict__ inv_off, const c64* __restrict__ inv, const c64* __restrict__ x,
               c64* __restrict__ z, int ne) {
    __shared__ c64 xs[2 * BEM_MAX_LEAF];
    const int leaf = blockIdx.x;
    const int r0 = leaf_r0[leaf], m = leaf_m[leaf], N = 2 * m;
    const int k = threadIdx.x;
    if (k < N) {
        const int64_t e = perm[r0 + (k < m ? k : k - m)];
        xs[k] = x[(k < m ? 0 : ne) + e];
    }
    __syncthreads();
    if (k >= N) return;
    const c64* Mi = inv + inv_off[leaf];
    c64 acc = mk<float>(0.0f, 0.0f);
    if (ADJ) {
        for (int l = 0; l < N; ++l) acc = acc + cconj(Mi[(int64_t)k * N + l]) * xs[l];
    } else {
        for (int l = 0; l < N; ++l) acc = acc + Mi[(int64_t)l * N + k] * xs[l];
    }
    const int64_t e = perm[r0 + (k < m ? k : k - m)];
    z[(k < m ? 0 : ne) + e] = acc;
}

cudaError_t bj_build(const int* leaf_r0, const int* leaf_m, const int64_t* item_off, int nleaf, int max_m,
                     const c64* near, int64_t op_stride, const int64_t* inv_off, c64* inv, int* flag,
                     cudaStream_t st) {
    if (nleaf <= 0) return cudaSuccess;
    const size_t smem = sizeof(c64) * (size_t)(2 * max_m) * (size_t)(2 * max_m);
    cudaFuncAttributes fa;
    BEM_CUDA_TRY(cudaFuncGetAttributes(&fa, k_bj_build));
    if (smem + fa.sharedSizeBytes > 48 * 1024)
        BEM_CUDA_TRY(cudaFuncSetAttribute(k_bj_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_bj_build<<<nleaf, BJ_THREADS, smem, st>>>(leaf_r0, leaf_m, item_off, near, op_stride, inv_off, inv, flag);
    return cudaGetLastError();
}

cudaError_t bj_apply(const int* leaf_r0, const int* leaf_m, const int64_t* perm, int nleaf, const int64_t* inv_off,
                     const c64* inv, const c64* x, c64* z, int ne, bool adjoint, cudaStream_t st) {
    if (nleaf <= 0) return cudaSuccess;
    if (adjoint)
        k_bj_apply<true><<<nleaf, 2 * BEM_MAX_LEAF, 0, st>>>(leaf_r0, leaf_m, perm, inv_off, inv, x, z, ne);
    else
        k_bj_apply<false><<<nleaf, 2 * BEM_MAX_LEAF, 0, st>>>(leaf_r0, leaf_m, perm, inv_off, inv, x, z, ne);
    return cudaGetLastError();
}

}  // namespace bem
