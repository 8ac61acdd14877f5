// The compressed PMCHWT product y = Z x (Eq. 8's system matrix applied to a
// vector, with its far blocks in the skeleton form U V^H of Eq. 10).
//
// Data layout (all in HBM, written once by assembly):
//   near items   one per (leaf row cluster, dense column range); A, B, C arrays
//                op_stride apart; element (i, 2cp + h) at 2 (cp m + i) + h, so
//                that thread i of a 64-thread group reads one 16-byte (complex64)
//                pair per column pair and a warp reads 512 contiguous bytes;
//   far factors  per block and operator: U (m rows) and W = conj(V) (n rows),
//                the same column-pair layout; t = W^T x = V^H x.
// Kernels per product (one stream, in order):
//   1. gather  xp = x[perm]           (tree order; complex vector, L2-resident)
//   2. vhx     t_b = V_b^H xp_sigma   one CTA per far block, largest first; the
//                                      block's xp slice staged in shared memory
//   3. rows    per leaf cluster tau:  y_tau = sum_near Z_{tau,sigma} xp_sigma
//                                             + sum_far U_b[tau rows] t_b
//              with the 2x2 PMCHWT structure [[A, B], [-B, C]] (B read once,
//              used in both rows); four 64-thread groups split the leaf's items
//              and are reduced in shared memory; y written once per row, in
//              edge order (deterministic, no atomics).
#include "common.cuh"

namespace bem {

// 16-byte pair loads/stores of two consecutive complex values
template <typename R>
struct Pair;
template <>
struct Pair<float> {
    typedef float4 V;
    static __device__ __forceinline__ void ld(const void* base, int64_t idx, c64& a, c64& b) {
        float4 v = __ldg(reinterpret_cast<const float4*>(base) + idx);
        a = mk<float>(v.x, v.y);
        b = mk<float>(v.z, v.w);
    }
};
template <>
struct Pair<double> {
    static __device__ __forceinline__ void ld(const void* base, int64_t idx, c128& a, c128& b) {
        const double2* p = reinterpret_cast<const double2*>(base) + 2 * idx;
        double2 u = __ldg(p), v = __ldg(p + 1);
        a = mk<double>(u.x, u.y);
        b = mk<double>(v.x, v.y);
    }
};

template <typename R>
__global__ void k_gather(const cx<R>* __restrict__ x, const int64_t* __restrict__ perm, cx<R>* __restrict__ xp,
                         int ne) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    int64_t e = perm[i];
    xp[i] = x[e];
    xp[ne + i] = x[ne + e];
}

#define VHX_THREADS 256
#define VHX_TILE 1024

// t for one far block: items (op, kp) spread over warps, rows tiled through shared memory
template <typename R>
__global__ void __launch_bounds__(VHX_THREADS) k_vhx(const FarRec* __restrict__ far, const int* __restrict__ order,
                                                     const cx<R>* __restrict__ arena, const cx<R>* __restrict__ xp,
                                                     cx<R>* __restrict__ t, int ne) {
    __shared__ cx<R> sxJ[VHX_TILE], sxM[VHX_TILE];
    __shared__ cx<R> tacc[4 * 2 * 64];  // up to 4 segments x 128 columns (rank cap)
    const FarRec F = far[order[blockIdx.x]];
    const int kpA = (F.rk[0] + 1) >> 1, kpB = (F.rk[1] + 1) >> 1, kpC = (F.rk[2] + 1) >> 1;
    const int nitems = kpA + kpB + kpC;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = VHX_THREADS / 32;
    // t segment offsets inside tacc (in complex elements)
    const int sA = 0, sBJ = 2 * kpA, sBM = 2 * (kpA + kpB), sC = 2 * (kpA + 2 * kpB);
    const int ttot = 2 * (kpA + 2 * kpB + kpC);
    for (int e = threadIdx.x; e < ttot; e += VHX_THREADS) tacc[e] = mk<R>(0, 0);
    for (int j0 = 0; j0 < F.n; j0 += VHX_TILE) {
        const int tn = min(VHX_TILE, F.n - j0);
        __syncthreads();
        for (int j = threadIdx.x; j < tn; j += VHX_THREADS) {
            sxJ[j] = xp[F.c0 + j0 + j];
            sxM[j] = xp[ne + F.c0 + j0 + j];
        }
        __syncthreads();
        for (int it = wid; it < nitems; it += nw) {
            int op, kp;
            if (it < kpA) {
                op = 0;
                kp = it;
            } else if (it < kpA + kpB) {
                op = 1;
                kp = it - kpA;
            } else {
                op = 2;
                kp = it - kpA - kpB;
            }
            const cx<R>* V = arena + F.off_v[op];
            cx<R> a0 = mk<R>(0, 0), a1 = a0, b0 = a0, b1 = a0;
            for (int j = lane; j < tn; j += 32) {
                cx<R> w0, w1;
                Pair<R>::ld(V, (int64_t)kp * F.n + j0 + j, w0, w1);
                if (op == 0) {
                    cx<R> xj = sxJ[j];
                    cfma(a0, w0, xj);
                    cfma(a1, w1, xj);
                } else if (op == 1) {
                    cx<R> xj = sxJ[j], xm = sxM[j];
                    cfma(a0, w0, xj);
                    cfma(a1, w1, xj);
                    cfma(b0, w0, xm);
                    cfma(b1, w1, xm);
                } else {
                    cx<R> xm = sxM[j];
                    cfma(a0, w0, xm);
                    cfma(a1, w1, xm);
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                a0.re += __shfl_xor_sync(0xffffffffu, a0.re, o);
                a0.im += __shfl_xor_sync(0xffffffffu, a0.im, o);
                a1.re += __shfl_xor_sync(0xffffffffu, a1.re, o);
                a1.im += __shfl_xor_sync(0xffffffffu, a1.im, o);
                b0.re += __shfl_xor_sync(0xffffffffu, b0.re, o);
                b0.im += __shfl_xor_sync(0xffffffffu, b0.im, o);
                b1.re += __shfl_xor_sync(0xffffffffu, b1.re, o);
                b1.im += __shfl_xor_sync(0xffffffffu, b1.im, o);
            }
            if (lane == 0) {
                int s = (op == 0) ? sA : ((op == 1) ? sBJ : sC);
                tacc[s + 2 * kp] = tacc[s + 2 * kp] + a0;
                tacc[s + 2 * kp + 1] = tacc[s + 2 * kp + 1] + a1;
                if (op == 1) {
                    tacc[sBM + 2 * kp] = tacc[sBM + 2 * kp] + b0;
                    tacc[sBM + 2 * kp + 1] = tacc[sBM + 2 * kp + 1] + b1;
                }
            }
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < ttot; e += VHX_THREADS) t[F.off_t + e] = tacc[e];
}

#define ROW_GROUPS 4
#define ROW_THREADS (64 * ROW_GROUPS)

template <typename R>
__global__ void __launch_bounds__(ROW_THREADS) k_rows(MatvecPlan p, const cx<R>* __restrict__ near,
                                                      const cx<R>* __restrict__ arena,
                                                      const cx<R>* __restrict__ xp, const cx<R>* __restrict__ t,
                                                      cx<R>* __restrict__ y) {
    __shared__ cx<R> sJ[ROW_GROUPS][64], sM[ROW_GROUPS][64];
    const int leaf = blockIdx.x;
    const int r0 = p.leaf_r0[leaf], m = p.leaf_m[leaf];
    const int gi = threadIdx.x >> 6, i = threadIdx.x & 63;
    const bool act = i < m;
    const int ne = p.ne;
    cx<R> aJ = mk<R>(0, 0), aM = aJ;
    // dense items
    const int n0 = p.near_ptr[leaf], n1 = p.near_ptr[leaf + 1];
    for (int it = n0 + gi; it < n1; it += ROW_GROUPS) {
        const int c0 = p.near_c0[it], n = p.near_n[it];
        const int64_t off = p.near_off[it];
        const cx<R>* A = near + off;
        const cx<R>* B = A + p.near_op_stride;
        const cx<R>* C = B + p.near_op_stride;
        const int npair = (n + 1) >> 1;
        if (act) {
            for (int cp = 0; cp < npair; ++cp) {
                cx<R> a0, a1, b0, b1, c0v, c1v;
                const int64_t idx = (int64_t)cp * m + i;
                Pair<R>::ld(A, idx, a0, a1);
                Pair<R>::ld(B, idx, b0, b1);
                Pair<R>::ld(C, idx, c0v, c1v);
                const int j = c0 + 2 * cp;
                cx<R> xJ0 = xp[j], xM0 = xp[ne + j];
                cx<R> xJ1 = mk<R>(0, 0), xM1 = xJ1;
                if (2 * cp + 1 < n) {
                    xJ1 = xp[j + 1];
                    xM1 = xp[ne + j + 1];
                }
                cfma(aJ, a0, xJ0);
                cfma(aJ, a1, xJ1);
                cfma(aJ, b0, xM0);
                cfma(aJ, b1, xM1);
                cfma(aM, c0v, xM0);
                cfma(aM, c1v, xM1);
                cx<R> bx = b0 * xJ0;
                cfma(bx, b1, xJ1);
                aM = aM - bx;
            }
        }
    }
    // far pieces
    const int f0 = p.farp_ptr[leaf], f1 = p.farp_ptr[leaf + 1];
    for (int it = f0 + gi; it < f1; it += ROW_GROUPS) {
        const FarRec F = p.far[p.farp_blk[it]];
        const int ro = p.farp_row[it];
        if (!act) continue;
        const int kpA = (F.rk[0] + 1) >> 1, kpB = (F.rk[1] + 1) >> 1, kpC = (F.rk[2] + 1) >> 1;
        const cx<R>* tb = t + F.off_t;
        const cx<R>* tA = tb;
        const cx<R>* tBJ = tb + 2 * kpA;
        const cx<R>* tBM = tBJ + 2 * kpB;
        const cx<R>* tC = tBM + 2 * kpB;
        const cx<R>* UA = arena + F.off_u[0];
        const cx<R>* UB = arena + F.off_u[1];
        const cx<R>* UC = arena + F.off_u[2];
        for (int kp = 0; kp < kpA; ++kp) {
            cx<R> u0, u1;
            Pair<R>::ld(UA, (int64_t)kp * F.m + ro + i, u0, u1);
            cfma(aJ, u0, tA[2 * kp]);
            cfma(aJ, u1, tA[2 * kp + 1]);
        }
        for (int kp = 0; kp < kpB; ++kp) {
            cx<R> u0, u1;
            Pair<R>::ld(UB, (int64_t)kp * F.m + ro + i, u0, u1);
            cfma(aJ, u0, tBM[2 * kp]);
            cfma(aJ, u1, tBM[2 * kp + 1]);
            cx<R> bx = u0 * tBJ[2 * kp];
            cfma(bx, u1, tBJ[2 * kp + 1]);
            aM = aM - bx;
        }
        for (int kp = 0; kp < kpC; ++kp) {
            cx<R> u0, u1;
            Pair<R>::ld(UC, (int64_t)kp * F.m + ro + i, u0, u1);
            cfma(aM, u0, tC[2 * kp]);
            cfma(aM, u1, tC[2 * kp + 1]);
        }
    }
    sJ[gi][i] = aJ;
    sM[gi][i] = aM;
    __syncthreads();
    if (gi == 0 && act) {
        cx<R> J = sJ[0][i], M = sM[0][i];
        for (int g2 = 1; g2 < ROW_GROUPS; ++g2) {
            J = J + sJ[g2][i];
            M = M + sM[g2][i];
        }
        const int64_t e = p.perm[r0 + i];
        y[e] = J;
        y[ne + e] = M;
    }
}

template <typename R>
cudaError_t matvec_run(const MatvecPlan& p, const void* near_entries, const void* arena, const cx<R>* x, cx<R>* y,
                       cx<R>* xp, cx<R>* t, int nrhs, int64_t t_len, cudaStream_t st, const cudaEvent_t* ev) {
    const int64_t nn = 2 * (int64_t)p.ne;
    for (int r = 0; r < nrhs; ++r) {
        const cx<R>* xr = x + r * nn;
        cx<R>* yr = y + r * nn;
        const cudaEvent_t* e = ev ? ev + 6 * r : nullptr;
        if (e) BEM_CUDA_TRY(cudaEventRecord(e[0], st));
        k_gather<R><<<(p.ne + 255) / 256, 256, 0, st>>>(xr, p.perm, xp, p.ne);
        BEM_CUDA_TRY(cudaGetLastError());
        if (e) BEM_CUDA_TRY(cudaEventRecord(e[1], st));
        if (e) BEM_CUDA_TRY(cudaEventRecord(e[2], st));
        if (p.nfar > 0) {
            k_vhx<R><<<p.nfar, VHX_THREADS, 0, st>>>(p.far, p.far_order, (const cx<R>*)arena, xp, t, p.ne);
            BEM_CUDA_TRY(cudaGetLastError());
        }
        if (e) BEM_CUDA_TRY(cudaEventRecord(e[3], st));
        if (e) BEM_CUDA_TRY(cudaEventRecord(e[4], st));
        k_rows<R><<<p.nleaf, ROW_THREADS, 0, st>>>(p, (const cx<R>*)near_entries, (const cx<R>*)arena, xp, t, yr);
        BEM_CUDA_TRY(cudaGetLastError());
        if (e) BEM_CUDA_TRY(cudaEventRecord(e[5], st));
    }
    (void)t_len;
    return cudaSuccess;
}

template cudaError_t matvec_run<float>(const MatvecPlan&, const void*, const void*, const c64*, c64*, c64*, c64*, int,
                                       int64_t, cudaStream_t, const cudaEvent_t*);
template cudaError_t matvec_run<double>(const MatvecPlan&, const void*, const void*, const c128*, c128*, c128*,
                                        c128*, int, int64_t, cudaStream_t, const cudaEvent_t*);

}  // namespace bem
