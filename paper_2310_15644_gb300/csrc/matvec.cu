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
//   2. vhx     t_b = V_b^H xp_sigma   64-thread CTAs of 8 column-pair items (8 lanes
//                                      each), largest blocks first
//   3. rows    per leaf cluster tau:  y_tau = sum_near Z_{tau,sigma} xp_sigma
//                                             + sum_far U_b[tau rows] t_b
//              with the 2x2 PMCHWT structure [[A, B], [-B, C]] (B read once,
//              used in both rows); four 64-thread groups split the leaf's items
//              and are reduced in shared memory; y written once per row, in
//              edge order (deterministic, no atomics).
#include "common.cuh"

namespace bem {

// 16-byte loads of two consecutive complex values of the stored operator.  The
// operator is read once per product, so the loads are marked streaming
// (evict-first): they must not push the reused vectors (x, t) out of L1 and L2.
template <typename R>
struct Pair;
template <>
struct Pair<float> {
    static __device__ __forceinline__ void ld(const void* base, int64_t idx, c64& a, c64& b) {
        float4 v = __ldcs(reinterpret_cast<const float4*>(base) + idx);
        a = mk<float>(v.x, v.y);
        b = mk<float>(v.z, v.w);
    }
};
template <>
struct Pair<double> {
    static __device__ __forceinline__ void ld(const void* base, int64_t idx, c128& a, c128& b) {
        const double2* p = reinterpret_cast<const double2*>(base) + 2 * idx;
        double2 u = __ldcs(p), v = __ldcs(p + 1);
        a = mk<double>(u.x, u.y);
        b = mk<double>(v.x, v.y);
    }
};

// load bypassing L1 (data written by other CTAs of the same launch)
__device__ __forceinline__ c64 ld_cg(const c64* q) {
    float2 v = __ldcg(reinterpret_cast<const float2*>(q));
    return mk<float>(v.x, v.y);
}
__device__ __forceinline__ c128 ld_cg(const c128* q) {
    double2 v = __ldcg(reinterpret_cast<const double2*>(q));
    return mk<double>(v.x, v.y);
}

template <typename R>
__global__ void k_gather(const cx<R>* __restrict__ x, const int64_t* __restrict__ perm, cx<R>* __restrict__ xp,
                         int ne) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    int64_t e = perm[i];
    xp[i] = x[e];
    xp[ne + i] = x[ne + e];
}

#define VHX_THREADS 64   // 8 items of 8 lanes
#define VHX_UNROLL 4

// t = W^T x for a slice of one far block's items.  An item is one column pair kp
// of one operator's W (A and C use x_J and x_M respectively; B uses both and gives
// the two t segments of B).  Unit u covers items [8 lo, 8 lo + 8) of block b; an
// item is handled by 8 lanes (rows jj, jj+8, ...) and its t values are written by
// the group's first lane -- no shared memory, no barrier, no cross-CTA sum.
template <typename R>
__device__ __forceinline__ void vhx_unit(const FarRec* __restrict__ far, int2 un, const cx<R>* __restrict__ arena,
                                         const cx<R>* __restrict__ xp, cx<R>* __restrict__ t, int ne) {
    const FarRec* Fp = far + un.x;
    const int n = Fp->n;
    const int kpA = (Fp->rk[0] + 1) >> 1, kpB = (Fp->rk[1] + 1) >> 1, kpC = (Fp->rk[2] + 1) >> 1;
    const int it = un.y * 8 + (threadIdx.x >> 3);
    const int jj = threadIdx.x & 7;
    if (it >= kpA + kpB + kpC) return;  // whole 8-lane group leaves this unit together
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
    // column pair kp of W, all rows: pair index kp*n + row (two complex values per pair)
    const cx<R>* V = arena + Fp->off_v[op] + 2 * (int64_t)kp * n;
    const cx<R>* xs = xp + ((op == 2) ? ne : 0) + Fp->c0;  // J for A and B, M for C
    const cx<R>* xm = xp + ne + Fp->c0;
    cx<R> a0 = mk<R>(0, 0), a1 = a0, b0 = a0, b1 = a0;
    int j = jj;
    for (; j + 8 * (VHX_UNROLL - 1) < n; j += 8 * VHX_UNROLL) {
        cx<R> w0[VHX_UNROLL], w1[VHX_UNROLL];
#pragma unroll
        for (int q = 0; q < VHX_UNROLL; ++q) Pair<R>::ld(V, j + 8 * q, w0[q], w1[q]);
#pragma unroll
        for (int q = 0; q < VHX_UNROLL; ++q) {
            const cx<R> xv = xs[j + 8 * q];
            cfma(a0, w0[q], xv);
            cfma(a1, w1[q], xv);
            if (op == 1) {
                const cx<R> xv2 = xm[j + 8 * q];
                cfma(b0, w0[q], xv2);
                cfma(b1, w1[q], xv2);
            }
        }
    }
    for (; j < n; j += 8) {
        cx<R> w0, w1;
        Pair<R>::ld(V, j, w0, w1);
        const cx<R> xv = xs[j];
        cfma(a0, w0, xv);
        cfma(a1, w1, xv);
        if (op == 1) {
            const cx<R> xv2 = xm[j];
            cfma(b0, w0, xv2);
            cfma(b1, w1, xv2);
        }
    }
    // sum over the 8 lanes of the group (xor offsets stay inside the group)
    const unsigned mask = 0xffu << (threadIdx.x & 24);
    for (int o = 4; o > 0; o >>= 1) {
        a0.re += __shfl_xor_sync(mask, a0.re, o);
        a0.im += __shfl_xor_sync(mask, a0.im, o);
        a1.re += __shfl_xor_sync(mask, a1.re, o);
        a1.im += __shfl_xor_sync(mask, a1.im, o);
        b0.re += __shfl_xor_sync(mask, b0.re, o);
        b0.im += __shfl_xor_sync(mask, b0.im, o);
        b1.re += __shfl_xor_sync(mask, b1.re, o);
        b1.im += __shfl_xor_sync(mask, b1.im, o);
    }
    if (jj == 0) {
        // t segments of the block: [tA | tB(J) | tB(M) | tC], 2 values per column pair
        cx<R>* tb = t + Fp->off_t;
        const int seg = (op == 0) ? 0 : ((op == 1) ? 2 * kpA : 2 * (kpA + 2 * kpB));
        tb[seg + 2 * kp] = a0;
        tb[seg + 2 * kp + 1] = a1;
        if (op == 1) {
            tb[2 * (kpA + kpB) + 2 * kp] = b0;
            tb[2 * (kpA + kpB) + 2 * kp + 1] = b1;
        }
    }
}

// one CTA per unit; the hardware scheduler balances the (largest-first) units
template <typename R>
__global__ void __launch_bounds__(VHX_THREADS) k_vhx(const FarRec* __restrict__ far, const int2* __restrict__ units,
                                                     int nunits, const cx<R>* __restrict__ arena,
                                                     const cx<R>* __restrict__ xp, cx<R>* __restrict__ t, int ne) {
    if ((int)blockIdx.x < nunits) vhx_unit<R>(far, units[blockIdx.x], arena, xp, t, ne);
}

#define ROW_THREADS (64 * BEM_ROW_GROUPS)
#define ROW_GROUPS BEM_ROW_GROUPS
#define ROW_UNROLL 4

// One dense item (leaf rows x n columns): y_J += A xJ + B xM, y_M += C xM - B xJ.
template <typename R>
__device__ __forceinline__ void dense_item(const cx<R>* __restrict__ A, int64_t stride, int m, int i, int n,
                                           const cx<R>* __restrict__ xJ, const cx<R>* __restrict__ xM, cx<R>& aJ,
                                           cx<R>& aM) {
    const cx<R>* B = A + stride;
    const cx<R>* C = B + stride;
    const int nfull = n >> 1;  // column pairs with both columns inside the item
    int cp = 0;
    for (; cp + ROW_UNROLL <= nfull; cp += ROW_UNROLL) {
        cx<R> a0[ROW_UNROLL], a1[ROW_UNROLL], b0[ROW_UNROLL], b1[ROW_UNROLL], c0[ROW_UNROLL], c1[ROW_UNROLL];
#pragma unroll
        for (int u = 0; u < ROW_UNROLL; ++u) {
            const int64_t idx = (int64_t)(cp + u) * m + i;
            Pair<R>::ld(A, idx, a0[u], a1[u]);
            Pair<R>::ld(B, idx, b0[u], b1[u]);
            Pair<R>::ld(C, idx, c0[u], c1[u]);
        }
#pragma unroll
        for (int u = 0; u < ROW_UNROLL; ++u) {
            const int j = 2 * (cp + u);
            const cx<R> xj0 = xJ[j], xj1 = xJ[j + 1], xm0 = xM[j], xm1 = xM[j + 1];
            cfma(aJ, a0[u], xj0);
            cfma(aJ, a1[u], xj1);
            cfma(aJ, b0[u], xm0);
            cfma(aJ, b1[u], xm1);
            cfma(aM, c0[u], xm0);
            cfma(aM, c1[u], xm1);
            cx<R> bx = b0[u] * xj0;
            cfma(bx, b1[u], xj1);
            aM = aM - bx;
        }
    }
    for (; cp < nfull; ++cp) {
        cx<R> a0, a1, b0, b1, c0, c1;
        const int64_t idx = (int64_t)cp * m + i;
        Pair<R>::ld(A, idx, a0, a1);
        Pair<R>::ld(B, idx, b0, b1);
        Pair<R>::ld(C, idx, c0, c1);
        const int j = 2 * cp;
        const cx<R> xj0 = xJ[j], xj1 = xJ[j + 1], xm0 = xM[j], xm1 = xM[j + 1];
        cfma(aJ, a0, xj0);
        cfma(aJ, a1, xj1);
        cfma(aJ, b0, xm0);
        cfma(aJ, b1, xm1);
        cfma(aM, c0, xm0);
        cfma(aM, c1, xm1);
        cx<R> bx = b0 * xj0;
        cfma(bx, b1, xj1);
        aM = aM - bx;
    }
    if (n & 1) {  // last column; its pair partner is a stored zero column
        cx<R> a0, a1, b0, b1, c0, c1;
        const int64_t idx = (int64_t)nfull * m + i;
        Pair<R>::ld(A, idx, a0, a1);
        Pair<R>::ld(B, idx, b0, b1);
        Pair<R>::ld(C, idx, c0, c1);
        const cx<R> xj0 = xJ[n - 1], xm0 = xM[n - 1];
        cfma(aJ, a0, xj0);
        cfma(aJ, b0, xm0);
        cfma(aM, c0, xm0);
        aM = aM - b0 * xj0;
    }
}

// y_J += U_A tA + U_B tBM, y_M += U_C tC - U_B tBJ for rows ro + i of one far block.
// U is slice-major: the leaf's slice (ms rows starting at ro) of operator q is one
// contiguous run, pair (kp, i) at ro * kpc + kp * ms + i.
template <typename R>
__device__ __forceinline__ void far_slice(const cx<R>* __restrict__ U, int kpc, int ms, int i,
                                          const cx<R>* __restrict__ tv, const cx<R>* __restrict__ tv2, int mode,
                                          cx<R>& aJ, cx<R>& aM) {
    // mode 0: aJ += U tv; mode 1: aJ += U tv (tBM), aM -= U tv2 (tBJ); mode 2: aM += U tv
    int kp = 0;
    for (; kp + ROW_UNROLL <= kpc; kp += ROW_UNROLL) {
        cx<R> u0[ROW_UNROLL], u1[ROW_UNROLL];
#pragma unroll
        for (int u = 0; u < ROW_UNROLL; ++u) Pair<R>::ld(U, (int64_t)(kp + u) * ms + i, u0[u], u1[u]);
#pragma unroll
        for (int u = 0; u < ROW_UNROLL; ++u) {
            const int k2 = 2 * (kp + u);
            if (mode == 0) {
                cfma(aJ, u0[u], tv[k2]);
                cfma(aJ, u1[u], tv[k2 + 1]);
            } else if (mode == 1) {
                cfma(aJ, u0[u], tv[k2]);
                cfma(aJ, u1[u], tv[k2 + 1]);
                cx<R> bx = u0[u] * tv2[k2];
                cfma(bx, u1[u], tv2[k2 + 1]);
                aM = aM - bx;
            } else {
                cfma(aM, u0[u], tv[k2]);
                cfma(aM, u1[u], tv[k2 + 1]);
            }
        }
    }
    for (; kp < kpc; ++kp) {
        cx<R> u0, u1;
        Pair<R>::ld(U, (int64_t)kp * ms + i, u0, u1);
        const int k2 = 2 * kp;
        if (mode == 0) {
            cfma(aJ, u0, tv[k2]);
            cfma(aJ, u1, tv[k2 + 1]);
        } else if (mode == 1) {
            cfma(aJ, u0, tv[k2]);
            cfma(aJ, u1, tv[k2 + 1]);
            cx<R> bx = u0 * tv2[k2];
            cfma(bx, u1, tv2[k2 + 1]);
            aM = aM - bx;
        } else {
            cfma(aM, u0, tv[k2]);
            cfma(aM, u1, tv[k2 + 1]);
        }
    }
}

template <typename R>
__device__ __forceinline__ void far_piece(const FarRec& F, int ro, int ms, int i, const cx<R>* __restrict__ arena,
                                          const cx<R>* __restrict__ t, cx<R>& aJ, cx<R>& aM) {
    const int kpA = (F.rk[0] + 1) >> 1, kpB = (F.rk[1] + 1) >> 1, kpC = (F.rk[2] + 1) >> 1;
    const cx<R>* tA = t + F.off_t;
    const cx<R>* tBJ = tA + 2 * kpA;
    const cx<R>* tBM = tBJ + 2 * kpB;
    const cx<R>* tC = tBM + 2 * kpB;
    far_slice<R>(arena + F.off_u[0] + 2 * (int64_t)ro * kpA, kpA, ms, i, tA, nullptr, 0, aJ, aM);
    far_slice<R>(arena + F.off_u[1] + 2 * (int64_t)ro * kpB, kpB, ms, i, tBM, tBJ, 1, aJ, aM);
    far_slice<R>(arena + F.off_u[2] + 2 * (int64_t)ro * kpC, kpC, ms, i, tC, nullptr, 2, aJ, aM);
}

// Grid: nleaf x parts CTAs.  CTA (leaf, part) runs work slots part*4 .. part*4+3 of
// its leaf, one per 64-thread group (a balanced split of the leaf's dense items and
// far pieces made at assembly).  With one part the CTA writes y; with several, each
// writes its partial rows, and the last CTA of the leaf to finish (arrival counter,
// after a memory fence) adds the parts in index order and writes y -- the sum does
// not depend on which CTA finishes last.
template <typename R>
__global__ void __launch_bounds__(ROW_THREADS) k_rows(MatvecPlan p, const cx<R>* __restrict__ near,
                                                      const cx<R>* __restrict__ arena,
                                                      const cx<R>* __restrict__ xp, const cx<R>* __restrict__ t,
                                                      cx<R>* __restrict__ y, cx<R>* __restrict__ ypart,
                                                      unsigned int* __restrict__ arrive) {
    __shared__ cx<R> sJ[ROW_GROUPS][64], sM[ROW_GROUPS][64];
    __shared__ bool s_last;
    const int P = p.parts;
    const int leaf = blockIdx.x / P, part = blockIdx.x % P;
    const int r0 = p.leaf_r0[leaf], m = p.leaf_m[leaf];
    const int gi = threadIdx.x >> 6, i = threadIdx.x & 63;
    const bool act = i < m;
    const int ne = p.ne;
    cx<R> aJ = mk<R>(0, 0), aM = aJ;
    const int slot = (leaf * P + part) * ROW_GROUPS + gi;
    const int w0 = p.work_ptr[slot], w1 = p.work_ptr[slot + 1];
    if (act) {
        for (int w = w0; w < w1; ++w) {
            const int item = p.work_item[w];
            if (item >= 0) {
                const int c0 = p.near_c0[item];
                dense_item<R>(near + p.near_off[item], p.near_op_stride, m, i, p.near_n[item], xp + c0,
                              xp + ne + c0, aJ, aM);
            } else {
                const int fp = -1 - item;
                const FarRec F = p.far[p.farp_blk[fp]];
                far_piece<R>(F, p.farp_row[fp], m, i, arena, t, aJ, aM);
            }
        }
    }
    sJ[gi][i] = aJ;
    sM[gi][i] = aM;
    __syncthreads();
    cx<R> J = mk<R>(0, 0), M = J;
    if (gi == 0) {
        J = sJ[0][i];
        M = sM[0][i];
        for (int g2 = 1; g2 < ROW_GROUPS; ++g2) {
            J = J + sJ[g2][i];
            M = M + sM[g2][i];
        }
    }
    if (P == 1) {
        if (gi == 0 && act) {
            const int64_t e = p.perm[r0 + i];
            y[e] = J;
            y[ne + e] = M;
        }
        return;
    }
    const int64_t nn = 2 * (int64_t)ne;
    if (gi == 0 && act) {
        ypart[part * nn + r0 + i] = J;
        ypart[part * nn + ne + r0 + i] = M;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(arrive + leaf, 1u) == (unsigned)(P - 1));
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (gi == 0 && act) {
        cx<R> sj = mk<R>(0, 0), sm = sj;
        for (int q = 0; q < P; ++q) {
            sj = sj + ld_cg(ypart + q * nn + r0 + i);
            sm = sm + ld_cg(ypart + q * nn + ne + r0 + i);
        }
        const int64_t e = p.perm[r0 + i];
        y[e] = sj;
        y[ne + e] = sm;
    }
    if (threadIdx.x == 0) arrive[leaf] = 0u;  // ready for the next product
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
        if (p.nvhx > 0) {
            k_vhx<R><<<p.nvhx, VHX_THREADS, 0, st>>>(p.far, p.vhx_units, p.nvhx, (const cx<R>*)arena, xp, t, p.ne);
            BEM_CUDA_TRY(cudaGetLastError());
        }
        if (e) BEM_CUDA_TRY(cudaEventRecord(e[3], st));
        if (e) BEM_CUDA_TRY(cudaEventRecord(e[4], st));
        k_rows<R><<<p.nleaf * p.parts, ROW_THREADS, 0, st>>>(p, (const cx<R>*)near_entries, (const cx<R>*)arena, xp,
                                                              t, yr, (cx<R>*)p.ypart, p.arrive);
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
