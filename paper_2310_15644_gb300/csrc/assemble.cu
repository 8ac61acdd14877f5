// Operator entries by quadrature: dense near blocks and adaptive cross
// approximation (ACA) of far blocks.
//
// An entry (m, n) of the PMCHWT blocks (Eq. 7 rows 2-3 and P11..P22 after Eq. 8,
// in the 3-D RWG form) sums the four triangle pairs of the two RWG supports.  A
// pair listed in the singular-pair table contributes its precomputed FP64 local
// matrix; every other pair is integrated with the 7 x 7-point product rule in the
// arithmetic of the stored operator (FP32 for complex64, FP64 for complex128),
// with coordinates taken relative to the test triangle's centroid:
//
//   T^_k += c_i c_j [ jk/(4 A A') sum w w' G (r - v_i).(r' - v_j) - j/(k A A') sum w w' G ]
//   K_k  += c_i c_j / (4 A A') sum w w' g (r - v_i).((r - r') x (r' - v_j))
//
// with G = e^{-jkR}/(4 pi R), grad G = g (r - r'), g = -(1 + jkR) e^{-jkR}/(4 pi R^3),
// c_i = +-l_i the signed edge length of the local basis.  The three stored blocks
// are A = T^_0 + eta_r T^_1, B = K_0 + K_1, C = T^_0 + T^_1 / eta_r.
//
// The far blocks are compressed into U V^H by partial-pivot ACA (the low-rank
// skeleton of Eq. 10, built here per admissible block by cross approximation
// instead of random sampling): one CTA per (block, operator), rows and columns
// evaluated by the same entry routine.
#include "common.cuh"
#include "geom.cuh"

namespace bem {

__device__ __forceinline__ int find_singular(const GeomDev& g, int a, int b) {
    int lo = g.sing_ptr[a], hi = g.sing_ptr[a + 1];
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        int v = g.sing_b[mid];
        if (v == b) return mid;
        if (v < b)
            lo = mid + 1;
        else
            hi = mid;
    }
    return -1;
}

template <typename R>
__device__ __forceinline__ R r_sqrt(R x);
template <>
__device__ __forceinline__ float r_sqrt<float>(float x) { return sqrtf(x); }
template <>
__device__ __forceinline__ double r_sqrt<double>(double x) { return sqrt(x); }

template <typename R>
__device__ __forceinline__ void r_sincos(R x, R* s, R* c);
template <>
__device__ __forceinline__ void r_sincos<float>(float x, float* s, float* c) { sincosf(x, s, c); }
template <>
__device__ __forceinline__ void r_sincos<double>(double x, double* s, double* c) { sincos(x, s, c); }

template <typename R>
__device__ __forceinline__ R r_exp(R x);
template <>
__device__ __forceinline__ float r_exp<float>(float x) { return expf(x); }
template <>
__device__ __forceinline__ double r_exp<double>(double x) { return exp(x); }

// Local integrals of one regular triangle pair for the basis functions with free
// vertices li (test) and lj (source), at k0 and k1.
//   WANT_T: ff = sum W G (r-v_i).(r'-v_j), i0 = sum W G
//   WANT_K: kk = sum W g (r-v_i).((r-r') x (r'-v_j))
template <typename R, bool WANT_T, bool WANT_K>
__device__ void regular_pair(const GeomDev& g, int a, int li, int b, int lj, cx<R> ff[2], cx<R> i0[2],
                             cx<R> kk[2]) {
    const double* oa = g.cen + 3 * a;
    R va[3][3], vb[3][3];
    for (int v = 0; v < 3; ++v)
        for (int d = 0; d < 3; ++d) {
            va[v][d] = (R)(g.tv[9 * a + 3 * v + d] - oa[d]);
            vb[v][d] = (R)(g.tv[9 * b + 3 * v + d] - oa[d]);
        }
    const R Aa = (R)g.area[a], Ab = (R)g.area[b];
    R pa[7][3], ua[7][3], wa[7];
    R pb[7][3], wbv[7][3], wb[7];
    for (int q = 0; q < 7; ++q) {
        double l0, l1, l2, w;
        rule7_d(q, l0, l1, l2, w);
        for (int d = 0; d < 3; ++d) {
            pa[q][d] = (R)l0 * va[0][d] + (R)l1 * va[1][d] + (R)l2 * va[2][d];
            ua[q][d] = pa[q][d] - va[li][d];
            pb[q][d] = (R)l0 * vb[0][d] + (R)l1 * vb[1][d] + (R)l2 * vb[2][d];
            wbv[q][d] = pb[q][d] - vb[lj][d];
        }
        wa[q] = (R)w * Aa;
        wb[q] = (R)w * Ab;
    }
    const R k0 = (R)g.k0;
    const R k1r = (R)g.k1.re, k1i = (R)g.k1.im;
    const R inv4pi = (R)(1.0 / (4.0 * BEM_PI));
    for (int s = 0; s < 2; ++s) ff[s] = i0[s] = kk[s] = mk<R>(0, 0);
#pragma unroll 1
    for (int p = 0; p < 7; ++p) {
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            R d0 = pa[p][0] - pb[q][0], d1 = pa[p][1] - pb[q][1], d2 = pa[p][2] - pb[q][2];
            R R2 = d0 * d0 + d1 * d1 + d2 * d2;
            R Rr = r_sqrt<R>(R2);
            R invR = (R)1 / Rr;
            R W = wa[p] * wb[q] * inv4pi * invR;
            R fpq = 0, kpq = 0;
            if (WANT_T) fpq = ua[p][0] * wbv[q][0] + ua[p][1] * wbv[q][1] + ua[p][2] * wbv[q][2];
            if (WANT_K) {
                // (r - v_i) . ((r - r') x (r' - v_j))
                R c0 = d1 * wbv[q][2] - d2 * wbv[q][1];
                R c1 = d2 * wbv[q][0] - d0 * wbv[q][2];
                R c2 = d0 * wbv[q][1] - d1 * wbv[q][0];
                kpq = ua[p][0] * c0 + ua[p][1] * c1 + ua[p][2] * c2;
            }
            // k0 (real)
            {
                R sn, cs;
                r_sincos<R>(k0 * Rr, &sn, &cs);
                cx<R> G = mk<R>(W * cs, -W * sn);  // W e^{-jk0R}/(4 pi R) including weights
                if (WANT_T) {
                    i0[0] = i0[0] + G;
                    ff[0] = ff[0] + fpq * G;
                }
                if (WANT_K) {
                    // g = -(1 + jkR) e^{-jkR} / (4 pi R^3)
                    R s2 = -invR * invR;
                    cx<R> one_jkR = mk<R>((R)1, k0 * Rr);
                    cx<R> gg = s2 * (one_jkR * G);
                    kk[0] = kk[0] + kpq * gg;
                }
            }
            // k1 (complex, Im k1 <= 0)
            {
                R sn, cs;
                r_sincos<R>(k1r * Rr, &sn, &cs);
                R am = r_exp<R>(k1i * Rr) * W;
                cx<R> G = mk<R>(am * cs, -am * sn);
                if (WANT_T) {
                    i0[1] = i0[1] + G;
                    ff[1] = ff[1] + fpq * G;
                }
                if (WANT_K) {
                    R s2 = -invR * invR;
                    cx<R> one_jkR = mk<R>((R)1 - k1i * Rr, k1r * Rr);
                    cx<R> gg = s2 * (one_jkR * G);
                    kk[1] = kk[1] + kpq * gg;
                }
            }
        }
    }
}

// Entries of A, B, C at RWG edges (m, n); OPS bit 0 = A, 1 = B, 2 = C.
template <typename R, int OPS>
__device__ void eval_entry(const GeomDev& g, int m, int n, cx<R> out[3]) {
    constexpr bool WT = (OPS & 5) != 0;
    constexpr bool WK = (OPS & 2) != 0;
    cx<R> T0 = mk<R>(0, 0), T1 = T0, K0 = T0, K1 = T0;
    const cx<R> jk0 = mk<R>(0, (R)g.k0);
    const cx<R> jk1 = mk<R>(-(R)g.k1.im, (R)g.k1.re);
    const cx<R> jok0 = mk<R>(0, (R)(1.0 / g.k0));
    const c128 jok1d = cdiv(mk<double>(0.0, 1.0), g.k1);
    const cx<R> jok1 = mk<R>((R)jok1d.re, (R)jok1d.im);
    for (int sa = 0; sa < 2; ++sa) {
        int a = g.edge_tri[2 * m + sa], li = g.edge_loc[2 * m + sa];
        for (int sb = 0; sb < 2; ++sb) {
            int b = g.edge_tri[2 * n + sb], lj = g.edge_loc[2 * n + sb];
            int slot = find_singular(g, a, b);
            if (slot >= 0) {
                const c128* v = g.sing_val + (int64_t)slot * 36;
                int ij = 3 * li + lj;
                if (WT) {
                    T0 = T0 + mk<R>((R)v[ij].re, (R)v[ij].im);
                    T1 = T1 + mk<R>((R)v[18 + ij].re, (R)v[18 + ij].im);
                }
                if (WK) {
                    K0 = K0 + mk<R>((R)v[9 + ij].re, (R)v[9 + ij].im);
                    K1 = K1 + mk<R>((R)v[27 + ij].re, (R)v[27 + ij].im);
                }
            } else {
                cx<R> ff[2], i0[2], kk[2];
                regular_pair<R, WT, WK>(g, a, li, b, lj, ff, i0, kk);
                double AA = g.area[a] * g.area[b];
                R cc = (R)(g.tri_coef[3 * a + li] * g.tri_coef[3 * b + lj]);
                R c4 = (R)(1.0 / (4.0 * AA)) * cc, c1 = (R)(1.0 / AA) * cc;
                if (WT) {
                    T0 = T0 + c4 * (jk0 * ff[0]) - c1 * (jok0 * i0[0]);
                    T1 = T1 + c4 * (jk1 * ff[1]) - c1 * (jok1 * i0[1]);
                }
                if (WK) {
                    K0 = K0 + c4 * kk[0];
                    K1 = K1 + c4 * kk[1];
                }
            }
        }
    }
    const cx<R> er = mk<R>((R)g.eta_r.re, (R)g.eta_r.im);
    const c128 ier = cdiv(mk<double>(1.0, 0.0), g.eta_r);
    const cx<R> ie = mk<R>((R)ier.re, (R)ier.im);
    if (OPS & 1) out[0] = T0 + er * T1;
    if (OPS & 2) out[1] = K0 + K1;
    if (OPS & 4) out[2] = T0 + ie * T1;
}

// ---------------------------------------------------------------------------
// near blocks: one CTA per block, entries written in the product layout
//   block (m x n), column pairs cp: element (i, 2cp + h) at complex index
//   off + 2 (cp m + i) + h; the A, B, C arrays are op_stride apart; an odd n is
//   padded with a zero column.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_near(GeomDev g, const int64_t* __restrict__ perm,
                                              const BlockDesc* __restrict__ blocks,
                                              const int64_t* __restrict__ entry_off, cx<R>* __restrict__ entries,
                                              int64_t op_stride) {
    BlockDesc B = blocks[blockIdx.x];
    int64_t off = entry_off[blockIdx.x];
    int npair = (B.n + 1) >> 1;
    int total = B.m * npair * 2;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        int h = e & 1;
        int rest = e >> 1;
        int i = rest % B.m;
        int cp = rest / B.m;
        int j = 2 * cp + h;
        cx<R> v[3];
        if (j < B.n) {
            int em = (int)perm[B.r0 + i], en = (int)perm[B.c0 + j];
            eval_entry<R, 7>(g, em, en, v);
        } else {
            v[0] = v[1] = v[2] = mk<R>(0, 0);
        }
        int64_t idx = off + 2 * ((int64_t)cp * B.m + i) + h;
        entries[idx] = v[0];
        entries[idx + op_stride] = v[1];
        entries[idx + 2 * op_stride] = v[2];
    }
}

template <typename R>
cudaError_t near_assemble(GeomDev g, const int64_t* perm, const BlockDesc* blocks, const int64_t* entry_off,
                          int nblocks, cx<R>* entries, int64_t op_stride, cudaStream_t st) {
    if (nblocks <= 0) return cudaSuccess;
    k_near<R><<<nblocks, 256, 0, st>>>(g, perm, blocks, entry_off, entries, op_stride);
    return cudaGetLastError();
}

template <typename R>
__global__ void k_eval(GeomDev g, const int* __restrict__ rows, const int* __restrict__ cols, int64_t count,
                       cx<R>* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    cx<R> v[3];
    eval_entry<R, 7>(g, rows[i], cols[i], v);
    out[3 * i] = v[0];
    out[3 * i + 1] = v[1];
    out[3 * i + 2] = v[2];
}

template <typename R>
cudaError_t eval_entries(GeomDev g, const int* rows, const int* cols, int64_t count, cx<R>* out,
                         cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    k_eval<R><<<(unsigned)((count + 127) / 128), 128, 0, st>>>(g, rows, cols, count, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// ACA
// ---------------------------------------------------------------------------
#define ACA_THREADS 256
#define ACA_RMAX 128

template <typename R, int OP>
__device__ __forceinline__ cx<R> entry_op(const GeomDev& g, int m, int n) {
    cx<R> v[3];
    eval_entry<R, (1 << OP)>(g, m, n, v);
    return v[OP];
}

// block-wide argmax of val with smallest index on ties; returns (val, idx) to all threads
__device__ __forceinline__ void argmax_merge(double& v, int& i, double v2, int i2) {
    if (v2 > v || (v2 == v && i2 < i)) {
        v = v2;
        i = i2;
    }
}

__device__ void block_argmax(double& v, int& i, double* sv, int* si) {
    for (int o = 16; o > 0; o >>= 1) {
        double v2 = __shfl_xor_sync(0xffffffffu, v, o);
        int i2 = __shfl_xor_sync(0xffffffffu, i, o);
        argmax_merge(v, i, v2, i2);
    }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) {
        sv[w] = v;
        si[w] = i;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bv = sv[0];
        int bi = si[0];
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) argmax_merge(bv, bi, sv[k], si[k]);
        sv[0] = bv;
        si[0] = bi;
    }
    __syncthreads();
    v = sv[0];
    i = si[0];
    __syncthreads();
}

__device__ double block_sum(double v, double* sv) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sv[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sv[k];
        sv[0] = s;
    }
    __syncthreads();
    double r = sv[0];
    __syncthreads();
    return r;
}

// Scratch of a task: U (m x rmax, column l at l*m), W (n x rmax, column l at l*n),
// the residual row (n); W = conj(V), so the block is approximated by U W^T = U V^H.
// `used` rows are kept in dynamic shared memory (m bytes).
template <typename R, int OP>
__device__ void aca_task(const GeomDev& g, const int64_t* __restrict__ perm, const AcaTask& T, cx<R>* scratch,
                         double tol, int* rank_out, int* flag_out) {
    extern __shared__ unsigned char used[];
    __shared__ cx<R> srow[ACA_RMAX];
    __shared__ double sred[ACA_THREADS / 32];
    __shared__ int sidx[ACA_THREADS / 32];
    __shared__ double scross[ACA_RMAX][4];
    const int m = T.m, n = T.n, rmax = T.rmax;
    cx<R>* U = scratch + T.scratch;
    cx<R>* W = U + (int64_t)m * rmax;
    cx<R>* row = W + (int64_t)n * rmax;
    const int tid = threadIdx.x, bs = blockDim.x;
    for (int i = tid; i < m; i += bs) used[i] = 0;
    __syncthreads();
    int i = 0, k = 0;
    double norm2 = 0.0;
    bool converged = false;
    while (k < rmax) {
        if (tid == 0) used[i] = 1;
        for (int l = tid; l < k; l += bs) srow[l] = U[(int64_t)l * m + i];
        __syncthreads();
        // residual row i
        double bv = -1.0;
        int bi = 0x7fffffff;
        const int em = (int)perm[T.r0 + i];
        for (int j = tid; j < n; j += bs) {
            cx<R> z = entry_op<R, OP>(g, em, (int)perm[T.c0 + j]);
            for (int l = 0; l < k; ++l) z = z - srow[l] * W[(int64_t)l * n + j];
            row[j] = z;
            argmax_merge(bv, bi, (double)cabs2(z), j);
        }
        block_argmax(bv, bi, sred, sidx);
        if (!(bv > 0.0)) {
            // zero residual row: move to the first unused row
            int fi = 0x7fffffff;
            for (int r = tid; r < m; r += bs)
                if (!used[r]) fi = min(fi, r);
            double dummy = 0.0;
            int f2 = fi;
            block_argmax(dummy, f2, sred, sidx);  // all values equal: picks the smallest index
            if (f2 == 0x7fffffff) {
                converged = true;
                break;
            }
            i = f2;
            continue;
        }
        const int jp = bi;
        const cx<R> piv = row[jp];
        __syncthreads();
        // w = row / pivot
        double nw2 = 0.0;
        for (int j = tid; j < n; j += bs) {
            cx<R> w = cdiv(row[j], piv);
            W[(int64_t)k * n + j] = w;
            nw2 += (double)cabs2(w);
        }
        nw2 = block_sum(nw2, sred);
        for (int l = tid; l < k; l += bs) srow[l] = W[(int64_t)l * n + jp];
        __syncthreads();
        // residual column jp
        double nu2 = 0.0;
        const int en = (int)perm[T.c0 + jp];
        for (int r = tid; r < m; r += bs) {
            cx<R> z = entry_op<R, OP>(g, (int)perm[T.r0 + r], en);
            for (int l = 0; l < k; ++l) z = z - srow[l] * U[(int64_t)l * m + r];
            U[(int64_t)k * m + r] = z;
            nu2 += (double)cabs2(z);
        }
        nu2 = block_sum(nu2, sred);  // also orders the U/W writes before the cross products
        // cross terms (u_l^H u)(w_l^H w): one warp per l
        const int wid = tid >> 5, lane = tid & 31, nwarp = bs >> 5;
        for (int l = wid; l < k; l += nwarp) {
            double ur = 0, ui = 0, wr = 0, wi = 0;
            for (int r = lane; r < m; r += 32) {
                cx<R> a = U[(int64_t)l * m + r], b = U[(int64_t)k * m + r];
                ur += (double)a.re * b.re + (double)a.im * b.im;
                ui += (double)a.re * b.im - (double)a.im * b.re;
            }
            for (int j = lane; j < n; j += 32) {
                cx<R> a = W[(int64_t)l * n + j], b = W[(int64_t)k * n + j];
                wr += (double)a.re * b.re + (double)a.im * b.im;
                wi += (double)a.re * b.im - (double)a.im * b.re;
            }
            for (int o = 16; o > 0; o >>= 1) {
                ur += __shfl_xor_sync(0xffffffffu, ur, o);
                ui += __shfl_xor_sync(0xffffffffu, ui, o);
                wr += __shfl_xor_sync(0xffffffffu, wr, o);
                wi += __shfl_xor_sync(0xffffffffu, wi, o);
            }
            if (lane == 0) {
                scross[l][0] = ur;
                scross[l][1] = ui;
                scross[l][2] = wr;
                scross[l][3] = wi;
            }
        }
        __syncthreads();
        if (tid == 0) {
            double cr = 0.0;
            for (int l = 0; l < k; ++l) cr += scross[l][0] * scross[l][2] - scross[l][1] * scross[l][3];
            sred[0] = nu2 * nw2 + 2.0 * cr;
        }
        __syncthreads();
        norm2 += sred[0];
        __syncthreads();
        ++k;
        if (sqrt(nu2 * nw2) <= tol * sqrt(fmax(norm2, 0.0))) {
            converged = true;
            break;
        }
        // next row: largest |u| among unused rows
        double cv = -1.0;
        int ci = 0x7fffffff;
        for (int r = tid; r < m; r += bs)
            if (!used[r]) argmax_merge(cv, ci, (double)cabs2(U[(int64_t)(k - 1) * m + r]), r);
        block_argmax(cv, ci, sred, sidx);
        if (ci == 0x7fffffff) {
            converged = true;
            break;
        }
        i = ci;
    }
    if (tid == 0) {
        *rank_out = k;
        *flag_out = (converged || k >= min(m, n)) ? 0 : 1;
    }
}

template <typename R>
__global__ void __launch_bounds__(ACA_THREADS) k_aca(GeomDev g, const int64_t* __restrict__ perm,
                                                     const AcaTask* __restrict__ tasks, cx<R>* scratch,
                                                     double tol, int* ranks, int* flags) {
    AcaTask T = tasks[blockIdx.x];
    if (T.op == 0)
        aca_task<R, 0>(g, perm, T, scratch, tol, ranks + blockIdx.x, flags + blockIdx.x);
    else if (T.op == 1)
        aca_task<R, 1>(g, perm, T, scratch, tol, ranks + blockIdx.x, flags + blockIdx.x);
    else
        aca_task<R, 2>(g, perm, T, scratch, tol, ranks + blockIdx.x, flags + blockIdx.x);
}

template <typename R>
cudaError_t aca_run(GeomDev g, const int64_t* perm, const AcaTask* tasks, int ntasks, cx<R>* scratch, double tol,
                    int* ranks, int* flags, cudaStream_t st, int max_m) {
    if (ntasks <= 0) return cudaSuccess;
    // dynamic shared memory: one byte per block row; opt in when it and the kernel's
    // static shared memory together pass the default 48 KiB
    size_t smem = (size_t)max_m;
    cudaFuncAttributes fa;
    BEM_CUDA_TRY(cudaFuncGetAttributes(&fa, k_aca<R>));
    if (smem + fa.sharedSizeBytes > 48 * 1024) {
        BEM_CUDA_TRY(cudaFuncSetAttribute(k_aca<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    k_aca<R><<<ntasks, ACA_THREADS, smem, st>>>(g, perm, tasks, scratch, tol, ranks, flags);
    return cudaGetLastError();
}

// Copy the rank-r factors to the product layout (an odd rank is padded with a
// zero column):
//   U  slice-major: the block's rows are cut at leaf boundaries; the slice of
//      leaf rows [ro, ro + ms) holds all column pairs kp, row i of the slice,
//      at pair index ro * kpc + kp * ms + i (kpc = padded rank / 2), so that the
//      rows kernel streams one contiguous run per (leaf, block, operator);
//   W = conj(V) column-pair-major: pair index kp * n + j, one contiguous run per
//      column pair for the V^H x kernel.
// pos_leaf_lo / pos_leaf_m give, for every tree position, its leaf's start and size.
template <typename R>
__global__ void k_compact(const AcaTask* __restrict__ tasks, const cx<R>* __restrict__ scratch,
                          const int* __restrict__ ranks, const int64_t* __restrict__ off_u,
                          const int64_t* __restrict__ off_v, cx<R>* __restrict__ arena,
                          const int* __restrict__ pos_leaf_lo, const int* __restrict__ pos_leaf_m) {
    AcaTask T = tasks[blockIdx.x];
    int r = ranks[blockIdx.x];
    int rp = r + (r & 1);
    int kpc = rp >> 1;
    const cx<R>* U = scratch + T.scratch;
    const cx<R>* W = U + (int64_t)T.m * T.rmax;
    cx<R>* Uo = arena + off_u[blockIdx.x];
    cx<R>* Vo = arena + off_v[blockIdx.x];
    int64_t nu = (int64_t)T.m * rp, nv = (int64_t)T.n * rp;
    for (int64_t e = threadIdx.x; e < nu; e += blockDim.x) {
        // source element (row i, column l) -> destination in the slice-major layout
        int i = (int)(e % T.m);
        int l = (int)(e / T.m);
        int kp = l >> 1, h = l & 1;
        int ro = pos_leaf_lo[T.r0 + i] - T.r0, ms = pos_leaf_m[T.r0 + i];
        int64_t pair = (int64_t)ro * kpc + (int64_t)kp * ms + (i - ro);
        Uo[2 * pair + h] = (l < r) ? U[(int64_t)l * T.m + i] : mk<R>(0, 0);
    }
    for (int64_t e = threadIdx.x; e < nv; e += blockDim.x) {
        int h = (int)(e & 1);
        int64_t rest = e >> 1;
        int j = (int)(rest % T.n);
        int kp = (int)(rest / T.n);
        int l = 2 * kp + h;
        Vo[e] = (l < r) ? W[(int64_t)l * T.n + j] : mk<R>(0, 0);
    }
}

template <typename R>
cudaError_t aca_compact(const AcaTask* tasks, int ntasks, const cx<R>* scratch, const int* ranks,
                        const int64_t* off_u, const int64_t* off_v, cx<R>* arena, const int* pos_leaf_lo,
                        const int* pos_leaf_m, cudaStream_t st) {
    if (ntasks <= 0) return cudaSuccess;
    k_compact<R><<<ntasks, 256, 0, st>>>(tasks, scratch, ranks, off_u, off_v, arena, pos_leaf_lo, pos_leaf_m);
    return cudaGetLastError();
}

template cudaError_t near_assemble<float>(GeomDev, const int64_t*, const BlockDesc*, const int64_t*, int, c64*,
                                          int64_t, cudaStream_t);
template cudaError_t near_assemble<double>(GeomDev, const int64_t*, const BlockDesc*, const int64_t*, int, c128*,
                                           int64_t, cudaStream_t);
template cudaError_t eval_entries<float>(GeomDev, const int*, const int*, int64_t, c64*, cudaStream_t);
template cudaError_t eval_entries<double>(GeomDev, const int*, const int*, int64_t, c128*, cudaStream_t);
template cudaError_t aca_run<float>(GeomDev, const int64_t*, const AcaTask*, int, c64*, double, int*, int*,
                                    cudaStream_t, int);
template cudaError_t aca_run<double>(GeomDev, const int64_t*, const AcaTask*, int, c128*, double, int*, int*,
                                     cudaStream_t, int);
template cudaError_t aca_compact<float>(const AcaTask*, int, const c64*, const int*, const int64_t*,
                                        const int64_t*, c64*, const int*, const int*, cudaStream_t);
template cudaError_t aca_compact<double>(const AcaTask*, int, const c128*, const int*, const int64_t*,
                                         const int64_t*, c128*, const int*, const int*, cudaStream_t);

}  // namespace bem
