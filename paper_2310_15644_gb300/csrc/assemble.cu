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
// skeleton of Eq. 17, built here per admissible block by cross approximation
// instead of random sampling): one CTA per (block, operator), rows and columns
// evaluated by the same entry routine.
#include "common.cuh"
#include "geom.cuh"

namespace bem {


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

// Geometry of a triangle pair (a test, b source) in the arithmetic R, with
// coordinates relative to a's centroid: vertices va, vb; areas; edge coefficients
// of the local bases (ca, cb); the squared centroid distance d2 and the larger
// longest edge dm (for the singular-pair test).
template <typename R>
struct PairGeom {
    R va[3][3], vb[3][3];
    R Aa, Ab, inv_AA;
    R ca[3], cb[3];
    R d2, dm;
};

template <typename R>
__device__ __forceinline__ void pair_geom(const GeomDev& g, int a, int b, PairGeom<R>& P);

template <>
__device__ __forceinline__ void pair_geom<float>(const GeomDev& g, int a, int b, PairGeom<float>& P) {
    const TriF* ta = g.trif + a;
    const TriF* tb = g.trif + b;
    const float4 ha = ta->c_hi, la = ta->c_lo, hb = tb->c_hi, lb = tb->c_lo;
    // centroid difference from the high and low parts
    const float dx = (hb.x - ha.x) + (lb.x - la.x);
    const float dy = (hb.y - ha.y) + (lb.y - la.y);
    const float dz = (hb.z - ha.z) + (lb.z - la.z);
    for (int v = 0; v < 3; ++v) {
        const float4 pa = ta->v[v], pb = tb->v[v];
        P.va[v][0] = pa.x;
        P.va[v][1] = pa.y;
        P.va[v][2] = pa.z;
        P.vb[v][0] = pb.x + dx;
        P.vb[v][1] = pb.y + dy;
        P.vb[v][2] = pb.z + dz;
    }
    const float4 ka = ta->coef, kb = tb->coef;
    P.Aa = ha.w;
    P.Ab = hb.w;
    P.inv_AA = ka.w * kb.w;
    P.ca[0] = ka.x;
    P.ca[1] = ka.y;
    P.ca[2] = ka.z;
    P.cb[0] = kb.x;
    P.cb[1] = kb.y;
    P.cb[2] = kb.z;
    P.d2 = dx * dx + dy * dy + dz * dz;
    P.dm = fmaxf(la.w, lb.w);
}

template <>
__device__ __forceinline__ void pair_geom<double>(const GeomDev& g, int a, int b, PairGeom<double>& P) {
    const double* oa = g.cen + 3 * a;
    for (int v = 0; v < 3; ++v)
        for (int d = 0; d < 3; ++d) {
            P.va[v][d] = g.tv[9 * a + 3 * v + d] - oa[d];
            P.vb[v][d] = g.tv[9 * b + 3 * v + d] - oa[d];
        }
    P.Aa = g.area[a];
    P.Ab = g.area[b];
    P.inv_AA = 1.0 / (P.Aa * P.Ab);
    for (int i = 0; i < 3; ++i) {
        P.ca[i] = g.tri_coef[3 * a + i];
        P.cb[i] = g.tri_coef[3 * b + i];
    }
    double dx = g.cen[3 * b] - oa[0], dy = g.cen[3 * b + 1] - oa[1], dz = g.cen[3 * b + 2] - oa[2];
    P.d2 = dx * dx + dy * dy + dz * dz;
    P.dm = fmax(g.diam[a], g.diam[b]);
}

// Local integrals of one regular triangle pair for the basis functions with free
// vertices li (test) and lj (source), at k0 and k1, over the test points
// p_lo <= p < p_hi of the 7-point rule (all 7 source points):
//   WANT_T: ff = sum W G (r-v_i).(r'-v_j), i0 = sum W G
//   WANT_K: kk = sum W g (r-v_i).((r-r') x (r'-v_j))
template <typename R, bool WANT_T, bool WANT_K>
__device__ __forceinline__ void regular_pair(const PairGeom<R>& P, const MediaConst<R>& M, int li, int lj, int p_lo,
                                             int p_hi, cx<R> ff[2], cx<R> i0[2], cx<R> kk[2]) {
    R pb[7][3], wbv[7][3], wb[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        R l0, l1, l2, w;
        rule7<R>(q, l0, l1, l2, w);
        for (int d = 0; d < 3; ++d) {
            pb[q][d] = l0 * P.vb[0][d] + l1 * P.vb[1][d] + l2 * P.vb[2][d];
            wbv[q][d] = pb[q][d] - P.vb[lj][d];
        }
        wb[q] = w * P.Ab;
    }
    const R k0 = M.k0, k1r = M.k1r, k1i = M.k1i;
    const R inv4pi = (R)(1.0 / (4.0 * BEM_PI));
    for (int s = 0; s < 2; ++s) ff[s] = i0[s] = kk[s] = mk<R>(0, 0);
#pragma unroll 1
    for (int p = p_lo; p < p_hi; ++p) {
        R pa[3], ua[3], wa;
        {
            R l0, l1, l2, w;
            rule7<R>(p, l0, l1, l2, w);
            for (int d = 0; d < 3; ++d) {
                pa[d] = l0 * P.va[0][d] + l1 * P.va[1][d] + l2 * P.va[2][d];
                ua[d] = pa[d] - P.va[li][d];
            }
            wa = w * P.Aa;
        }
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            R d0 = pa[0] - pb[q][0], d1 = pa[1] - pb[q][1], d2 = pa[2] - pb[q][2];
            R R2 = d0 * d0 + d1 * d1 + d2 * d2;
            R Rr = r_sqrt<R>(R2);
            R invR = (R)1 / Rr;
            R W = wa * wb[q] * inv4pi * invR;
            R fpq = 0, kpq = 0;
            if (WANT_T) fpq = ua[0] * wbv[q][0] + ua[1] * wbv[q][1] + ua[2] * wbv[q][2];
            if (WANT_K) {
                // (r - v_i) . ((r - r') x (r' - v_j))
                R c0 = d1 * wbv[q][2] - d2 * wbv[q][1];
                R c1 = d2 * wbv[q][0] - d0 * wbv[q][2];
                R c2 = d0 * wbv[q][1] - d1 * wbv[q][0];
                kpq = ua[0] * c0 + ua[1] * c1 + ua[2] * c2;
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

// T^_0, T^_1, K_0, K_1 contributions of the triangle pair (a with local basis li,
// b with lj) over test points [p_lo, p_hi): the singular-pair table's FP64 local
// matrix when the pair is listed (counted once, by the call with p_lo == 0), else
// the product rule.  Only pairs whose centroids are closer than twice the larger
// longest edge (with a margin for rounding) can be listed, so the table search is
// skipped for the others.
template <typename R, bool WT, bool WK>
__device__ __forceinline__ void pair_terms(const GeomDev& g, int a, int li, int b, int lj, int p_lo, int p_hi,
                                           cx<R>& T0, cx<R>& T1, cx<R>& K0, cx<R>& K1) {
    PairGeom<R> P;
    pair_geom<R>(g, a, b, P);
    const R lim = (R)2 * P.dm;
    const int slot = (P.d2 > lim * lim * (R)1.001) ? -1 : find_singular(g, a, b);
    if (slot >= 0) {
        if (p_lo != 0) return;
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
        return;
    }
    const MediaConst<R>& M = media<R>(g);
    cx<R> ff[2], i0[2], kk[2];
    regular_pair<R, WT, WK>(P, M, li, lj, p_lo, p_hi, ff, i0, kk);
    const R cc = P.ca[li] * P.cb[lj];
    const R c1 = P.inv_AA * cc, c4 = (R)0.25 * c1;
    if (WT) {
        T0 = T0 + c4 * (M.jk0 * ff[0]) - c1 * (M.jok0 * i0[0]);
        T1 = T1 + c4 * (M.jk1 * ff[1]) - c1 * (M.jok1 * i0[1]);
    }
    if (WK) {
        K0 = K0 + c4 * kk[0];
        K1 = K1 + c4 * kk[1];
    }
}

// A = T^_0 + eta_r T^_1, B = K_0 + K_1, C = T^_0 + T^_1 / eta_r; for one region of a
// layered body (w0 = 0) the k1 medium alone: A = eta_r T^_1, B = K_1, C = T^_1 / eta_r
template <typename R>
__device__ __forceinline__ void combine_ops(const GeomDev& g, int ops, cx<R> T0, cx<R> T1, cx<R> K0, cx<R> K1,
                                            cx<R> out[3]) {
    const MediaConst<R>& M = media<R>(g);
    if (M.w0 == (R)0) {
        if (ops & 1) out[0] = M.er * T1;
        if (ops & 2) out[1] = K1;
        if (ops & 4) out[2] = M.ie * T1;
        return;
    }
    if (ops & 1) out[0] = T0 + M.er * T1;
    if (ops & 2) out[1] = K0 + K1;
    if (ops & 4) out[2] = T0 + M.ie * T1;
}

// Entries of A, B, C at RWG edges (m, n); OPS bit 0 = A, 1 = B, 2 = C.  One thread.
template <typename R, int OPS>
__device__ void eval_entry(const GeomDev& g, int m, int n, cx<R> out[3]) {
    constexpr bool WT = (OPS & 5) != 0;
    constexpr bool WK = (OPS & 2) != 0;
    cx<R> T0 = mk<R>(0, 0), T1 = T0, K0 = T0, K1 = T0;
    for (int sa = 0; sa < 2; ++sa) {
        int a = g.edge_tri[2 * m + sa], li = g.edge_loc[2 * m + sa];
        for (int sb = 0; sb < 2; ++sb) {
            int b = g.edge_tri[2 * n + sb], lj = g.edge_loc[2 * n + sb];
            pair_terms<R, WT, WK>(g, a, li, b, lj, 0, 7, T0, T1, K0, K1);
        }
    }
    combine_ops<R>(g, OPS, T0, T1, K0, K1, out);
}

// Entry (m, n) of operator OP (0 = A, 1 = B, 2 = C) by one warp: lane L < 28 takes
// the triangle pair (L / 14, (L / 7) mod 2) of the two supports at test point
// L mod 7; the warp's sum, returned to every lane, is the entry.
template <typename R, int OP>
__device__ __forceinline__ cx<R> entry_warp(const GeomDev& g, int m, int n, int lane) {
    constexpr bool WT = OP != 1, WK = OP == 1;
    cx<R> T0 = mk<R>(0, 0), T1 = T0, K0 = T0, K1 = T0;
    if (lane < 28) {
        const int sa = lane / 14, sb = (lane / 7) & 1, p = lane % 7;
        const int a = g.edge_tri[2 * m + sa], li = g.edge_loc[2 * m + sa];
        const int b = g.edge_tri[2 * n + sb], lj = g.edge_loc[2 * n + sb];
        pair_terms<R, WT, WK>(g, a, li, b, lj, p, p + 1, T0, T1, K0, K1);
    }
    cx<R> out[3];
    combine_ops<R>(g, 1 << OP, T0, T1, K0, K1, out);
    cx<R> v = out[OP];
    for (int o = 16; o > 0; o >>= 1) {
        v.re += __shfl_xor_sync(0xffffffffu, v.re, o);
        v.im += __shfl_xor_sync(0xffffffffu, v.im, o);
    }
    return v;
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
#define ACA_THREADS_WIDE 1024
#define ACA_MAX_CHECKS 8      // sampled-row checks per task before the stopping test is accepted
#define ACA_CHECK_FACTOR 4.0  // a checked row resumes the iteration above 4x its share of the tolerance
#define ACA_RMAX 128

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
    __shared__ double sred[32];
    __shared__ int sidx[32];
    __shared__ double scross[ACA_RMAX][4];
    __shared__ int vis[ACA_RMAX + ACA_MAX_CHECKS + 1];  // rows visited (pivot, zero or checked), ascending
    __shared__ int nvis, s_check;
    const int m = T.m, n = T.n, rmax = T.rmax;
    cx<R>* U = scratch + T.scratch;
    cx<R>* W = U + (int64_t)m * rmax;
    cx<R>* row = W + (int64_t)n * rmax;
    const int tid = threadIdx.x, bs = blockDim.x;
    const int wid = tid >> 5, lane = tid & 31, nwarp = bs >> 5;
    for (int i = tid; i < m; i += bs) used[i] = 0;
    if (tid == 0) nvis = 0;
    __syncthreads();
    // mark row r visited (thread 0; callers synchronise); the ordered list keeps the
    // first rows visited if it fills up (only the choice of check rows uses it)
    auto visit = [&](int r) {
        if (used[r]) return;
        used[r] = 1;
        if (nvis >= ACA_RMAX + ACA_MAX_CHECKS + 1) return;
        int q = nvis++;
        while (q > 0 && vis[q - 1] > r) {
            vis[q] = vis[q - 1];
            --q;
        }
        vis[q] = r;
    };
    // residual of row r after k terms into row[]; returns its squared norm and the
    // position and size of its largest entry (all threads)
    auto residual_row = [&](int r, int kk, double& bv, int& bi) -> double {
        for (int l = tid; l < kk; l += bs) srow[l] = U[(int64_t)l * m + r];
        __syncthreads();
        const int em = (int)perm[T.r0 + r];
        for (int j = wid; j < n; j += nwarp) {
            cx<R> z = entry_warp<R, OP>(g, em, (int)perm[T.c0 + j], lane);
            if (lane == 0) row[j] = z;
        }
        __syncthreads();
        bv = -1.0;
        bi = 0x7fffffff;
        double e2 = 0.0;
        for (int j = tid; j < n; j += bs) {
            cx<R> z = row[j];
#pragma unroll 4
            for (int l = 0; l < kk; ++l) z = z - srow[l] * W[(int64_t)l * n + j];
            row[j] = z;
            const double a2 = (double)cabs2(z);
            e2 += a2;
            argmax_merge(bv, bi, a2, j);
        }
        block_argmax(bv, bi, sred, sidx);
        return block_sum(e2, sred);
    };
    int i = 0, k = 0, checks = 0;
    double norm2 = 0.0;
    bool converged = false;
    while (k < rmax) {
        if (tid == 0) visit(i);
        __syncthreads();
        // residual row i: entries by warps, then the rank-k update by threads
        double bv;
        int bi;
        residual_row(i, k, bv, bi);
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
        for (int r = wid; r < m; r += nwarp) {
            cx<R> z = entry_warp<R, OP>(g, (int)perm[T.r0 + r], en, lane);
            if (lane == 0) U[(int64_t)k * m + r] = z;
        }
        __syncthreads();
        for (int r = tid; r < m; r += bs) {
            cx<R> z = U[(int64_t)k * m + r];
#pragma unroll 4
            for (int l = 0; l < k; ++l) z = z - srow[l] * U[(int64_t)l * m + r];
            U[(int64_t)k * m + r] = z;
            nu2 += (double)cabs2(z);
        }
        nu2 = block_sum(nu2, sred);  // also orders the U/W writes before the cross products
        // cross terms (u_l^H u)(w_l^H w): one warp per l
        for (int l = wid; l < k; l += nwarp) {
            // per-lane sums in the factors' arithmetic, across lanes in FP64 (the sums
            // only steer the stopping test)
            R ur_ = 0, ui_ = 0, wr_ = 0, wi_ = 0;
            for (int r = lane; r < m; r += 32) {
                cx<R> a = U[(int64_t)l * m + r], b = U[(int64_t)k * m + r];
                ur_ += a.re * b.re + a.im * b.im;
                ui_ += a.re * b.im - a.im * b.re;
            }
            for (int j = lane; j < n; j += 32) {
                cx<R> a = W[(int64_t)l * n + j], b = W[(int64_t)k * n + j];
                wr_ += a.re * b.re + a.im * b.im;
                wi_ += a.re * b.im - a.im * b.re;
            }
            double ur = ur_, ui = ui_, wr = wr_, wi = wi_;
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
            // The partial-pivot criterion only sees the rows it has visited: a block
            // whose entries vanish on a sub-block (the double-layer kernel between
            // coplanar faces of a box, say) can look converged while a whole group
            // of rows is still missing.  Before stopping, the residual of the unvisited
            // row farthest (in tree order) from every visited row is computed; if
            // its energy exceeds ACA_CHECK_FACTOR times the per-row share
            // tol^2 |S|^2 / m of the tolerance, that row becomes the next pivot row.
            int resume = -1;
            while (resume < 0 && checks < ACA_MAX_CHECKS) {
                if (tid == 0) {
                    int best = -1, bd = 0;
                    if (vis[0] > 0) {
                        best = 0;
                        bd = vis[0];
                    }
                    for (int q = 0; q + 1 < nvis; ++q) {
                        const int gap = vis[q + 1] - vis[q];
                        if (gap >= 2 && gap / 2 > bd) {
                            best = vis[q] + gap / 2;
                            bd = gap / 2;
                        }
                    }
                    if (vis[nvis - 1] < m - 1 && m - 1 - vis[nvis - 1] > bd) best = m - 1;
                    s_check = best;
                    if (best >= 0) visit(best);
                }
                __syncthreads();
                const int ic = s_check;
                if (ic < 0) break;
                ++checks;
                double cv;
                int ci;
                const double e2 = residual_row(ic, k, cv, ci);
                if (e2 > ACA_CHECK_FACTOR * tol * tol * fmax(norm2, 0.0) / m) resume = ic;
            }
            if (resume < 0) {
                converged = true;
                break;
            }
            i = resume;
            continue;
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

// CTAs per SM the register budget is sized for: the FP32 kernel fits 64 registers
// per thread (four 256-thread CTAs per SM); the FP64 one keeps its registers.
template <typename R>
struct AcaOccupancy {
    static constexpr int ctas = 1;
};
template <>
struct AcaOccupancy<float> {
    static constexpr int ctas = 4;
};

// One CTA per task; one kernel per operator keeps each kernel's code small.
template <typename R, int OP>
__global__ void __launch_bounds__(ACA_THREADS, AcaOccupancy<R>::ctas)
    k_aca(GeomDev g, const int64_t* __restrict__ perm, const AcaTask* __restrict__ tasks, cx<R>* scratch, double tol,
          int* ranks, int* flags) {
    AcaTask T = tasks[blockIdx.x];
    aca_task<R, OP>(g, perm, T, scratch, tol, ranks + blockIdx.x, flags + blockIdx.x);
}

// The same with a whole SM (1024 threads) per task, for the few largest blocks:
// a batch holds few of them, and each one's rows and columns are long enough to
// keep 32 warps busy.  FP32 only.
template <int OP>
__global__ void __launch_bounds__(ACA_THREADS_WIDE, 1)
    k_aca_wide(GeomDev g, const int64_t* __restrict__ perm, const AcaTask* __restrict__ tasks, c64* scratch,
               double tol, int* ranks, int* flags) {
    AcaTask T = tasks[blockIdx.x];
    aca_task<float, OP>(g, perm, T, scratch, tol, ranks + blockIdx.x, flags + blockIdx.x);
}

template <typename K>
static cudaError_t aca_smem_optin(K kernel, size_t smem) {
    // dynamic shared memory: one byte per block row; opt in when it and the kernel's
    // static shared memory together pass the default 48 KiB
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e == cudaSuccess && smem + fa.sharedSizeBytes > 48 * 1024)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e;
}

template <typename R, int OP>
static cudaError_t aca_launch(GeomDev g, const int64_t* perm, const AcaTask* tasks, int ntasks, cx<R>* scratch,
                              double tol, int* ranks, int* flags, cudaStream_t st, size_t smem, bool wide) {
    if (ntasks <= 0) return cudaSuccess;
    if constexpr (sizeof(R) == 4) {
        if (wide) {
            BEM_CUDA_TRY(aca_smem_optin(k_aca_wide<OP>, smem));
            k_aca_wide<OP><<<ntasks, ACA_THREADS_WIDE, smem, st>>>(g, perm, tasks, scratch, tol, ranks, flags);
            return cudaGetLastError();
        }
    }
    if (wide) return cudaErrorInvalidValue;
    BEM_CUDA_TRY(aca_smem_optin(k_aca<R, OP>, smem));
    k_aca<R, OP><<<ntasks, ACA_THREADS, smem, st>>>(g, perm, tasks, scratch, tol, ranks, flags);
    return cudaGetLastError();
}

// Tasks are grouped as counts[6]: wide A, B, C (FP32 only), then ordinary A, B, C.
// The wide kernels run on a second stream beside the ordinary ones.
template <typename R>
cudaError_t aca_run(GeomDev g, const int64_t* perm, const AcaTask* tasks, const int counts[6], cx<R>* scratch,
                    double tol, int* ranks, int* flags, cudaStream_t st, int max_m) {
    const size_t smem = (size_t)max_m;
    int off[7] = {0};
    for (int q = 0; q < 6; ++q) off[q + 1] = off[q] + counts[q];
    const bool any_wide = off[3] > 0, any_norm = off[6] > off[3];
    cudaStream_t side = st;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaError_t e = cudaSuccess;
    if (any_wide && any_norm) {
        e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev_fork, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ev_fork, 0);
    }
    for (int q = 0; q < 6 && e == cudaSuccess; ++q) {
        const bool wide = q < 3;
        const int op = q % 3;
        cudaStream_t s = wide ? side : st;
        const AcaTask* tq = tasks + off[q];
        int *rq = ranks + off[q], *fq = flags + off[q];
        if (op == 0) e = aca_launch<R, 0>(g, perm, tq, counts[q], scratch, tol, rq, fq, s, smem, wide);
        if (op == 1) e = aca_launch<R, 1>(g, perm, tq, counts[q], scratch, tol, rq, fq, s, smem, wide);
        if (op == 2) e = aca_launch<R, 2>(g, perm, tq, counts[q], scratch, tol, rq, fq, s, smem, wide);
    }
    if (side != st) {
        if (e == cudaSuccess) e = cudaEventRecord(ev_join, side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev_join, 0);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        cudaStreamDestroy(side);
    }
    return e;
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
template cudaError_t aca_run<float>(GeomDev, const int64_t*, const AcaTask*, const int*, c64*, double, int*, int*,
                                    cudaStream_t, int);
template cudaError_t aca_run<double>(GeomDev, const int64_t*, const AcaTask*, const int*, c128*, double, int*, int*,
                                     cudaStream_t, int);
template cudaError_t aca_compact<float>(const AcaTask*, int, const c64*, const int*, const int64_t*,
                                        const int64_t*, c64*, const int*, const int*, cudaStream_t);
template cudaError_t aca_compact<double>(const AcaTask*, int, const c128*, const int*, const int64_t*,
                                         const int64_t*, c128*, const int*, const int*, cudaStream_t);

}  // namespace bem
