// SVD recompression of the ACA factors of each far block and operator.  ACA stops
// with a rank k above the optimum for its tolerance; with B = A C^T (A = U, m x k;
// C = W = conj(V), n x k, the ACA scratch layout) the best rank-r form is read off
// a k x k core:
//   G_A = A^H A = R_A^H R_A,  G_C = C^H C = R_C^H R_C   (FP64 Gram matrices and
//        Cholesky factors: A = Q_A R_A, C = Q_C R_C with orthonormal Q)
//   M = R_A R_C^T = X S Y^H                              (one-sided Jacobi SVD)
//   B = Q_A M Q_C^T;  keep the r largest singular values, r the smallest rank with
//   sum_{i > r} s_i^2 <= tol^2 sum_i s_i^2 (the ACA tolerance, relative Frobenius)
// and, since Q_A X S = A R_C^T Y and S Y^H Q_C^T = (C R_A^T conj(X))^T,
//   U' = A (R_C^T Y_r S_r^{-1/2}),   W' = C (R_A^T conj(M Y)_r S_r^{-3/2})
// with no triangular solve.  Products of the stored values are exact in FP64, so
// the Gram matrices carry the small singular values that squaring would lose in
// FP32; the core, its SVD (in the operator's precision) and the final transforms
// lose only absolute errors of the order eps |A| |C|.  A rank-deficient Gram matrix
// drops the pivot (the column is a combination of the earlier ones).
// One CTA of RC_THREADS per task, everything but the tall factors in shared memory;
// tasks with k < 2 or k above RC_KMAX keep their ACA factors.
#include "common.cuh"

namespace bem {
namespace {

constexpr int RC_THREADS = 256;
constexpr int RC_WARPS = RC_THREADS / 32;
constexpr int RC_MAX_SWEEPS = 30;

template <typename R>
struct RcCfg;
template <>
struct RcCfg<float> {
    static constexpr int KMAX = 64;
    static constexpr float JTOL = 2e-7f;  // Jacobi: rotate while |gamma| > JTOL sqrt(alpha beta)
};
template <>
struct RcCfg<double> {
    static constexpr int KMAX = 48;
    static constexpr double JTOL = 4e-16;
};

// shared memory: R_A, R_C (FP64, k x k, row-major), M and Y (R, column-major)
template <typename R>
constexpr size_t rc_smem_bytes() {
    return (size_t)RcCfg<R>::KMAX * RcCfg<R>::KMAX * (2 * sizeof(c128) + 2 * sizeof(cx<R>)) +
           RcCfg<R>::KMAX * (sizeof(double) + sizeof(int)) + 64;
}

template <typename R>
__device__ __forceinline__ R warp_sum_r(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// G = X^H X (FP64, k x k, row-major, Hermitian) for X = the first k columns of an
// nrow x ld column-major array; rows staged through `stage` (cap rows at a time).
template <typename R>
__device__ void gram(const cx<R>* __restrict__ X, int nrow, int k, c128* G, cx<R>* stage, int cap) {
    const int ne = k * (k + 1) / 2;
    constexpr int PER = (RcCfg<R>::KMAX * (RcCfg<R>::KMAX + 1) / 2 + RC_THREADS - 1) / RC_THREADS;
    double ar[PER], ai[PER];
    int pp[PER], qq[PER];
#pragma unroll
    for (int s = 0; s < PER; ++s) {
        ar[s] = ai[s] = 0.0;
        const int e = threadIdx.x + s * RC_THREADS;
        // entry e -> (p, q), p <= q, row-major over the upper triangle
        int p = 0, rem = e;
        while (p < k && rem >= k - p) {
            rem -= k - p;
            ++p;
        }
        pp[s] = e < ne ? p : -1;
        qq[s] = e < ne ? p + rem : -1;
    }
    for (int r0 = 0; r0 < nrow; r0 += cap) {
        const int nr = min(cap, nrow - r0);
        __syncthreads();
        for (int e = threadIdx.x; e < nr * k; e += RC_THREADS) {
            const int l = e / nr, i = e - l * nr;  // column l, row r0 + i (coalesced over i)
            stage[i * k + l] = X[(int64_t)l * nrow + r0 + i];
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < PER; ++s) {
            if (pp[s] < 0) continue;
            const int p = pp[s], q = qq[s];
            double sr = 0.0, si = 0.0;
            for (int i = 0; i < nr; ++i) {
                const cx<R> a = stage[i * k + p], b = stage[i * k + q];
                // conj(a) b, products of the stored values exact in FP64
                sr = fma((double)a.re, (double)b.re, sr);
                sr = fma((double)a.im, (double)b.im, sr);
                si = fma((double)a.re, (double)b.im, si);
                si = fma(-(double)a.im, (double)b.re, si);
            }
            ar[s] += sr;
            ai[s] += si;
        }
    }
#pragma unroll
    for (int s = 0; s < PER; ++s) {
        if (pp[s] < 0) continue;
        const int p = pp[s], q = qq[s];
        G[p * k + q] = mk<double>(ar[s], ai[s]);
        G[q * k + p] = mk<double>(ar[s], -ai[s]);
    }
    __syncthreads();
}

// In place on the upper triangles of Ga and Gc (row-major k x k): G = R^H R with R
// upper triangular; a pivot at or below thr times the largest diagonal entry drops
// its row (R row j = 0: column j depends on the earlier columns).
__device__ void cholesky2(c128* Ga, c128* Gc, int k, int* s_drop) {
    __shared__ double s_thr[2];
    if (threadIdx.x < 2) {
        const c128* G = threadIdx.x == 0 ? Ga : Gc;
        double mx = 0.0;
        for (int j = 0; j < k; ++j) mx = fmax(mx, G[j * k + j].re);
        s_thr[threadIdx.x] = 1e-12 * mx;
    }
    __syncthreads();
    for (int j = 0; j < k; ++j) {
        if (threadIdx.x < 2) {
            c128* G = threadIdx.x == 0 ? Ga : Gc;
            const double piv = G[j * k + j].re;
            const bool drop = !(piv > s_thr[threadIdx.x]);
            s_drop[threadIdx.x] = drop;
            G[j * k + j] = mk<double>(drop ? 0.0 : sqrt(piv), 0.0);
        }
        __syncthreads();
        // row j beyond the diagonal: scaled, or zeroed when dropped
        for (int e = threadIdx.x; e < 2 * (k - j - 1); e += RC_THREADS) {
            const int w = e / (k - j - 1), c = j + 1 + e % (k - j - 1);
            c128* G = w == 0 ? Ga : Gc;
            const double d = G[j * k + j].re;
            G[j * k + c] = s_drop[w] ? mk<double>(0.0, 0.0) : (1.0 / d) * G[j * k + c];
        }
        __syncthreads();
        // trailing upper triangle: G[i][c] -= conj(R[j][i]) R[j][c], j < i <= c
        const int t = k - j - 1;
        for (int e = threadIdx.x; e < 2 * t * t; e += RC_THREADS) {
            const int w = e / (t * t), rest = e - w * t * t;
            const int i = j + 1 + rest / t, c = j + 1 + rest % t;
            if (c < i || s_drop[w]) continue;
            c128* G = w == 0 ? Ga : Gc;
            const c128 a = G[j * k + i], b = G[j * k + c];
            G[i * k + c] = G[i * k + c] - cconj(a) * b;
        }
        __syncthreads();
    }
}

// One-sided Jacobi on the k columns of M (column-major, leading dimension k),
// accumulating the rotations in Y (starts as the identity): M Y = X S on exit.
// Round-robin pairing: every round takes k/2 disjoint column pairs, one warp per pair.
template <typename R>
__device__ void jacobi_svd(cx<R>* M, cx<R>* Y, int k) {
    __shared__ int s_rot;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int kk = k + (k & 1);
    for (int sweep = 0; sweep < RC_MAX_SWEEPS; ++sweep) {
        if (threadIdx.x == 0) s_rot = 0;
        __syncthreads();
        int rotated = 0;
        for (int rd = 0; rd < kk - 1; ++rd) {
            for (int u = warp; u < kk / 2; u += RC_WARPS) {
                const int su = u, sv = kk - 1 - u;
                const int p = su == 0 ? 0 : 1 + (su - 1 + rd) % (kk - 1);
                const int q = sv == 0 ? 0 : 1 + (sv - 1 + rd) % (kk - 1);
                if (p >= k || q >= k) continue;
                cx<R>* mp = M + p * k;
                cx<R>* mq = M + q * k;
                R al = 0, be = 0, gr = 0, gi = 0;
                for (int i = lane; i < k; i += 32) {
                    const cx<R> a = mp[i], b = mq[i];
                    al += a.re * a.re + a.im * a.im;
                    be += b.re * b.re + b.im * b.im;
                    gr += a.re * b.re + a.im * b.im;  // conj(a) b
                    gi += a.re * b.im - a.im * b.re;
                }
                al = warp_sum_r(al);
                be = warp_sum_r(be);
                gr = warp_sum_r(gr);
                gi = warp_sum_r(gi);
                const R g = sqrt(gr * gr + gi * gi);
                if (!(g > RcCfg<R>::JTOL * sqrt(al * be)) || al == 0 || be == 0) continue;
                rotated = 1;
                const R zeta = (be - al) / (2 * g);
                const R t = (zeta >= 0 ? (R)1 : (R)-1) / (fabs(zeta) + sqrt((R)1 + zeta * zeta));
                const R c = (R)1 / sqrt((R)1 + t * t), s = c * t;
                const R er = gr / g, ei = gi / g;  // e^{i phi} = gamma / |gamma|
                // p' = c p - s e^{-i phi} q,  q' = s e^{i phi} p + c q  (columns of M and Y)
                auto rot = [&](cx<R>* xp, cx<R>* xq, int len) {
                    for (int i = lane; i < len; i += 32) {
                        const cx<R> a = xp[i], b = xq[i];
                        const cx<R> eb = mk<R>(er * b.re + ei * b.im, er * b.im - ei * b.re);  // e^{-i phi} b
                        const cx<R> ea = mk<R>(er * a.re - ei * a.im, er * a.im + ei * a.re);  // e^{i phi} a
                        xp[i] = mk<R>(c * a.re - s * eb.re, c * a.im - s * eb.im);
                        xq[i] = mk<R>(s * ea.re + c * b.re, s * ea.im + c * b.im);
                    }
                };
                rot(mp, mq, k);
                rot(Y + p * k, Y + q * k, k);
            }
            __syncthreads();
        }
        if (rotated && lane == 0) atomicOr(&s_rot, 1);
        __syncthreads();
        if (!s_rot) break;
    }
}

// X (nrow x ld column-major, first k columns) <- X T (k x r, column-major in shared
// memory), in place: each thread stages its own row, then writes its r outputs.
template <typename R>
__device__ void transform_rows(cx<R>* X, int nrow, int k, int r, const cx<R>* T, cx<R>* rowbuf, int rows_per_pass) {
    for (int base = 0; base < nrow; base += rows_per_pass) {
        __syncthreads();
        const int nr = min(rows_per_pass, nrow - base);
        for (int e = threadIdx.x; e < nr * k; e += RC_THREADS) {
            const int l = e / nr, i = e - l * nr;  // coalesced over rows
            rowbuf[i * k + l] = X[(int64_t)l * nrow + base + i];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nr; i += RC_THREADS) {
            const cx<R>* a = rowbuf + i * k;
            for (int c = 0; c < r; ++c) {
                cx<R> acc = mk<R>(0, 0);
                for (int l = 0; l < k; ++l) cfma(acc, a[l], T[c * k + l]);
                X[(int64_t)c * nrow + base + i] = acc;
            }
        }
    }
    __syncthreads();
}

template <typename R>
__global__ void __launch_bounds__(RC_THREADS, 1)
    k_recompress(const AcaTask* __restrict__ tasks, cx<R>* scratch, int* ranks, const int* flags, double tol,
                 cx<R>* ws, const int64_t* ws_off) {
    constexpr int KM = RcCfg<R>::KMAX;
    extern __shared__ __align__(16) unsigned char rsm[];
    c128* Ga = reinterpret_cast<c128*>(rsm);
    c128* Gc = Ga + KM * KM;
    cx<R>* M = reinterpret_cast<cx<R>*>(Gc + KM * KM);
    cx<R>* Y = M + KM * KM;
    double* sig2 = reinterpret_cast<double*>(Y + KM * KM);
    int* order = reinterpret_cast<int*>(sig2 + KM);
    __shared__ int s_drop[2];
    __shared__ int s_r;
    const int b = blockIdx.x;
    const int k = ranks[b];
    if (flags[b] || k < 2 || k > KM) return;
    const AcaTask T = tasks[b];
    cx<R>* A = scratch + T.scratch;                 // m x rmax, column-major
    cx<R>* C = A + (int64_t)T.m * T.rmax;          // n x rmax
    // 1. Gram matrices (rows staged through M and Y)
    const int cap = (int)((2 * (size_t)KM * KM) / k);
    gram<R>(A, T.m, k, Ga, M, cap);
    gram<R>(C, T.n, k, Gc, M, cap);
    // 2. Cholesky factors R_A, R_C (upper triangles of Ga, Gc)
    cholesky2(Ga, Gc, k, s_drop);
    // 3. core M = R_A R_C^T (column-major), Y = I
    for (int e = threadIdx.x; e < k * k; e += RC_THREADS) {
        const int i = e % k, j = e / k;
        double sr = 0.0, si = 0.0;
        for (int l = max(i, j); l < k; ++l) {
            const c128 a = Ga[i * k + l], c = Gc[j * k + l];
            sr += a.re * c.re - a.im * c.im;
            si += a.re * c.im + a.im * c.re;
        }
        M[j * k + i] = mk<R>((R)sr, (R)si);
        Y[j * k + i] = mk<R>(i == j ? (R)1 : (R)0, 0);
    }
    __syncthreads();
    // 4. SVD of the core: M Y = X S
    jacobi_svd<R>(M, Y, k);
    // 5. singular values, order, truncation rank
    for (int j = threadIdx.x; j < k; j += RC_THREADS) {
        double s = 0.0;
        for (int i = 0; i < k; ++i) s += (double)M[j * k + i].re * M[j * k + i].re + (double)M[j * k + i].im * M[j * k + i].im;
        sig2[j] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int j = 0; j < k; ++j) order[j] = j;
        for (int a = 0; a < k; ++a)  // selection sort, largest first (k <= KMAX)
            for (int c = a + 1; c < k; ++c)
                if (sig2[order[c]] > sig2[order[a]]) {
                    const int tmp = order[a];
                    order[a] = order[c];
                    order[c] = tmp;
                }
        double total = 0.0;
        for (int j = 0; j < k; ++j) total += sig2[j];
        int r = k;
        double tail = 0.0;
        while (r > 1 && tail + sig2[order[r - 1]] <= tol * tol * total) tail += sig2[order[--r]];
        s_r = (total > 0.0 && sig2[order[r - 1]] > 0.0) ? r : k;
    }
    __syncthreads();
    const int r = s_r;
    if (r >= k) return;  // nothing to gain: the ACA factors stay
    // 6. T_A = R_C^T Y_r S^{-1/2}, T_C = R_A^T conj(M Y)_r S^{-3/2} (k x r each, column-major, to ws)
    cx<R>* Ta = ws + ws_off[b];
    cx<R>* Tc = Ta + (int64_t)k * k;
    for (int e = threadIdx.x; e < k * r; e += RC_THREADS) {
        const int l = e % k, c = e / k;
        const int oc = order[c];
        const double s = sqrt(sig2[oc]);
        const double fa = 1.0 / sqrt(s), fc = 1.0 / (s * sqrt(s));
        double ar = 0.0, ai = 0.0, cr = 0.0, ci = 0.0;
        for (int j = 0; j <= l; ++j) {
            const c128 rc = Gc[j * k + l], ra = Ga[j * k + l];
            const cx<R> y = Y[oc * k + j], x = M[oc * k + j];
            ar += rc.re * (double)y.re - rc.im * (double)y.im;
            ai += rc.re * (double)y.im + rc.im * (double)y.re;
            cr += ra.re * (double)x.re + ra.im * (double)x.im;  // ra conj(x)
            ci += ra.im * (double)x.re - ra.re * (double)x.im;
        }
        Ta[c * k + l] = mk<R>((R)(ar * fa), (R)(ai * fa));
        Tc[c * k + l] = mk<R>((R)(cr * fc), (R)(ci * fc));
    }
    __syncthreads();
    // 7. U' = A T_A, W' = C T_C in place (shared memory: T, then staged rows)
    cx<R>* Ts = reinterpret_cast<cx<R>*>(rsm);
    cx<R>* rowbuf = Ts + KM * KM;
    const size_t total_smem = rc_smem_bytes<R>() - 64;
    const int rows = (int)min((size_t)RC_THREADS, (total_smem - sizeof(cx<R>) * KM * KM) / (sizeof(cx<R>) * k));
    for (int side = 0; side < 2; ++side) {
        const cx<R>* Tg = side == 0 ? Ta : Tc;
        for (int e = threadIdx.x; e < k * r; e += RC_THREADS) Ts[e] = Tg[e];
        __syncthreads();
        transform_rows<R>(side == 0 ? A : C, side == 0 ? T.m : T.n, k, r, Ts, rowbuf, rows);
    }
    if (threadIdx.x == 0) ranks[b] = r;
}

}  // namespace

template <typename R>
int recompress_kmax() {
    return RcCfg<R>::KMAX;
}

template <typename R>
cudaError_t aca_recompress(const AcaTask* tasks, int ntasks, cx<R>* scratch, int* ranks, const int* flags,
                           double tol, cx<R>* ws, const int64_t* ws_off, cudaStream_t st) {
    if (ntasks <= 0) return cudaSuccess;
    const size_t sm = rc_smem_bytes<R>();
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(k_recompress<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_recompress<R><<<ntasks, RC_THREADS, sm, st>>>(tasks, scratch, ranks, flags, tol, ws, ws_off);
    return cudaGetLastError();
}

template int recompress_kmax<float>();
template int recompress_kmax<double>();
template cudaError_t aca_recompress<float>(const AcaTask*, int, c64*, int*, const int*, double, c64*,
                                           const int64_t*, cudaStream_t);
template cudaError_t aca_recompress<double>(const AcaTask*, int, c128*, int*, const int*, double, c128*,
                                            const int64_t*, cudaStream_t);

}  // namespace bem
