// Batched restarted GMRES with every step on the device.  The right-hand sides of
// one solve advance together: iteration j applies the operator once to the nrhs
// basis vectors V_j (one product call over all of them), then each right-hand side
// r orthogonalises its own w = Z v_j against its own basis v_0 .. v_j, updates its
// Hessenberg column with Givens rotations and estimates its residual, without a
// host round trip.  Right-hand sides that have converged (or hit the iteration
// cap) drop out: their kernels return at once and their basis columns stay zero.
//
// The Krylov solve is not in the paper (its Eq. 18 inverts the compressed
// operator directly); it is the iterative counterpart applied to the same
// compressed product, and the batching mirrors the paper's many-right-hand-side
// solve (Woodbury inverse, Section III) in iterative form.
//
// Orthogonalisation: classical Gram-Schmidt, h = V^H w, w -= V h, repeated for a
// right-hand side only when the first pass cancelled nearly all of w
// (|w_after| < 0.22 |w_before|; a second pass then restores orthogonality to
// working precision, "twice is enough").  Without it, the orthogonality lost in
// one step is about eps |w_before|^2 / |w_after|^2 <= 20 eps, below the accuracy
// the FP32 basis stores anyway.  Precision follows the
// vectors (R = float for complex64, double for complex128): products and sums
// over a thread's rows and a warp's lanes (a pairwise tree) in R, sums across
// warps and CTAs in FP64 in a fixed order (results do not depend on scheduling);
// for complex64 the error of one inner product is within about 14 * 2^-24 *
// sum |v_i| |w_i|, the level of the stored FP32 basis.  The Hessenberg matrix,
// rotations and the restart's triangular solve are in R as well (the usual
// working precision of a mixed-precision inner solver): one thread per
// right-hand side, so that an FP64 instruction, slow to issue on this GPU, is
// never spent on a single lane.
//
// Vector layout: a CTA covers `chunk` consecutive rows of one right-hand side
// (a multiple of 256 threads x the complex values of one 16-byte load); thread t
// loads units t, t + 256, ... of 16 bytes (two complex64 or one complex128).
#include "common.cuh"

namespace bem {

namespace {

constexpr int BG_THREADS = 256;
constexpr int BG_WARPS = BG_THREADS / 32;
constexpr int BG_LD = 4;               // 16-byte loads per vector per thread (at most)
constexpr int QG = 4;                  // basis vectors per step of the inner-product loop
constexpr int QGU = 8;                 // basis vectors per step of the update loop
constexpr double REORTH_KEEP2 = 0.05;  // second pass if |w_after|^2 < 0.05 |w_before|^2

// 16-byte packs of complex values
template <typename R>
struct Pk;
template <>
struct Pk<float> {
    static constexpr int PC = 2;
    static __device__ __forceinline__ void ld(const c64* p, c64 (&v)[2]) {
        const float4 f = *reinterpret_cast<const float4*>(p);
        v[0] = mk<float>(f.x, f.y);
        v[1] = mk<float>(f.z, f.w);
    }
    static __device__ __forceinline__ void st(c64* p, const c64 (&v)[2]) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0].re, v[0].im, v[1].re, v[1].im);
    }
};
template <>
struct Pk<double> {
    static constexpr int PC = 1;
    static __device__ __forceinline__ void ld(const c128* p, c128 (&v)[1]) {
        const double2 f = *reinterpret_cast<const double2*>(p);
        v[0] = mk<double>(f.x, f.y);
    }
    static __device__ __forceinline__ void st(c128* p, const c128 (&v)[1]) {
        *reinterpret_cast<double2*>(p) = make_double2(v[0].re, v[0].im);
    }
};

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// first row of load unit k of this thread (PC rows follow), and whether it exists
template <typename R>
__device__ __forceinline__ int64_t unit_row(const BgsArgs& a, int k) {
    return (int64_t)blockIdx.x * a.chunk + ((int64_t)threadIdx.x + (int64_t)k * BG_THREADS) * Pk<R>::PC;
}
template <typename R>
__device__ __forceinline__ bool unit_ok(const BgsArgs& a, int k, int64_t i) {
    return k * BG_THREADS * Pk<R>::PC < a.chunk && i < a.n;  // n and chunk are multiples of PC
}

// CTA arrival for a last-CTA reduction; true in the CTA that arrived last (its
// view of the other CTAs' partials is then complete)
__device__ __forceinline__ bool last_arrival(unsigned* cnt, int nblk, int* s_flag) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(cnt, 1u);
        *s_flag = prev == (unsigned)(nblk - 1);
        if (*s_flag) *cnt = 0u;  // every CTA of this right-hand side has arrived
    }
    __syncthreads();
    if (*(volatile int*)s_flag) {
        __threadfence();
        return true;
    }
    return false;
}

// sum over b < nblk of p[b * stride] by one warp: lane l takes b = l, l + 32, ...
// in order, then a fixed xor tree (deterministic)
__device__ __forceinline__ double warp_sum_blocks(const double* p, int nblk, int stride) {
    double s = 0;
    for (int b = threadIdx.x & 31; b < nblk; b += 32) s += __ldcg(p + (int64_t)b * stride);
    return warp_sum(s);
}

// h[q] = sum_i conj(V_q[i]) w[i] for q <= j (and |w|^2 in pass 1), w = basis slot
// j + 1 of right-hand side r (the product's output).  Pass 1 runs for the active
// right-hand sides, pass 2 for those flagged for a second pass.  CTA (blk, s) of a
// right-hand side takes rows chunk blk and basis vectors [s qs, (s + 1) qs): with
// few right-hand sides the basis is split too, so that enough loads are in flight.
template <typename R>
__global__ void __launch_bounds__(BG_THREADS) k_bgs_dot(BgsArgs a, int j, int pass, int qs) {
    constexpr int PC = Pk<R>::PC;
    extern __shared__ double sh[];  // [qs + 1][BG_WARPS][2]
    __shared__ int s_flag;
    const int r = blockIdx.y;
    const int flag = a.state[r];
    if (!(flag & (pass == 1 ? BGS_ACTIVE : BGS_REORTH))) return;
    const int blk = blockIdx.x % a.nblk, sl = blockIdx.x / a.nblk;
    const int nslab = gridDim.x / a.nblk;
    const int64_t n = a.n;
    const cx<R>* V = reinterpret_cast<const cx<R>*>(a.V) + (int64_t)r * n;
    const int64_t slot = (int64_t)a.nrhs * n;
    const cx<R>* w = V + (int64_t)(j + 1) * slot;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t row0 = (int64_t)blk * a.chunk;
    auto urow = [&](int k) { return row0 + ((int64_t)threadIdx.x + (int64_t)k * BG_THREADS) * PC; };
    cx<R> wv[BG_LD][PC];
    R nrm = 0;
#pragma unroll
    for (int k = 0; k < BG_LD; ++k) {
        const int64_t i = urow(k);
        if (unit_ok<R>(a, k, i)) {
            Pk<R>::ld(w + i, wv[k]);
        } else {
#pragma unroll
            for (int p = 0; p < PC; ++p) wv[k][p] = mk<R>(0, 0);
        }
#pragma unroll
        for (int p = 0; p < PC; ++p) nrm += wv[k][p].re * wv[k][p].re + wv[k][p].im * wv[k][p].im;
    }
    const int nq = j + 1;
    const int q0 = sl * qs, q1 = min(nq, q0 + qs);
    for (int q = q0; q < q1; q += QG) {
        cx<R> acc[QG];
#pragma unroll
        for (int u = 0; u < QG; ++u) acc[u] = mk<R>(0, 0);
#pragma unroll
        for (int k = 0; k < BG_LD; ++k) {
            const int64_t i = urow(k);
            if (!(k * BG_THREADS * PC < a.chunk && i < n)) continue;
#pragma unroll
            for (int u = 0; u < QG; ++u) {
                if (q + u >= q1) continue;
                cx<R> v[PC];
                Pk<R>::ld(V + (int64_t)(q + u) * slot + i, v);
#pragma unroll
                for (int p = 0; p < PC; ++p) cfma_conj(acc[u], v[p], wv[k][p]);
            }
        }
#pragma unroll
        for (int u = 0; u < QG; ++u) {
            acc[u].re = warp_sum(acc[u].re);
            acc[u].im = warp_sum(acc[u].im);
        }
        if (lane == 0) {
#pragma unroll
            for (int u = 0; u < QG; ++u)
                if (q + u < q1) {
                    sh[((q + u - q0) * BG_WARPS + warp) * 2] = (double)acc[u].re;
                    sh[((q + u - q0) * BG_WARPS + warp) * 2 + 1] = (double)acc[u].im;
                }
        }
    }
    nrm = warp_sum(nrm);
    if (lane == 0) {
        sh[(qs * BG_WARPS + warp) * 2] = (double)nrm;
        sh[(qs * BG_WARPS + warp) * 2 + 1] = 0.0;
    }
    __syncthreads();
    const int stride = a.m + 2;
    double* part = reinterpret_cast<double*>(a.part);  // [r][q][blk][re, im]
    // this CTA's basis vectors, and |w|^2 (slab 0 only) at q = nq
    for (int t = threadIdx.x; t <= q1 - q0; t += BG_THREADS) {
        const int q = t < q1 - q0 ? q0 + t : nq;
        const int ts = t < q1 - q0 ? t : qs;
        if (q == nq && sl != 0) continue;
        double re = 0, im = 0;
        for (int u = 0; u < BG_WARPS; ++u) {
            re += sh[(ts * BG_WARPS + u) * 2];
            im += sh[(ts * BG_WARPS + u) * 2 + 1];
        }
        double* d = part + 2 * (((int64_t)r * stride + q) * a.nblk + blk);
        d[0] = re;
        d[1] = im;
    }
    if (!last_arrival(a.cnt + r, a.nblk * nslab, &s_flag)) return;
    cx<R>* h = reinterpret_cast<cx<R>*>(pass == 1 ? a.h1 : a.h2) + (int64_t)r * (a.m + 1);
    for (int q = warp; q <= nq; q += BG_WARPS) {
        const double* d = part + 2 * ((int64_t)r * stride + q) * a.nblk;
        const double re = warp_sum_blocks(d, a.nblk, 2);
        const double im = warp_sum_blocks(d + 1, a.nblk, 2);
        if (lane == 0) {
            if (q < nq)
                h[q] = mk<R>((R)re, (R)im);
            else if (pass == 1)
                a.wn0[r] = re;
        }
    }
}

// w -= sum_{q <= j} h[q] V_q (h from pass `pass`), and |w|^2 after the update; the
// last CTA of pass 1 flags the right-hand side for a second pass when most of w
// cancelled.
template <typename R>
__global__ void __launch_bounds__(BG_THREADS) k_bgs_update(BgsArgs a, int j, int pass) {
    constexpr int PC = Pk<R>::PC;
    extern __shared__ double sh[];  // [BG_WARPS] norms, then the coefficients as cx<R>
    __shared__ int s_flag;
    const int r = blockIdx.y;
    const int flag = a.state[r];
    if (!(flag & (pass == 1 ? BGS_ACTIVE : BGS_REORTH))) return;
    const int64_t n = a.n;
    cx<R>* V = reinterpret_cast<cx<R>*>(a.V) + (int64_t)r * n;
    const int64_t slot = (int64_t)a.nrhs * n;
    cx<R>* w = V + (int64_t)(j + 1) * slot;
    const int nq = j + 1;
    double* wsum = sh;
    cx<R>* hc = reinterpret_cast<cx<R>*>(sh + BG_WARPS);
    const cx<R>* h = reinterpret_cast<const cx<R>*>(pass == 1 ? a.h1 : a.h2) + (int64_t)r * (a.m + 1);
    for (int q = threadIdx.x; q < nq; q += BG_THREADS) hc[q] = mk<R>(-h[q].re, -h[q].im);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    cx<R> wv[BG_LD][PC];
#pragma unroll
    for (int k = 0; k < BG_LD; ++k) {
        const int64_t i = unit_row<R>(a, k);
        if (unit_ok<R>(a, k, i)) {
            Pk<R>::ld(w + i, wv[k]);
        } else {
#pragma unroll
            for (int p = 0; p < PC; ++p) wv[k][p] = mk<R>(0, 0);
        }
    }
    for (int q = 0; q < nq; q += QGU) {
        cx<R> c[QGU];
#pragma unroll
        for (int u = 0; u < QGU; ++u) c[u] = q + u < nq ? hc[q + u] : mk<R>(0, 0);
#pragma unroll
        for (int k = 0; k < BG_LD; ++k) {
            const int64_t i = unit_row<R>(a, k);
            if (!unit_ok<R>(a, k, i)) continue;
#pragma unroll
            for (int u = 0; u < QGU; ++u) {
                if (q + u >= nq) continue;
                cx<R> v[PC];
                Pk<R>::ld(V + (int64_t)(q + u) * slot + i, v);
#pragma unroll
                for (int p = 0; p < PC; ++p) cfma(wv[k][p], c[u], v[p]);
            }
        }
    }
    R nrm = 0;
#pragma unroll
    for (int k = 0; k < BG_LD; ++k) {
        const int64_t i = unit_row<R>(a, k);
        if (unit_ok<R>(a, k, i)) {
            Pk<R>::st(w + i, wv[k]);
#pragma unroll
            for (int p = 0; p < PC; ++p) nrm += wv[k][p].re * wv[k][p].re + wv[k][p].im * wv[k][p].im;
        }
    }
    nrm = warp_sum(nrm);
    if (lane == 0) wsum[warp] = (double)nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int u = 0; u < BG_WARPS; ++u) s += wsum[u];
        a.npart[(int64_t)r * a.nblk + blockIdx.x] = s;
    }
    if (!last_arrival(a.cnt + r, a.nblk, &s_flag)) return;
    if (warp == 0) {
        const double s = warp_sum_blocks(a.npart + (int64_t)r * a.nblk, a.nblk, 1);
        if (lane == 0) {
            if (pass == 1) {
                a.wn1[r] = s;
                a.state[r] = s < REORTH_KEEP2 * a.wn0[r] ? (flag | BGS_REORTH) : (flag & ~BGS_REORTH);
            } else {
                a.wn2[r] = s;
            }
        }
    }
}

// One thread per right-hand side (one CTA): Hessenberg column j from the passes,
// the earlier rotations applied to it, a new rotation zeroing its subdiagonal, the
// rotated residual vector g and its last entry |g_{j+1}| (the residual norm of the
// iterate).  A right-hand side stops when that reaches its tolerance, when the
// Krylov space is exhausted (|w| = 0), at the restart length or at the iteration
// cap; `scale` then becomes 0 so its next basis vector is zero.  The rotations
// have real cosines.  Thread 0 publishes how many right-hand sides remain active.
// With few right-hand sides (`staged`) the CTA first copies every column and the
// earlier rotations into shared memory, so that the sequential rotations read
// nothing from global memory.
template <typename R>
__global__ void k_bgs_givens(BgsArgs a, int j, int staged) {
    extern __shared__ double gsm[];  // staged: columns [nrhs][j + 1], sines [nrhs][j], cosines [nrhs][j]
    __shared__ int s_count;
    if (threadIdx.x == 0) s_count = 0;
    const int m = a.m;
    cx<R>* scol = reinterpret_cast<cx<R>*>(gsm);
    cx<R>* ssn = scol + (size_t)a.nrhs * (j + 1);
    R* scs = reinterpret_cast<R*>(ssn + (size_t)a.nrhs * j);
    if (staged) {
        for (int e = threadIdx.x; e < a.nrhs * (j + 1); e += blockDim.x) {
            const int r = e / (j + 1), i = e - r * (j + 1);
            const int flag = a.state[r];
            const cx<R> v = reinterpret_cast<const cx<R>*>(a.h1)[(int64_t)r * (m + 1) + i];
            scol[e] = (flag & BGS_REORTH) ? v + reinterpret_cast<const cx<R>*>(a.h2)[(int64_t)r * (m + 1) + i] : v;
        }
        for (int e = threadIdx.x; e < a.nrhs * j; e += blockDim.x) {
            const int r = e / j, i = e - r * j;
            ssn[e] = reinterpret_cast<const cx<R>*>(a.sn)[(int64_t)r * m + i];
            scs[e] = reinterpret_cast<const R*>(a.cs)[(int64_t)r * m + i];
        }
    }
    __syncthreads();
    int mine = 0;
    for (int r = threadIdx.x; r < a.nrhs; r += blockDim.x) {
        const int flag = a.state[r];
        if (!(flag & BGS_ACTIVE)) continue;
        const bool two = (flag & BGS_REORTH) != 0;
        cx<R>* __restrict__ H = reinterpret_cast<cx<R>*>(a.H) + (int64_t)r * (m + 1) * m;
        cx<R>* __restrict__ g = reinterpret_cast<cx<R>*>(a.g) + (int64_t)r * (m + 1);
        R* __restrict__ cs = reinterpret_cast<R*>(a.cs) + (int64_t)r * m;
        cx<R>* __restrict__ sn = reinterpret_cast<cx<R>*>(a.sn) + (int64_t)r * m;
        const cx<R>* __restrict__ h1 = reinterpret_cast<const cx<R>*>(a.h1) + (int64_t)r * (m + 1);
        const cx<R>* __restrict__ h2 = reinterpret_cast<const cx<R>*>(a.h2) + (int64_t)r * (m + 1);
        const cx<R>* sc = scol + (size_t)r * (j + 1);
        const cx<R>* ss = ssn + (size_t)r * j;
        const R* sk = scs + (size_t)r * j;
        const R hn = (R)sqrt(fmax(two ? a.wn2[r] : a.wn1[r], 0.0));
        cx<R> prev = staged ? sc[0] : (two ? h1[0] + h2[0] : h1[0]);
#pragma unroll 4
        for (int i = 0; i < j; ++i) {
            const cx<R> b = staged ? sc[i + 1] : (two ? h1[i + 1] + h2[i + 1] : h1[i + 1]);
            const R c = staged ? sk[i] : cs[i];
            const cx<R> s = staged ? ss[i] : sn[i];
            cx<R> top = c * prev;
            cfma(top, s, b);
            H[(int64_t)i * m + j] = top;
            cx<R> bot = c * b;
            cfma(bot, mk<R>(-s.re, s.im), prev);  // - conj(s) prev
            prev = bot;
        }
        const R na = sqrt(cabs2(prev));
        const R t = sqrt(na * na + hn * hn);
        R c;
        cx<R> s;
        if (na == 0) {
            c = 0;
            s = mk<R>(1, 0);
        } else {
            c = na / t;
            s = (hn / (na * t)) * prev;
        }
        cs[j] = c;
        sn[j] = s;
        cx<R> d = c * prev;
        d.re += s.re * hn;
        d.im += s.im * hn;
        H[(int64_t)j * m + j] = d;
        const cx<R> gj = g[j];
        g[j + 1] = mk<R>(-(s.re * gj.re + s.im * gj.im), -(s.re * gj.im - s.im * gj.re));  // -conj(s) g_j
        g[j] = c * gj;
        const R res = sqrt(cabs2(g[j + 1]));
        const int it = a.it[r] + 1;
        a.it[r] = it;
        a.res[r] = (double)res;
        const bool done = (double)res <= a.tol[r] || hn == 0 || j + 1 >= m || it >= a.maxit || !(res == res);
        a.scale[r] = done ? 0.0 : 1.0 / (double)hn;
        int f = flag & ~BGS_REORTH;
        if (done) {
            a.kk[r] = j + 1;
            f &= ~BGS_ACTIVE;
        } else {
            ++mine;
        }
        a.state[r] = f;
    }
    if (mine) atomicAdd(&s_count, mine);
    __syncthreads();
    if (threadIdx.x == 0) {
        *(volatile int*)a.host_active = s_count;
        __threadfence_system();
    }
}

// basis slot `slot` of every right-hand side scaled by its `scale` (0: zeroed)
template <typename R>
__global__ void __launch_bounds__(BG_THREADS) k_bgs_scale(BgsArgs a, int slot) {
    constexpr int PC = Pk<R>::PC;
    const int r = blockIdx.y;
    cx<R>* v = reinterpret_cast<cx<R>*>(a.V) + ((int64_t)slot * a.nrhs + r) * a.n;
    const R s = (R)a.scale[r];
#pragma unroll
    for (int k = 0; k < BG_LD; ++k) {
        const int64_t i = unit_row<R>(a, k);
        if (!unit_ok<R>(a, k, i)) continue;
        cx<R> u[PC];
        Pk<R>::ld(v + i, u);
#pragma unroll
        for (int p = 0; p < PC; ++p) u[p] = mk<R>(u[p].re * s, u[p].im * s);
        Pk<R>::st(v + i, u);
    }
}

// One thread per right-hand side: y = R^-1 g over the kk columns the cycle built
// (R the rotated, upper triangular Hessenberg matrix).
template <typename R>
__global__ void k_bgs_trisolve(BgsArgs a) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.nrhs) return;
    const int m = a.m, k = min(a.kk[r], m);
    const cx<R>* H = reinterpret_cast<const cx<R>*>(a.H) + (int64_t)r * (m + 1) * m;
    const cx<R>* g = reinterpret_cast<const cx<R>*>(a.g) + (int64_t)r * (m + 1);
    cx<R>* y = reinterpret_cast<cx<R>*>(a.y) + (int64_t)r * m;
    for (int i = k - 1; i >= 0; --i) {
        cx<R> acc = g[i];
        for (int l = i + 1; l < k; ++l) acc = acc - H[(int64_t)i * m + l] * y[l];
        const cx<R> d = H[(int64_t)i * m + i];
        y[i] = (d.re == 0 && d.im == 0) ? mk<R>(0, 0) : cdiv(acc, d);
    }
}

// x_r += sum_{q < kk_r} y_r[q] V_q (the cycle's correction)
template <typename R>
__global__ void __launch_bounds__(BG_THREADS) k_bgs_xupdate(BgsArgs a) {
    constexpr int PC = Pk<R>::PC;
    extern __shared__ double sh[];
    const int r = blockIdx.y;
    const int k = min(a.kk[r], a.m);
    if (k <= 0) return;
    const int64_t n = a.n;
    const cx<R>* V = reinterpret_cast<const cx<R>*>(a.V) + (int64_t)r * n;
    const int64_t slot = (int64_t)a.nrhs * n;
    cx<R>* x = reinterpret_cast<cx<R>*>(a.x) + (int64_t)r * n;
    cx<R>* yc = reinterpret_cast<cx<R>*>(sh);
    const cx<R>* y = reinterpret_cast<const cx<R>*>(a.y) + (int64_t)r * a.m;
    for (int q = threadIdx.x; q < k; q += BG_THREADS) yc[q] = y[q];
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BG_LD; ++kk) {
        const int64_t i = unit_row<R>(a, kk);
        if (!unit_ok<R>(a, kk, i)) continue;
        cx<R> acc[PC];
        Pk<R>::ld(x + i, acc);
        for (int q = 0; q < k; ++q) {
            cx<R> v[PC];
            Pk<R>::ld(V + (int64_t)q * slot + i, v);
#pragma unroll
            for (int p = 0; p < PC; ++p) cfma(acc[p], yc[q], v[p]);
        }
        Pk<R>::st(x + i, acc);
    }
}

// Start of a cycle: basis slot 0 = b - Z x (slot 0 holds Z x; or b alone when
// `x_zero`), beta = |b - Z x| per right-hand side, g_0 = beta, and the right-hand
// side active while beta is above its tolerance and iterations remain; `scale` =
// 1 / beta for the normalisation that follows (the rest of g is written by the
// rotations before it is read).  A right-hand side also stops when three cycles in
// a row reached the tolerance by their estimate but the recomputed residual did not
// follow (rounding floor of the product, which outer refinement then removes).
template <typename R>
__global__ void __launch_bounds__(BG_THREADS) k_bgs_resid(BgsArgs a, int x_zero) {
    constexpr int PC = Pk<R>::PC;
    __shared__ double wsum[BG_WARPS];
    __shared__ int s_flag;
    const int r = blockIdx.y;
    const int64_t n = a.n;
    cx<R>* v0 = reinterpret_cast<cx<R>*>(a.V) + (int64_t)r * n;
    const cx<R>* b = reinterpret_cast<const cx<R>*>(a.b) + (int64_t)r * n;
    R nrm = 0;
#pragma unroll
    for (int k = 0; k < BG_LD; ++k) {
        const int64_t i = unit_row<R>(a, k);
        if (!unit_ok<R>(a, k, i)) continue;
        cx<R> bv[PC], zv[PC];
        Pk<R>::ld(b + i, bv);
        if (!x_zero) {
            Pk<R>::ld(v0 + i, zv);
#pragma unroll
            for (int p = 0; p < PC; ++p) bv[p] = bv[p] - zv[p];
        }
        Pk<R>::st(v0 + i, bv);
#pragma unroll
        for (int p = 0; p < PC; ++p) nrm += bv[p].re * bv[p].re + bv[p].im * bv[p].im;
    }
    nrm = warp_sum(nrm);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = (double)nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int u = 0; u < BG_WARPS; ++u) s += wsum[u];
        a.npart[(int64_t)r * a.nblk + blockIdx.x] = s;
    }
    if (!last_arrival(a.cnt + r, a.nblk, &s_flag)) return;
    if (threadIdx.x < 32) {
        const double s = warp_sum_blocks(a.npart + (int64_t)r * a.nblk, a.nblk, 1);
        if (threadIdx.x == 0) {
            const double beta = sqrt(s);
            // rounding floor of the product: a cycle met the tolerance by its residual
            // estimate, yet the recomputed residual is above it and less than half the
            // previous cycle's; the third such cycle in a row stops the right-hand side
            int misses = x_zero ? 0 : (a.state[r] >> BGS_MISS_SHIFT) & 0xff;
            if (!x_zero)
                misses = (a.res[r] <= a.tol[r] && beta > a.tol[r] && beta > 0.5 * a.beta[r]) ? misses + 1 : 0;
            a.beta[r] = beta;
            const bool act = beta > a.tol[r] && a.it[r] < a.maxit && beta == beta && misses < 3;
            a.state[r] = (act ? BGS_ACTIVE : 0) | (misses << BGS_MISS_SHIFT);
            a.scale[r] = act ? 1.0 / beta : 0.0;
            a.kk[r] = 0;
            reinterpret_cast<cx<R>*>(a.g)[(int64_t)r * (a.m + 1)] = mk<R>((R)beta, 0);
        }
    }
}

// how many right-hand sides are active (after k_bgs_resid), published to the host
__global__ void k_bgs_count(BgsArgs a) {
    __shared__ int s_count;
    if (threadIdx.x == 0) s_count = 0;
    __syncthreads();
    int mine = 0;
    for (int r = threadIdx.x; r < a.nrhs; r += blockDim.x) mine += (a.state[r] & BGS_ACTIVE) ? 1 : 0;
    if (mine) atomicAdd(&s_count, mine);
    __syncthreads();
    if (threadIdx.x == 0) {
        *(volatile int*)a.host_active = s_count;
        __threadfence_system();
    }
}

// out[r] = |v_r|^2 for the nrhs columns of n values at a.V (R per thread and warp,
// FP64 beyond)
template <typename R>
__global__ void __launch_bounds__(BG_THREADS) k_colnorm2(BgsArgs a, double* out) {
    constexpr int PC = Pk<R>::PC;
    __shared__ double wsum[BG_WARPS];
    __shared__ int s_flag;
    const int r = blockIdx.y;
    const cx<R>* col = reinterpret_cast<const cx<R>*>(a.V) + (int64_t)r * a.n;
    R nrm = 0;
#pragma unroll
    for (int k = 0; k < BG_LD; ++k) {
        const int64_t i = unit_row<R>(a, k);
        if (!unit_ok<R>(a, k, i)) continue;
        cx<R> u[PC];
        Pk<R>::ld(col + i, u);
#pragma unroll
        for (int p = 0; p < PC; ++p) nrm += u[p].re * u[p].re + u[p].im * u[p].im;
    }
    nrm = warp_sum(nrm);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = (double)nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int u = 0; u < BG_WARPS; ++u) t += wsum[u];
        a.npart[(int64_t)r * a.nblk + blockIdx.x] = t;
    }
    if (!last_arrival(a.cnt + r, a.nblk, &s_flag)) return;
    if (threadIdx.x < 32) {
        const double t = warp_sum_blocks(a.npart + (int64_t)r * a.nblk, a.nblk, 1);
        if (threadIdx.x == 0) out[r] = t;
    }
}

}  // namespace

void bgs_layout(int64_t n, int nrhs, int esize, int* chunk, int* nblk) {
    // aim at 4 CTAs per SM of 152 over all right-hand sides; a chunk is a multiple of
    // 256 threads x the complex values of one 16-byte load, at most BG_LD loads each
    const int64_t gran = (int64_t)BG_THREADS * (16 / esize);
    const int64_t want = (608 + nrhs - 1) / nrhs;
    int64_t c = (n + want - 1) / want;
    c = ((c + gran - 1) / gran) * gran;
    if (c > gran * BG_LD) c = gran * BG_LD;
    *chunk = (int)c;
    *nblk = (int)((n + c - 1) / c);
}

template <typename R>
cudaError_t bgs_iteration(const BgsArgs& a, int j, cudaStream_t st) {
    const dim3 grid(a.nblk, a.nrhs);
    // inner products: split the basis into slabs of qs vectors when the row chunks
    // of all right-hand sides give fewer than 8 CTAs per SM
    const int nq = j + 1;
    const int want = (8 * 152 + a.nblk * a.nrhs - 1) / (a.nblk * a.nrhs);
    const int nslab = std::max(1, std::min(want, (nq + QG - 1) / QG));
    const int qs = ((nq + nslab - 1) / nslab + QG - 1) / QG * QG;
    const int nsl = (nq + qs - 1) / qs;
    const dim3 gdot(a.nblk * nsl, a.nrhs);
    const size_t sd = sizeof(double) * 2 * BG_WARPS * (size_t)(qs + 1);
    const size_t su = sizeof(double) * BG_WARPS + sizeof(cx<R>) * (size_t)(j + 1);
    for (int pass = 1; pass <= 2; ++pass) {
        k_bgs_dot<R><<<gdot, BG_THREADS, sd, st>>>(a, j, pass, qs);
        k_bgs_update<R><<<grid, BG_THREADS, su, st>>>(a, j, pass);
    }
    const size_t sg = (sizeof(cx<R>) * (size_t)(2 * j + 1) + sizeof(R) * (size_t)j) * a.nrhs;
    const bool staged = sg <= 32768;
    k_bgs_givens<R><<<1, std::min(1024, ((a.nrhs + 31) / 32) * 32), staged ? sg : 0, st>>>(a, j, staged ? 1 : 0);
    k_bgs_scale<R><<<grid, BG_THREADS, 0, st>>>(a, j + 1);
    return cudaGetLastError();
}

template <typename R>
cudaError_t bgs_cycle_start(const BgsArgs& a, bool x_zero, cudaStream_t st) {
    k_bgs_resid<R><<<dim3(a.nblk, a.nrhs), BG_THREADS, 0, st>>>(a, x_zero ? 1 : 0);
    k_bgs_count<<<1, 1024, 0, st>>>(a);
    k_bgs_scale<R><<<dim3(a.nblk, a.nrhs), BG_THREADS, 0, st>>>(a, 0);
    return cudaGetLastError();
}

template <typename R>
cudaError_t bgs_cycle_end(const BgsArgs& a, cudaStream_t st) {
    k_bgs_trisolve<R><<<(a.nrhs + 63) / 64, 64, 0, st>>>(a);
    k_bgs_xupdate<R><<<dim3(a.nblk, a.nrhs), BG_THREADS, sizeof(cx<R>) * (size_t)a.m, st>>>(a);
    return cudaGetLastError();
}

cudaError_t col_norms2(const void* v, bool fp64, int64_t n, int k, double* npart, int npart_cap, unsigned* cnt,
                       double* out, cudaStream_t st) {
    BgsArgs a{};
    a.V = const_cast<void*>(v);
    a.n = n;
    a.nrhs = k;
    a.npart = npart;
    a.cnt = cnt;
    bgs_layout(n, k, fp64 ? 16 : 8, &a.chunk, &a.nblk);
    if (a.nblk > npart_cap) return cudaErrorInvalidValue;  // partials would not fit
    if (fp64)
        k_colnorm2<double><<<dim3(a.nblk, k), BG_THREADS, 0, st>>>(a, out);
    else
        k_colnorm2<float><<<dim3(a.nblk, k), BG_THREADS, 0, st>>>(a, out);
    return cudaGetLastError();
}

template cudaError_t bgs_iteration<float>(const BgsArgs&, int, cudaStream_t);
template cudaError_t bgs_iteration<double>(const BgsArgs&, int, cudaStream_t);
template cudaError_t bgs_cycle_start<float>(const BgsArgs&, bool, cudaStream_t);
template cudaError_t bgs_cycle_start<double>(const BgsArgs&, bool, cudaStream_t);
template cudaError_t bgs_cycle_end<float>(const BgsArgs&, cudaStream_t);
template cudaError_t bgs_cycle_end<double>(const BgsArgs&, cudaStream_t);

}  // namespace bem
