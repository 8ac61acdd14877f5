// The paper's two-dimensional fast direct solver (Sec. III) on the GPU, FP64:
//   C_p = N~ G^-1 S + (G/2 - D*~) G^-1 (G/2 + D*)     (Eq. 16, Calderon-preconditioned
//         CFIE; ~ marks the complexified wavenumber k~ = k0 - 0.4 j k0^(1/3) a^(-2/3))
//   C_p,c: the same operator of the regular polygon with the same vertex count and
//         perimeter, circulant, inverted by FFT
//   C_p - C_p,c ~ U V^T: adaptive randomized range finder on Gaussian test blocks
//         (Eq. 17), and C_p^-1 b by the Woodbury identity (Eq. 18).
// Building blocks: a tiled complex GEMM on general strides, solves with the Gram
// matrix of the hat functions (cyclic tridiagonal, Thomas elimination with the
// Sherman-Morrison correction, one thread per row or column), a batched FFT of any
// length (Bluestein's chirp convolution on a radix-2 Stockham transform in shared
// memory), block Gram-Schmidt, and an LU solve of the small Woodbury core.
#include "common.cuh"

#include <cstdio>

namespace bem2p {

using bem::DevBuf;
using bem::dalloc;
using bem::dfree;

// ---------------------------------------------------------------------------
// complex GEMM: C = alpha op(A) op(B) + beta C, operands addressed by strides
// (element (i, l) of A at A[i * ars + l * acs]; conj flags per operand)
// ---------------------------------------------------------------------------
constexpr int GT = 16;  // tile edge; 16 x 16 threads, one output each

struct Mat {
    const c128* p;
    int64_t rs, cs;
    int conj;
};

__global__ void __launch_bounds__(GT* GT) k_zgemm(int m, int n, int kd, c128 alpha, Mat A, Mat B, c128 beta,
                                                   c128* C, int64_t crs, int64_t ccs) {
    __shared__ c128 sa[GT][GT + 1], sb[GT][GT + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = blockIdx.y * GT + ty, j = blockIdx.x * GT + tx;
    c128 acc = mk<double>(0, 0);
    for (int l0 = 0; l0 < kd; l0 += GT) {
        {
            const int l = l0 + tx;
            c128 v = mk<double>(0, 0);
            if (i < m && l < kd) v = A.p[(int64_t)i * A.rs + (int64_t)l * A.cs];
            if (A.conj) v.im = -v.im;
            sa[ty][tx] = v;
        }
        {
            const int l = l0 + ty;
            c128 v = mk<double>(0, 0);
            if (l < kd && j < n) v = B.p[(int64_t)l * B.rs + (int64_t)j * B.cs];
            if (B.conj) v.im = -v.im;
            sb[ty][tx] = v;
        }
        __syncthreads();
#pragma unroll
        for (int l = 0; l < GT; ++l) cfma(acc, sa[ty][l], sb[l][tx]);
        __syncthreads();
    }
    if (i < m && j < n) {
        c128* c = C + (int64_t)i * crs + (int64_t)j * ccs;
        const c128 old = (beta.re == 0 && beta.im == 0) ? mk<double>(0, 0) : beta * *c;
        *c = old + alpha * acc;
    }
}

cudaError_t zgemm(int m, int n, int kd, c128 alpha, Mat A, Mat B, c128 beta, c128* C, int64_t crs, int64_t ccs,
                  cudaStream_t st) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    dim3 grid((n + GT - 1) / GT, (m + GT - 1) / GT), block(GT, GT);
    k_zgemm<<<grid, block, 0, st>>>(m, n, kd, alpha, A, B, beta, C, crs, ccs);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Gram matrix of the hat functions on a closed polygon: G_ii = (L_{i-1} + L_i) / 3,
// G_{i,i+1} = G_{i+1,i} = L_i / 6 (segment i runs from vertex i to i + 1).  Solves
// G y = x along one row or column of a matrix: the cyclic tridiagonal system is
// split as T + u v^T (T tridiagonal, u = (gamma, 0, .., c_n), v = (1, 0, .., a_1 /
// gamma)) and solved by two Thomas sweeps (Sherman-Morrison).  The factors of T
// are the same for every right-hand side and come from the host.
// ---------------------------------------------------------------------------
struct GramLU {
    const double* l;    // n: sub-diagonal multipliers of T's elimination
    const double* d;    // n: pivots
    const double* up;   // n: super-diagonal of T
    const double* z;    // n: T^-1 u
    double vz1;         // 1 + v . z
    double v_last;      // v_{n-1} = a_0 / gamma
    int n;
};

// y = G^-1 x for the vector at x (stride s), written in place
__device__ void gram_solve(const GramLU& g, c128* x, int64_t s) {
    const int n = g.n;
    // T w = x: forward elimination, back substitution
    for (int i = 1; i < n; ++i) x[i * s] = x[i * s] - g.l[i] * x[(i - 1) * s];
    x[(n - 1) * s] = (1.0 / g.d[n - 1]) * x[(n - 1) * s];
    for (int i = n - 2; i >= 0; --i) x[i * s] = (1.0 / g.d[i]) * (x[i * s] - g.up[i] * x[(i + 1) * s]);
    // y = w - z (v . w) / (1 + v . z)
    const c128 vw = x[0] + g.v_last * x[(n - 1) * s];
    const c128 f = (1.0 / g.vz1) * vw;
    for (int i = 0; i < n; ++i) x[i * s] = x[i * s] - g.z[i] * f;
}

// rows (right = 1: X <- X G^-1, one thread per row) or columns (X <- G^-1 X)
__global__ void k_gram_solve(GramLU g, c128* X, int right) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= g.n) return;
    if (right)
        gram_solve(g, X + (int64_t)r * g.n, 1);  // G symmetric: (X G^-1)_row = G^-1 x_row
    else
        gram_solve(g, X + r, g.n);
}

// X <- X + s G (the tridiagonal pattern added in place)
__global__ void k_add_gram(c128* X, int n, const double* L, double s) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int ip = (i + 1) % n, im = (i + n - 1) % n;
    X[(int64_t)i * n + i].re += s * (L[im] + L[i]) / 3.0;
    X[(int64_t)i * n + ip].re += s * L[i] / 6.0;
    X[(int64_t)i * n + im].re += s * L[im] / 6.0;
}

// ---------------------------------------------------------------------------
// FFT of any length n (numpy's convention: forward sum_j x_j exp(-2 pi i jk/n),
// inverse with 1/n), batched over vectors at x + b * bstride with element stride
// s.  Bluestein: with jk = (j^2 + k^2 - (k - j)^2) / 2,
//   X_k = w_k sum_j (x_j w_j) conj(w_{k-j}),  w_j = exp(-pi i j^2 / n)
// (signs flipped for the inverse), a linear convolution of length 2n - 1 done as a
// cyclic one of length M = 2^p >= 2n - 1 by two radix-2 transforms.  The spectrum
// of the chirp is computed once per (n, direction) and kept.  One CTA per vector,
// the whole length-M work array and its ping-pong copy in shared memory
// (M <= 4096: n <= 2048).
// ---------------------------------------------------------------------------
constexpr int FFT_THREADS = 512;
constexpr int FFT_MAXM = 4096;

// exp(sign pi i j^2 / n) with j^2 reduced mod 2n in integers (exact phase)
__device__ __forceinline__ c128 chirp(int64_t j, int n, double sign) {
    const int64_t q = (j * j) % (2 * (int64_t)n);
    double sn, cs;
    sincospi(sign * (double)q / (double)n, &sn, &cs);
    return mk<double>(cs, sn);
}

// in-place radix-2 Stockham transform of a[0..M) in shared memory (ping-pong with
// b), forward (dir = -1) or inverse without scaling (dir = +1); result in a
__device__ void stockham(c128* a, c128* b, int M, double dir) {
    c128* src = a;
    c128* dst = b;
    for (int half = M / 2, len = 1; half >= 1; half >>= 1, len <<= 1) {
        // stage: M/2 butterflies; element (p, q): p < len (twiddle), q < half
        for (int t = threadIdx.x; t < M / 2; t += blockDim.x) {
            const int p = t / half, q = t - p * half;
            double sn, cs;
            sincospi(dir * (double)p / (double)len, &sn, &cs);
            const c128 w = mk<double>(cs, sn);
            const c128 u = src[q + half * (2 * p)];
            const c128 v = src[q + half * (2 * p + 1)];
            const c128 wv = w * v;
            dst[q + half * p] = u + wv;
            dst[q + half * (p + len)] = u - wv;
        }
        __syncthreads();
        c128* tmp = src;
        src = dst;
        dst = tmp;
    }
    if (src != a) {
        for (int t = threadIdx.x; t < M; t += blockDim.x) a[t] = src[t];
        __syncthreads();
    }
}

// spectrum of the chirp kernel h_m = conj(w_m) = exp(-sign pi i m^2 / n) for
// m in (-n, n), placed cyclically in length M
__global__ void k_chirp_spectrum(c128* H, int n, int M, double sign) {
    extern __shared__ c128 fsm[];
    c128* a = fsm;
    c128* b = fsm + M;
    for (int t = threadIdx.x; t < M; t += blockDim.x) {
        const int64_t m = t < n ? t : (t > M - n ? (int64_t)M - t : -1);  // |m| of the cyclic position
        a[t] = m < 0 ? mk<double>(0, 0) : chirp(m, n, -sign);
    }
    __syncthreads();
    stockham(a, b, M, -1.0);
    for (int t = threadIdx.x; t < M; t += blockDim.x) H[t] = a[t];
}

__global__ void k_bluestein(c128* x, int n, int64_t s, int64_t bstride, int M, const c128* __restrict__ H,
                            double sign, double scale) {
    extern __shared__ c128 fsm[];
    c128* a = fsm;
    c128* b = fsm + M;
    c128* v = x + (int64_t)blockIdx.x * bstride;
    for (int t = threadIdx.x; t < M; t += blockDim.x) a[t] = t < n ? v[t * s] * chirp(t, n, sign) : mk<double>(0, 0);
    __syncthreads();
    stockham(a, b, M, -1.0);
    for (int t = threadIdx.x; t < M; t += blockDim.x) a[t] = a[t] * H[t];
    __syncthreads();
    stockham(a, b, M, 1.0);
    const double inv = scale / (double)M;
    for (int t = threadIdx.x; t < n; t += blockDim.x) v[t * s] = (inv * a[t]) * chirp(t, n, sign);
}

// X[i][j] <- s * Y[j][i] (n x n row-major, out of place)
__global__ void k_transpose_scaled(const c128* __restrict__ Y, c128* __restrict__ X, int n, double s) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * n) return;
    const int i = (int)(e / n), j = (int)(e % n);
    X[e] = s * Y[(int64_t)j * n + i];
}

// x[i + b * n] /= lam[i] (spectra of nb columns)
__global__ void k_spectrum_divide(c128* x, const c128* __restrict__ lam, int n, int nb) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * nb) return;
    x[e] = cdiv(x[e], lam[e % n]);
}

// A <- A + I (r x r row-major)
__global__ void k_add_identity(c128* A, int r) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < r) A[(int64_t)i * r + i].re += 1.0;
}

// out[c] = |Y_c| for the nb columns of Y (n x nb column-major), one CTA per column
__global__ void k_col_norms(const c128* __restrict__ Y, int n, double* out) {
    __shared__ double red[32];
    const c128* y = Y + (int64_t)blockIdx.x * n;
    double s = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += cabs2(y[i]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        out[blockIdx.x] = sqrt(t);
    }
}

// block reduction of a complex value over the CTA (fixed order)
__device__ c128 block_sum(c128 v, c128* red) {
    for (int o = 16; o > 0; o >>= 1) {
        v.re += __shfl_xor_sync(0xffffffffu, v.re, o);
        v.im += __shfl_xor_sync(0xffffffffu, v.im, o);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    c128 t = mk<double>(0, 0);
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = t + red[w];
    return t;
}

// Gram-Schmidt (twice) of the nb columns of Y (n x nb column-major) among
// themselves, each normalised: the orthonormal basis of the block.  One CTA.
__global__ void k_block_qr(c128* Y, int n, int nb) {
    __shared__ c128 red[32];
    for (int c = 0; c < nb; ++c) {
        c128* y = Y + (int64_t)c * n;
        for (int pass = 0; pass < 2; ++pass)
            for (int d = 0; d < c; ++d) {
                const c128* q = Y + (int64_t)d * n;
                c128 h = mk<double>(0, 0);
                for (int i = threadIdx.x; i < n; i += blockDim.x) h = h + cconj(q[i]) * y[i];
                h = block_sum(h, red);
                __syncthreads();
                for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = y[i] - h * q[i];
                __syncthreads();
            }
        double s = 0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) s += cabs2(y[i]);
        const c128 ss = block_sum(mk<double>(s, 0), red);
        const double nrm = sqrt(ss.re);
        __syncthreads();
        const double f = nrm > 0 ? 1.0 / nrm : 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = f * y[i];
        __syncthreads();
    }
}

// Solve A Z = R in place (A r x r row-major, R r x nr column-major) by LU with
// partial pivoting; one CTA.  status[0] = 1 if a pivot is exactly zero.
__global__ void k_lu_solve(c128* A, int r, c128* R, int nr, int* status) {
    __shared__ int s_p;
    __shared__ double s_best[32];
    __shared__ int s_idx[32];
    for (int k = 0; k < r; ++k) {
        // pivot: largest |A_ik| for i >= k (smallest index on ties)
        double best = -1.0;
        int bi = k;
        for (int i = k + threadIdx.x; i < r; i += blockDim.x) {
            const double v = cabs2(A[(int64_t)i * r + k]);
            if (v > best) {
                best = v;
                bi = i;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if ((threadIdx.x & 31) == 0) {
            s_best[threadIdx.x >> 5] = best;
            s_idx[threadIdx.x >> 5] = bi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = -1.0;
            int p = k;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
                if (s_best[w] > b || (s_best[w] == b && s_idx[w] < p)) {
                    b = s_best[w];
                    p = s_idx[w];
                }
            s_p = p;
            if (!(b > 0.0)) status[0] = 1;
        }
        __syncthreads();
        const int p = s_p;
        if (p != k) {
            for (int j = threadIdx.x; j < r; j += blockDim.x) {
                const c128 t = A[(int64_t)k * r + j];
                A[(int64_t)k * r + j] = A[(int64_t)p * r + j];
                A[(int64_t)p * r + j] = t;
            }
            for (int c = threadIdx.x; c < nr; c += blockDim.x) {
                const c128 t = R[(int64_t)c * r + k];
                R[(int64_t)c * r + k] = R[(int64_t)c * r + p];
                R[(int64_t)c * r + p] = t;
            }
        }
        __syncthreads();
        const c128 piv = A[(int64_t)k * r + k];
        const int rows = r - k - 1;
        // multipliers in column k, then the trailing update and the right-hand sides
        for (int i = k + 1 + threadIdx.x; i < r; i += blockDim.x)
            A[(int64_t)i * r + k] = (piv.re == 0 && piv.im == 0) ? mk<double>(0, 0) : cdiv(A[(int64_t)i * r + k], piv);
        __syncthreads();
        for (int64_t e = threadIdx.x; e < (int64_t)rows * (r - k - 1 + nr); e += blockDim.x) {
            const int i = k + 1 + (int)(e / (r - k - 1 + nr));
            const int jj = (int)(e % (r - k - 1 + nr));
            const c128 l = A[(int64_t)i * r + k];
            if (jj < r - k - 1) {
                const int j = k + 1 + jj;
                A[(int64_t)i * r + j] = A[(int64_t)i * r + j] - l * A[(int64_t)k * r + j];
            } else {
                const int c = jj - (r - k - 1);
                R[(int64_t)c * r + i] = R[(int64_t)c * r + i] - l * R[(int64_t)c * r + k];
            }
        }
        __syncthreads();
    }
    // back substitution, one thread per right-hand side
    for (int c = threadIdx.x; c < nr; c += blockDim.x) {
        c128* z = R + (int64_t)c * r;
        for (int i = r - 1; i >= 0; --i) {
            c128 acc = z[i];
            for (int j = i + 1; j < r; ++j) acc = acc - A[(int64_t)i * r + j] * z[j];
            const c128 d = A[(int64_t)i * r + i];
            z[i] = (d.re == 0 && d.im == 0) ? mk<double>(0, 0) : cdiv(acc, d);
        }
    }
}

}  // namespace bem2p

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
void bem_ctx_set_error(bem_ctx* c, const char* msg);  // bem_api.cu

namespace {

using bem2p::Mat;
using bem::DevBuf;
using bem::dalloc;
using bem::dfree;

struct Scope {  // device buffers freed on every exit path
    std::vector<DevBuf*> b;
    ~Scope() {
        for (DevBuf* x : b) dfree(*x);
    }
};

bem_status set_err(bem_ctx* ctx, bem_status s, const char* msg) {
    if (ctx) bem_ctx_set_error(ctx, msg);
    return s;
}

#define PP_TRY(expr)                                                            \
    do {                                                                        \
        cudaError_t _e = (expr);                                                \
        if (_e != cudaSuccess)                                                  \
            return set_err(ctx, _e == cudaErrorMemoryAllocation ? BEM_ENOMEM : BEM_ECUDA, #expr); \
    } while (0)

// segment lengths of a counter-clockwise polygon; false if it is not one
bool polygon_lengths(const double* v, int n, std::vector<double>& L) {
    if (!v || n < 3) return false;
    L.resize(n);
    double area2 = 0;
    for (int i = 0; i < n; ++i) {
        const int j = (i + 1) % n;
        const double dx = v[2 * j] - v[2 * i], dy = v[2 * j + 1] - v[2 * i + 1];
        L[i] = std::sqrt(dx * dx + dy * dy);
        if (!(L[i] > 0)) return false;
        area2 += v[2 * i] * v[2 * j + 1] - v[2 * j] * v[2 * i + 1];
    }
    return area2 > 0;
}

// factors of the hat-function Gram matrix for bem2p::gram_solve (host, FP64)
struct GramHost {
    std::vector<double> l, d, up, z;
    double vz1 = 0, v_last = 0;
};
GramHost gram_factor(const std::vector<double>& L) {
    const int n = (int)L.size();
    GramHost g;
    std::vector<double> b(n), c(n), e(n);
    for (int i = 0; i < n; ++i) {
        b[i] = (L[(i + n - 1) % n] + L[i]) / 3.0;
        c[i] = L[(i + n - 1) % n] / 6.0;  // row i, column i - 1
        e[i] = L[i] / 6.0;                // row i, column i + 1
    }
    const double alpha = L[n - 1] / 6.0, beta = L[n - 1] / 6.0;  // corners (0, n-1), (n-1, 0)
    const double gamma = -b[0];
    b[0] -= gamma;
    b[n - 1] -= alpha * beta / gamma;
    g.l.assign(n, 0.0);
    g.d.assign(n, 0.0);
    g.up = e;
    g.d[0] = b[0];
    for (int i = 1; i < n; ++i) {
        g.l[i] = c[i] / g.d[i - 1];
        g.d[i] = b[i] - g.l[i] * e[i - 1];
    }
    // z = T^-1 u, u = (gamma, 0, .., 0, beta)
    std::vector<double> z(n, 0.0);
    z[0] = gamma;
    z[n - 1] = beta;
    for (int i = 1; i < n; ++i) z[i] -= g.l[i] * z[i - 1];
    z[n - 1] /= g.d[n - 1];
    for (int i = n - 2; i >= 0; --i) z[i] = (z[i] - e[i] * z[i + 1]) / g.d[i];
    g.z = z;
    g.v_last = alpha / gamma;
    g.vz1 = 1.0 + z[0] + g.v_last * z[n - 1];
    return g;
}

cudaError_t upload_d(DevBuf& b, const std::vector<double>& v, cudaStream_t st) {
    cudaError_t e = dalloc(b, sizeof(double) * v.size());
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(b.p, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice, st);
}

Mat mat(const c128* p, int64_t rs, int64_t cs, int conj = 0) {
    Mat m;
    m.p = p;
    m.rs = rs;
    m.cs = cs;
    m.conj = conj;
    return m;
}

unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

bem_status planar_operators_row0(bem_ctx* ctx, const double* verts, int n, bem_c128 k, int fp32, void* S, void* D,
                                 void* N, void* stream);  // planar.cu

namespace {

bem_status fft_run(bem_ctx* ctx, c128* x, int n, int64_t s, int nb, int64_t bs, bool inverse, cudaStream_t st);

// true when vertex i + 1 is vertex i turned by 2 pi / n about the centroid: the
// polygon is regular and every operator on it (S, D, N, G and C_p) is circulant
bool regular_polygon(const double* v, int n) {
    double cx = 0, cy = 0;
    for (int i = 0; i < n; ++i) {
        cx += v[2 * i];
        cy += v[2 * i + 1];
    }
    cx /= n;
    cy /= n;
    const double c = std::cos(2.0 * BEM_PI / n), s = std::sin(2.0 * BEM_PI / n);
    const double r0 = std::hypot(v[0] - cx, v[1] - cy);
    for (int i = 0; i < n; ++i) {
        const int j = (i + 1) % n;
        const double x = v[2 * i] - cx, y = v[2 * i + 1] - cy;
        if (std::hypot(v[2 * j] - cx - (c * x - s * y), v[2 * j + 1] - cy - (s * x + c * y)) > 1e-11 * r0) return false;
    }
    return true;
}

// Circulant X[i][j] = r[(j - i) mod n] has eigenvalues lam_m = sum_k r_k e^{2 pi i k m / n}
// = n ifft(r)_m (eigenvectors e^{2 pi i j m / n}); X^T has lam_{-m}.  lam holds ifft of the
// rows of S, D, N, D~, N~, G; out receives the eigenvalues of C_p, L_e, L_h.
__global__ void k_circ_combine(const c128* __restrict__ lam, int n, c128* __restrict__ out) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    const int mm = (n - m) % n;
    const double sc = (double)n;
    const c128 lS = sc * lam[m], lDT = sc * lam[n + mm], lNt = sc * lam[4 * n + m], lDtT = sc * lam[3 * n + mm];
    const c128 lG = sc * lam[5 * n + m];
    const c128 g2 = 0.5 * lG;
    const c128 le = cdiv(lNt, lG), lh = cdiv(g2 - lDtT, lG);
    out[m] = le * lS + lh * (g2 + lDT);  // N~ G^-1 S + (G/2 - D~*) G^-1 (G/2 + D*)
    out[n + m] = le;
    out[2 * n + m] = lh;
}

// dense circulant from its row: out[i][j] = scale * row[(j - i) mod n]
__global__ void k_circ_expand(const c128* __restrict__ row, int n, double scale, c128* __restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * n) return;
    const int i = (int)(idx / n), j = (int)(idx % n);
    out[idx] = scale * row[(j - i + n) % n];
}

// C_p (and L_e, L_h) of a regular polygon from the first rows of its operators
bem_status calderon_circulant(bem_ctx* ctx, const double* verts, int n, bem_c128 k0, bem_c128 kt, int fp32,
                              const std::vector<double>& L, void* Cp, void* Le, void* Lh, cudaStream_t st) {
    DevBuf rows, outs;
    Scope sc{{&rows, &outs}};
    PP_TRY(dalloc(rows, sizeof(c128) * 6 * n));
    PP_TRY(dalloc(outs, sizeof(c128) * 3 * n));
    c128* r = (c128*)rows.p;
    bem_status s;
    if ((s = planar_operators_row0(ctx, verts, n, k0, fp32, r, r + n, r + 2 * n, st)) != BEM_OK) return s;
    if ((s = planar_operators_row0(ctx, verts, n, kt, fp32, nullptr, r + 3 * n, r + 4 * n, st)) != BEM_OK) return s;
    std::vector<c128> g(n, mk<double>(0.0, 0.0));  // row 0 of the hat-function Gram matrix
    g[0] = mk<double>((L[n - 1] + L[0]) / 3.0, 0.0);
    g[1] = g[1] + mk<double>(L[0] / 6.0, 0.0);
    g[n - 1] = g[n - 1] + mk<double>(L[n - 1] / 6.0, 0.0);
    PP_TRY(cudaMemcpyAsync(r + 5 * n, g.data(), sizeof(c128) * n, cudaMemcpyHostToDevice, st));
    if ((s = fft_run(ctx, r, n, 1, 6, n, true, st)) != BEM_OK) return s;
    c128* o = (c128*)outs.p;
    k_circ_combine<<<blocks_for(n, 128), 128, 0, st>>>(r, n, o);
    PP_TRY(cudaGetLastError());
    if ((s = fft_run(ctx, o, n, 1, 3, n, false, st)) != BEM_OK) return s;  // rows (times n)
    const unsigned bnn = blocks_for((int64_t)n * n, 256);
    void* dst[3] = {Cp, Le, Lh};
    for (int q = 0; q < 3; ++q)
        if (dst[q]) {
            k_circ_expand<<<bnn, 256, 0, st>>>(o + (int64_t)q * n, n, 1.0 / n, (c128*)dst[q]);
            PP_TRY(cudaGetLastError());
        }
    PP_TRY(cudaStreamSynchronize(st));
    return BEM_OK;
}

}  // namespace

extern "C" bem_status bem_planar_calderon(bem_ctx* ctx, const double* verts, int n, double k0, double a, int fp32,
                                          void* Cp, void* Le, void* Lh, void* stream) {
    using namespace bem2p;
    std::vector<double> L;
    if (!polygon_lengths(verts, n, L))
        return set_err(ctx, BEM_EINVAL, "bem_planar_calderon: need a counter-clockwise polygon of >= 3 distinct vertices");
    if (!(k0 > 0) || !Cp) return set_err(ctx, BEM_EINVAL, "bem_planar_calderon: need k0 > 0 and Cp");
    if (n > 46340) return set_err(ctx, BEM_EINVAL, "bem_planar_calderon: more than 46340 vertices");
    cudaStream_t st = (cudaStream_t)stream;
    double per = 0;
    for (double x : L) per += x;
    if (!(a > 0)) a = per / (2.0 * BEM_PI);
    const bem_c128 kk0{k0, 0.0};
    const bem_c128 kt{k0, -0.4 * std::cbrt(k0) * std::pow(a, -2.0 / 3.0)};  // k~ = k0 - 0.4 j k0^(1/3) a^(-2/3)
    // a regular polygon (the circular counterpart): everything is circulant, so the
    // first rows and FFT eigenvalues replace the dense assembly and products
    if (n <= FFT_MAXM / 2 && regular_polygon(verts, n))
        return calderon_circulant(ctx, verts, n, kk0, kt, fp32, L, Cp, Le, Lh, st);
    const size_t nn = (size_t)n * n;
    DevBuf S, D, N, Dt, Nt, W1, W2, P, gl, gd, gu, gz, dL;
    Scope sc{{&S, &D, &N, &Dt, &Nt, &W1, &W2, &P, &gl, &gd, &gu, &gz, &dL}};
    for (DevBuf* b : {&S, &D, &N, &Dt, &Nt, &W1, &W2, &P}) PP_TRY(dalloc(*b, sizeof(c128) * nn));
    bem_status s;
    if ((s = bem_planar_operators(ctx, verts, n, kk0, fp32, S.p, D.p, N.p, stream)) != BEM_OK) return s;
    if ((s = bem_planar_operators(ctx, verts, n, kt, fp32, nullptr, Dt.p, Nt.p, stream)) != BEM_OK) return s;
    const GramHost gh = gram_factor(L);
    PP_TRY(upload_d(gl, gh.l, st));
    PP_TRY(upload_d(gd, gh.d, st));
    PP_TRY(upload_d(gu, gh.up, st));
    PP_TRY(upload_d(gz, gh.z, st));
    PP_TRY(upload_d(dL, L, st));
    GramLU g;
    g.l = (const double*)gl.p;
    g.d = (const double*)gd.p;
    g.up = (const double*)gu.p;
    g.z = (const double*)gz.p;
    g.vz1 = gh.vz1;
    g.v_last = gh.v_last;
    g.n = n;
    c128* le = (c128*)W1.p;  // L_e = N~ G^-1
    c128* lh = (c128*)W2.p;  // L_h = (G/2 - D*~) G^-1
    const unsigned bn = blocks_for(n, 128), bnn = blocks_for((int64_t)nn, 256);
    PP_TRY(cudaMemcpyAsync(le, Nt.p, sizeof(c128) * nn, cudaMemcpyDeviceToDevice, st));
    k_gram_solve<<<bn, 128, 0, st>>>(g, le, 1);
    PP_TRY(cudaGetLastError());
    k_transpose_scaled<<<bnn, 256, 0, st>>>((const c128*)Dt.p, lh, n, -1.0);  // -D~^T = -D*~
    k_add_gram<<<bn, 128, 0, st>>>(lh, n, (const double*)dL.p, 0.5);
    k_gram_solve<<<bn, 128, 0, st>>>(g, lh, 1);
    k_transpose_scaled<<<bnn, 256, 0, st>>>((const c128*)D.p, (c128*)P.p, n, 1.0);  // D* = D^T
    k_add_gram<<<bn, 128, 0, st>>>((c128*)P.p, n, (const double*)dL.p, 0.5);      // G/2 + D*
    PP_TRY(cudaGetLastError());
    const c128 one = mk<double>(1, 0), zero = mk<double>(0, 0);
    c128* cp = (c128*)Cp;
    PP_TRY(zgemm(n, n, n, one, mat(le, n, 1), mat((const c128*)S.p, n, 1), zero, cp, n, 1, st));
    PP_TRY(zgemm(n, n, n, one, mat(lh, n, 1), mat((const c128*)P.p, n, 1), one, cp, n, 1, st));
    if (Le) PP_TRY(cudaMemcpyAsync(Le, le, sizeof(c128) * nn, cudaMemcpyDeviceToDevice, st));
    if (Lh) PP_TRY(cudaMemcpyAsync(Lh, lh, sizeof(c128) * nn, cudaMemcpyDeviceToDevice, st));
    PP_TRY(cudaStreamSynchronize(st));
    return BEM_OK;
}

namespace {

// batched FFT (numpy convention) of nb vectors of length n at x + b * bs, stride s
bem_status fft_run(bem_ctx* ctx, c128* x, int n, int64_t s, int nb, int64_t bs, bool inverse, cudaStream_t st) {
    using namespace bem2p;
    int M = 1;
    while (M < 2 * n - 1) M <<= 1;
    if (n < 1 || M > FFT_MAXM) return set_err(ctx, BEM_EINVAL, "bem_fft: length must be 1..2048");
    if (nb <= 0) return BEM_OK;
    const size_t smem = 2 * sizeof(c128) * M;
    static bool attr = false;
    if (!attr) {
        PP_TRY(cudaFuncSetAttribute(k_chirp_spectrum, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(2 * sizeof(c128) * FFT_MAXM)));
        PP_TRY(cudaFuncSetAttribute(k_bluestein, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(2 * sizeof(c128) * FFT_MAXM)));
        attr = true;
    }
    const double sign = inverse ? 1.0 : -1.0;
    DevBuf H;
    Scope sc{{&H}};
    PP_TRY(dalloc(H, sizeof(c128) * M));
    k_chirp_spectrum<<<1, FFT_THREADS, smem, st>>>((c128*)H.p, n, M, sign);
    PP_TRY(cudaGetLastError());
    k_bluestein<<<nb, FFT_THREADS, smem, st>>>(x, n, s, bs, M, (const c128*)H.p, sign, inverse ? 1.0 / n : 1.0);
    PP_TRY(cudaGetLastError());
    PP_TRY(cudaStreamSynchronize(st));  // H is freed on return
    return BEM_OK;
}

}  // namespace

extern "C" bem_status bem_fft(bem_ctx* ctx, void* x, int n, long long stride, int batch, long long batch_stride,
                              int inverse, void* stream) {
    if (!x || stride < 1 || batch < 0) return set_err(ctx, BEM_EINVAL, "bem_fft: bad arguments");
    return fft_run(ctx, (c128*)x, n, stride, batch, batch_stride, inverse != 0, (cudaStream_t)stream);
}

extern "C" bem_status bem_planar_skeleton(bem_ctx* ctx, const void* A, int n, const void* omega, int p, double tol,
                                          int block, void* U, void* Vt, int* rank, void* stream) {
    using namespace bem2p;
    if (!A || !omega || !U || !rank || n < 1 || p < 1 || block < 1 || !(tol > 0))
        return set_err(ctx, BEM_EINVAL, "bem_planar_skeleton: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const c128* a = (const c128*)A;
    const c128* om = (const c128*)omega;
    c128* Q = (c128*)U;  // n x p capacity, column-major
    DevBuf Y, H, nr;
    Scope sc{{&Y, &H, &nr}};
    PP_TRY(dalloc(Y, sizeof(c128) * (size_t)n * block));
    PP_TRY(dalloc(H, sizeof(c128) * (size_t)p * block));
    PP_TRY(dalloc(nr, sizeof(double) * block));
    const c128 one = mk<double>(1, 0), zero = mk<double>(0, 0), mone = mk<double>(-1, 0);
    std::vector<double> norms(block);
    double ref = -1;
    int r = 0;
    bool done = false;
    for (int c0 = 0; c0 < p && !done; c0 += block) {
        const int b = std::min(block, p - c0);
        c128* y = (c128*)Y.p;
        // Y = A Omega_block (A row-major, Omega and Y column-major)
        PP_TRY(zgemm(n, b, n, one, mat(a, n, 1), mat(om + (int64_t)c0 * n, 1, n), zero, y, 1, n, st));
        if (ref < 0) {
            k_col_norms<<<b, 256, 0, st>>>(y, n, (double*)nr.p);
            PP_TRY(cudaMemcpyAsync(norms.data(), nr.p, sizeof(double) * b, cudaMemcpyDeviceToHost, st));
            PP_TRY(cudaStreamSynchronize(st));
            ref = *std::max_element(norms.begin(), norms.begin() + b);
        }
        for (int pass = 0; pass < 2 && r > 0; ++pass) {
            // H = Q^H Y (r x b; element (i, l) of Q^H is conj(Q[l + i n])), Y -= Q H
            PP_TRY(zgemm(r, b, n, one, mat(Q, n, 1, 1), mat(y, 1, n), zero, (c128*)H.p, 1, r, st));
            PP_TRY(zgemm(n, b, r, mone, mat(Q, 1, n), mat((const c128*)H.p, 1, r), one, y, 1, n, st));
        }
        k_col_norms<<<b, 256, 0, st>>>(y, n, (double*)nr.p);
        PP_TRY(cudaMemcpyAsync(norms.data(), nr.p, sizeof(double) * b, cudaMemcpyDeviceToHost, st));
        PP_TRY(cudaStreamSynchronize(st));
        if (*std::max_element(norms.begin(), norms.begin() + b) <= tol * ref) {
            done = true;
            break;
        }
        k_block_qr<<<1, 256, 0, st>>>(y, n, b);
        const int take = std::min(b, n - r);
        PP_TRY(cudaMemcpyAsync(Q + (int64_t)r * n, y, sizeof(c128) * (size_t)n * take, cudaMemcpyDeviceToDevice, st));
        r += take;
        if (r >= n) done = true;  // the whole space: the skeleton is exact
    }
    if (!done) return set_err(ctx, BEM_ENOCONV, "bem_planar_skeleton: the test vectors ran out before the tolerance");
    // V^T = Q^H A (r x n, row-major)
    if (Vt) PP_TRY(zgemm(r, n, n, one, mat(Q, n, 1, 1), mat(a, n, 1), zero, (c128*)Vt, n, 1, st));
    PP_TRY(cudaStreamSynchronize(st));
    *rank = r;
    return BEM_OK;
}

extern "C" bem_status bem_planar_woodbury_solve(bem_ctx* ctx, const void* cc0, int n, const void* U, const void* Vt,
                                                int r, const void* b, void* x, int nrhs, void* stream) {
    using namespace bem2p;
    if (!cc0 || !b || !x || n < 1 || nrhs < 1 || r < 0 || (r > 0 && (!U || !Vt)))
        return set_err(ctx, BEM_EINVAL, "bem_planar_woodbury_solve: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    DevBuf lam, CU, cap, rhs, stat;
    Scope sc{{&lam, &CU, &cap, &rhs, &stat}};
    PP_TRY(dalloc(lam, sizeof(c128) * n));
    PP_TRY(cudaMemcpyAsync(lam.p, cc0, sizeof(c128) * n, cudaMemcpyDeviceToDevice, st));
    bem_status s;
    if ((s = fft_run(ctx, (c128*)lam.p, n, 1, 1, n, false, st)) != BEM_OK) return s;  // eigenvalues of C_p,c
    // y = C_c^-1 b by FFT, in x
    c128* y = (c128*)x;
    PP_TRY(cudaMemcpyAsync(y, b, sizeof(c128) * (size_t)n * nrhs, cudaMemcpyDeviceToDevice, st));
    if ((s = fft_run(ctx, y, n, 1, nrhs, n, false, st)) != BEM_OK) return s;
    k_spectrum_divide<<<blocks_for((int64_t)n * nrhs, 256), 256, 0, st>>>(y, (const c128*)lam.p, n, nrhs);
    PP_TRY(cudaGetLastError());
    if ((s = fft_run(ctx, y, n, 1, nrhs, n, true, st)) != BEM_OK) return s;
    if (r == 0) {
        PP_TRY(cudaStreamSynchronize(st));
        return BEM_OK;
    }
    // CU = C_c^-1 U (n x r column-major)
    PP_TRY(dalloc(CU, sizeof(c128) * (size_t)n * r));
    PP_TRY(cudaMemcpyAsync(CU.p, U, sizeof(c128) * (size_t)n * r, cudaMemcpyDeviceToDevice, st));
    if ((s = fft_run(ctx, (c128*)CU.p, n, 1, r, n, false, st)) != BEM_OK) return s;
    k_spectrum_divide<<<blocks_for((int64_t)n * r, 256), 256, 0, st>>>((c128*)CU.p, (const c128*)lam.p, n, r);
    PP_TRY(cudaGetLastError());
    if ((s = fft_run(ctx, (c128*)CU.p, n, 1, r, n, true, st)) != BEM_OK) return s;
    // cap = I + V^T CU (r x r row-major); rhs = V^T y (r x nrhs column-major)
    PP_TRY(dalloc(cap, sizeof(c128) * (size_t)r * r));
    PP_TRY(dalloc(rhs, sizeof(c128) * (size_t)r * nrhs));
    PP_TRY(dalloc(stat, sizeof(int)));
    PP_TRY(cudaMemsetAsync(stat.p, 0, sizeof(int), st));
    const c128 one = mk<double>(1, 0), zero = mk<double>(0, 0), mone = mk<double>(-1, 0);
    const c128* vt = (const c128*)Vt;
    PP_TRY(zgemm(r, r, n, one, mat(vt, n, 1), mat((const c128*)CU.p, 1, n), zero, (c128*)cap.p, r, 1, st));
    k_add_identity<<<blocks_for(r, 128), 128, 0, st>>>((c128*)cap.p, r);
    PP_TRY(cudaGetLastError());
    PP_TRY(zgemm(r, nrhs, n, one, mat(vt, n, 1), mat(y, 1, n), zero, (c128*)rhs.p, 1, r, st));
    // z = cap^-1 rhs; x = y - CU z
    k_lu_solve<<<1, 256, 0, st>>>((c128*)cap.p, r, (c128*)rhs.p, nrhs, (int*)stat.p);
    PP_TRY(cudaGetLastError());
    PP_TRY(zgemm(n, nrhs, r, mone, mat((const c128*)CU.p, 1, n), mat((const c128*)rhs.p, 1, r), one, y, 1, n, st));
    int hst = 0;
    PP_TRY(cudaMemcpyAsync(&hst, stat.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    PP_TRY(cudaStreamSynchronize(st));
    if (hst) return set_err(ctx, BEM_EINVAL, "bem_planar_woodbury_solve: the Woodbury core is singular");
    return BEM_OK;
}
