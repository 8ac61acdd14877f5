// Vector kernels of the CG-type solvers, the iterative refinement and the
// gradient's weighted sums: inner products and norms with FP64 accumulation
// (fixed reduction trees, so results do not depend on scheduling), linear
// combinations, casts between complex64 and complex128, and the residual
// r = b - Z x.  The Krylov solves are not in the paper (its Eq. 18 inverts the
// compressed operator directly); they are the iterative counterpart applied to
// the same compressed product.  The batched GMRES has its own kernels (gmres.cu).
#include "common.cuh"

namespace bem {

template <typename R>
__device__ __forceinline__ c128 to128(cx<R> a) {
    return mk<double>((double)a.re, (double)a.im);
}

template <typename S, typename D>
__global__ void k_cast(const cx<S>* __restrict__ s, cx<D>* __restrict__ d, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = mk<D>((D)s[i].re, (D)s[i].im);
}

template <typename R>
cudaError_t kv_cast(const void* src, int src_dtype, cx<R>* dst, int64_t n, cudaStream_t st) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (src_dtype == BEM_C64)
        k_cast<float, R><<<blocks, 256, 0, st>>>((const c64*)src, dst, n);
    else
        k_cast<double, R><<<blocks, 256, 0, st>>>((const c128*)src, dst, n);
    return cudaGetLastError();
}
template cudaError_t kv_cast<float>(const void*, int, c64*, int64_t, cudaStream_t);
template cudaError_t kv_cast<double>(const void*, int, c128*, int64_t, cudaStream_t);

// partial[l * npart + blk] = sum over this CTA's rows of conj(V_l[i]) w[i], l < k
template <typename R>
__global__ void k_multidot(const cx<R>* __restrict__ V, int64_t ld, int k, const cx<R>* __restrict__ w, int64_t n,
                           c128* __restrict__ partial) {
    __shared__ double sre[32], sim[32];
    int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    int64_t a = blockIdx.x * chunk, b = min(n, a + chunk);
    for (int l = 0; l < k; ++l) {
        double re = 0, im = 0;
        const cx<R>* v = V + (int64_t)l * ld;
        for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) {
            cx<R> x = v[i], y = w[i];
            re += (double)x.re * y.re + (double)x.im * y.im;
            im += (double)x.re * y.im - (double)x.im * y.re;
        }
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
        }
        int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 0) {
            sre[wid] = re;
            sim[wid] = im;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double r2 = 0, i2 = 0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
                r2 += sre[q];
                i2 += sim[q];
            }
            partial[(int64_t)l * gridDim.x + blockIdx.x] = mk<double>(r2, i2);
        }
        __syncthreads();
    }
}

cudaError_t kv_multidot(const void* V, int dtype, int64_t ld, int k, const void* w, int64_t n, c128* out_partial,
                        int npart, cudaStream_t st) {
    if (k <= 0) return cudaSuccess;
    if (dtype == BEM_C64)
        k_multidot<float><<<npart, 256, 0, st>>>((const c64*)V, ld, k, (const c64*)w, n, out_partial);
    else
        k_multidot<double><<<npart, 256, 0, st>>>((const c128*)V, ld, k, (const c128*)w, n, out_partial);
    return cudaGetLastError();
}

// out[c] = sum_p partial[c * npart + p], in a fixed order (one thread per output)
__global__ void k_reduce_c(const c128* __restrict__ partial, int npart, int count, c128* __restrict__ out) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= count) return;
    c128 s = mk<double>(0, 0);
    for (int p = 0; p < npart; ++p) s = s + partial[(int64_t)c * npart + p];
    out[c] = s;
}
cudaError_t kv_reduce_partials(const c128* partial, int npart, int count, c128* out, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    k_reduce_c<<<(count + 63) / 64, 64, 0, st>>>(partial, npart, count, out);
    return cudaGetLastError();
}
__global__ void k_reduce_r(const double* __restrict__ partial, int npart, int count, double* __restrict__ out) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= count) return;
    double s = 0;
    for (int p = 0; p < npart; ++p) s += partial[(int64_t)c * npart + p];
    out[c] = s;
}
cudaError_t kv_reduce_real(const double* partial, int npart, int count, double* out, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    k_reduce_r<<<(count + 63) / 64, 64, 0, st>>>(partial, npart, count, out);
    return cudaGetLastError();
}

// w[i] += sign * sum_l h[l] V_l[i]
template <typename R>
__global__ void k_update(cx<R>* __restrict__ w, const cx<R>* __restrict__ V, int64_t ld, int k,
                         const c128* __restrict__ h, double sign, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        c128 acc = mk<double>(0, 0);
        for (int l = 0; l < k; ++l) cfma(acc, h[l], to128(V[(int64_t)l * ld + i]));
        c128 cur = to128(w[i]);
        cur = cur + sign * acc;
        w[i] = mk<R>((R)cur.re, (R)cur.im);
    }
}

cudaError_t kv_update(void* w, const void* V, int dtype, int64_t ld, int k, const c128* h, double sign, int64_t n,
                      cudaStream_t st) {
    if (k <= 0) return cudaSuccess;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (dtype == BEM_C64)
        k_update<float><<<blocks, 256, 0, st>>>((c64*)w, (const c64*)V, ld, k, h, sign, n);
    else
        k_update<double><<<blocks, 256, 0, st>>>((c128*)w, (const c128*)V, ld, k, h, sign, n);
    return cudaGetLastError();
}

// y (complex128) += sign * sum_l coef[l] X_l, X of either precision
template <typename R>
__global__ void k_axpy128(c128* __restrict__ y, const cx<R>* __restrict__ X, int64_t ld, int k,
                          const c128* __restrict__ coef, double sign, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        c128 acc = mk<double>(0, 0);
        for (int l = 0; l < k; ++l) cfma(acc, coef[l], to128(X[(int64_t)l * ld + i]));
        y[i] = y[i] + sign * acc;
    }
}

cudaError_t kv_axpy_c128(c128* y, const void* x, int dtype, const c128* coef, double sign, int64_t n, int k,
                         int64_t ld, cudaStream_t st) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (dtype == BEM_C64)
        k_axpy128<float><<<blocks, 256, 0, st>>>(y, (const c64*)x, ld, k, coef, sign, n);
    else
        k_axpy128<double><<<blocks, 256, 0, st>>>(y, (const c128*)x, ld, k, coef, sign, n);
    return cudaGetLastError();
}

template <typename R>
__global__ void k_norm2(const cx<R>* __restrict__ w, int64_t n, double* __restrict__ partial) {
    __shared__ double sh[32];
    double s = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += (double)w[i].re * w[i].re + (double)w[i].im * w[i].im;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[wid] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
        partial[blockIdx.x] = t;
    }
}

cudaError_t kv_norm2(const void* w, int dtype, int64_t n, double* out_partial, int npart, cudaStream_t st) {
    if (dtype == BEM_C64)
        k_norm2<float><<<npart, 256, 0, st>>>((const c64*)w, n, out_partial);
    else
        k_norm2<double><<<npart, 256, 0, st>>>((const c128*)w, n, out_partial);
    return cudaGetLastError();
}

template <typename R>
__global__ void k_sub(const cx<R>* __restrict__ b, const cx<R>* __restrict__ zx, cx<R>* __restrict__ r, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = b[i] - zx[i];
}
cudaError_t kv_sub(const void* b, const void* zx, void* r, int dtype, int64_t n, cudaStream_t st) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (dtype == BEM_C64)
        k_sub<float><<<blocks, 256, 0, st>>>((const c64*)b, (const c64*)zx, (c64*)r, n);
    else
        k_sub<double><<<blocks, 256, 0, st>>>((const c128*)b, (const c128*)zx, (c128*)r, n);
    return cudaGetLastError();
}

// z = a x + b y + c w (complex coefficients, FP64 arithmetic, any of x, y, w may be
// null; z may alias them): the fused vector update of the CG-type solvers.
template <typename R>
__global__ void k_lincomb(cx<R>* z, c128 a, const cx<R>* x, c128 b, const cx<R>* y, c128 c, const cx<R>* w,
                          int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        c128 acc = mk<double>(0, 0);
        if (x) acc = acc + a * to128(x[i]);
        if (y) acc = acc + b * to128(y[i]);
        if (w) acc = acc + c * to128(w[i]);
        z[i] = mk<R>((R)acc.re, (R)acc.im);
    }
}

cudaError_t kv_lincomb(void* z, int dtype, c128 a, const void* x, c128 b, const void* y, c128 c, const void* w,
                       int64_t n, cudaStream_t st) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (dtype == BEM_C64)
        k_lincomb<float><<<blocks, 256, 0, st>>>((c64*)z, a, (const c64*)x, b, (const c64*)y, c, (const c64*)w, n);
    else
        k_lincomb<double><<<blocks, 256, 0, st>>>((c128*)z, a, (const c128*)x, b, (const c128*)y, c, (const c128*)w,
                                                  n);
    return cudaGetLastError();
}

// Layered bodies (several closed surfaces between homogeneous regions): the
// product is a sum over regions of each region's single-medium operator acting
// on the currents of that region's boundary, taken with the sign +1 where the
// region lies on the surface's normal side and -1 behind it.  These two kernels
// move a vector between the body's unknowns and one region's: element e of the
// region's boundary is edge edges[e] of the body, in both halves [J ; M] of each
// of the nrhs columns (column-major, 2 ne and 2 ns long).
template <typename R>
__global__ void k_region_gather(const cx<R>* __restrict__ x, int64_t ne, const int* __restrict__ edges,
                                const signed char* __restrict__ sign, int64_t ns, int64_t total,
                                cx<R>* __restrict__ xs) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t col = i / (2 * ns), rem = i - col * 2 * ns;
        const int64_t h = rem >= ns ? 1 : 0, e = rem - h * ns;
        cx<R> v = x[col * 2 * ne + h * ne + edges[e]];
        if (sign[e] < 0) v = mk<R>(-v.re, -v.im);
        xs[i] = v;
    }
}

template <typename R>
__global__ void k_region_scatter_add(const cx<R>* __restrict__ ys, int64_t ne, const int* __restrict__ edges,
                                     const signed char* __restrict__ sign, int64_t ns, int64_t total,
                                     cx<R>* __restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t col = i / (2 * ns), rem = i - col * 2 * ns;
        const int64_t h = rem >= ns ? 1 : 0, e = rem - h * ns;
        cx<R> v = ys[i];
        if (sign[e] < 0) v = mk<R>(-v.re, -v.im);
        cx<R>& d = y[col * 2 * ne + h * ne + edges[e]];
        d = d + v;
    }
}

static int region_blocks(int64_t total) {
    int64_t b = (total + 255) / 256;
    return (int)(b > 16 * 152 ? 16 * 152 : b);
}

cudaError_t region_gather(const void* x, int esize, int64_t ne, const int* edges, const signed char* sign,
                          int64_t ns, int nrhs, void* xs, cudaStream_t st) {
    const int64_t total = 2 * ns * (int64_t)nrhs;
    if (total <= 0) return cudaSuccess;
    if (esize == 16)
        k_region_gather<double><<<region_blocks(total), 256, 0, st>>>((const c128*)x, ne, edges, sign, ns, total,
                                                                      (c128*)xs);
    else
        k_region_gather<float><<<region_blocks(total), 256, 0, st>>>((const c64*)x, ne, edges, sign, ns, total,
                                                                     (c64*)xs);
    return cudaGetLastError();
}

cudaError_t region_scatter_add(const void* ys, int esize, int64_t ne, const int* edges, const signed char* sign,
                               int64_t ns, int nrhs, void* y, cudaStream_t st) {
    const int64_t total = 2 * ns * (int64_t)nrhs;
    if (total <= 0) return cudaSuccess;
    if (esize == 16)
        k_region_scatter_add<double><<<region_blocks(total), 256, 0, st>>>((const c128*)ys, ne, edges, sign, ns,
                                                                           total, (c128*)y);
    else
        k_region_scatter_add<float><<<region_blocks(total), 256, 0, st>>>((const c64*)ys, ne, edges, sign, ns,
                                                                          total, (c64*)y);
    return cudaGetLastError();
}

}  // namespace bem
