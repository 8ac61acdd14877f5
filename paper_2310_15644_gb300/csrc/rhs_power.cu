// Plane-wave right-hand sides and power functionals.
//
// Right-hand side (tested incident fields after Eq. 8): for every RWG edge n and
// plane wave r, e_n = int f_n . E_inc and (eta0 h)_n = int f_n . (khat x E_inc),
// E_inc = e0 exp(-j k0 khat.r), by the 7-point rule on T+ and T-, in FP64.
//
// Powers (the dosimetric output, Sec. I): with J = n x H, M = E x n,
//   absorbed     Re(xJ^H X xM),   X[m,n] = int f_m . (n x f_n)  (per triangle, exact)
//   extinguished Re(xJ^H bJ + bM^H xM)
//   scattered    oint |E_far|^2 dOmega, E_far = (j k0 / 4pi)(rhat x L - N_t),
//                N = int (eta0 J) e^{j k0 rhat.r}, L = int M e^{j k0 rhat.r},
// all in units of 1/(2 eta0), summed in FP64 with fixed reduction trees.
#include "common.cuh"
#include "geom.cuh"

namespace bem {

template <typename R>
__global__ void k_rhs(GeomDev g, const double* __restrict__ khat, const c128* __restrict__ e0, int nrhs,
                      cx<R>* __restrict__ b) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    if (n >= g.ne) return;
    d3 kh = ld3(khat + 3 * r);
    c128 E0[3] = {e0[3 * r], e0[3 * r + 1], e0[3 * r + 2]};
    c128 ee = mk<double>(0, 0), hh = ee;
    for (int s = 0; s < 2; ++s) {
        int tri = g.edge_tri[2 * n + s], li = g.edge_loc[2 * n + s];
        d3 v[3];
        for (int i = 0; i < 3; ++i) v[i] = ld3(g.tv + 9 * tri + 3 * i);
        double A = g.area[tri];
        double c = g.tri_coef[3 * tri + li] / (2.0 * A);
        for (int q = 0; q < 7; ++q) {
            double l0, l1, l2, w;
            rule7_d(q, l0, l1, l2, w);
            d3 rq = l0 * v[0] + l1 * v[1] + l2 * v[2];
            d3 f = c * (rq - v[li]);
            double ph = -g.k0 * dot(kh, rq);
            double sn, cs;
            sincos(ph, &sn, &cs);
            c128 e = mk<double>(cs, sn);
            c128 E[3] = {e * E0[0], e * E0[1], e * E0[2]};
            // khat x E
            c128 H[3] = {kh.y * E[2] - kh.z * E[1], kh.z * E[0] - kh.x * E[2], kh.x * E[1] - kh.y * E[0]};
            double wA = w * A;
            ee = ee + wA * (f.x * E[0] + f.y * E[1] + f.z * E[2]);
            hh = hh + wA * (f.x * H[0] + f.y * H[1] + f.z * H[2]);
        }
    }
    int64_t base = (int64_t)r * 2 * g.ne;
    b[base + n] = mk<R>((R)ee.re, (R)ee.im);
    b[base + g.ne + n] = mk<R>((R)hh.re, (R)hh.im);
}

template <typename R>
cudaError_t rhs_planewave(GeomDev g, const double* khat, const c128* e0, int nrhs, cx<R>* b, cudaStream_t st) {
    if (nrhs <= 0) return cudaSuccess;
    dim3 grid((g.ne + 127) / 128, nrhs);
    k_rhs<R><<<grid, 128, 0, st>>>(g, khat, e0, nrhs, b);
    return cudaGetLastError();
}
template cudaError_t rhs_planewave<float>(GeomDev, const double*, const c128*, int, c64*, cudaStream_t);
template cudaError_t rhs_planewave<double>(GeomDev, const double*, const c128*, int, c128*, cudaStream_t);

__device__ double block_sum_d(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
    __syncthreads();
    return s;  // valid in thread 0
}

// absorbed power per triangle and per-CTA partial sums (grid.y = right-hand side)
__global__ void k_pabs(GeomDev g, const c128* __restrict__ x, double* __restrict__ per_tri,
                       double* __restrict__ partial) {
    __shared__ double sh[32];
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    const c128* xr = x + (int64_t)r * 2 * g.ne;
    double p = 0.0;
    if (t < g.nt) {
        d3 v[3];
        for (int i = 0; i < 3; ++i) v[i] = ld3(g.tv + 9 * t + 3 * i);
        d3 n = ld3(g.nrm + 3 * t);
        double A = g.area[t];
        double X[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int q = 0; q < 7; ++q) {
            double l0, l1, l2, w;
            rule7_d(q, l0, l1, l2, w);
            d3 rq = l0 * v[0] + l1 * v[1] + l2 * v[2];
            d3 f[3];
            for (int i = 0; i < 3; ++i) f[i] = (g.tri_coef[3 * t + i] / (2.0 * A)) * (rq - v[i]);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) X[i][j] += w * A * dot(f[i], cross(n, f[j]));
        }
        c128 acc = mk<double>(0, 0);
        for (int i = 0; i < 3; ++i) {
            c128 xj = xr[g.tri_edge[3 * t + i]];
            for (int j = 0; j < 3; ++j) {
                c128 xm = xr[g.ne + g.tri_edge[3 * t + j]];
                cfma_conj(acc, xj, X[i][j] * xm);
            }
        }
        p = acc.re;
        if (per_tri && r == 0) per_tri[t] = p / A;
    }
    double s = block_sum_d(p, sh);
    if (threadIdx.x == 0 && partial) partial[(int64_t)r * gridDim.x + blockIdx.x] = s;
}

// Local 3 x 3 twisted Gram matrix of triangle t: X[i][j] = int_t f_i . (n x f_j) dS
// (7-point rule, exact for this quadratic integrand), FP64.
__device__ void twisted_gram_local(const GeomDev& g, int t, double X[3][3]) {
    d3 v[3];
    for (int i = 0; i < 3; ++i) v[i] = ld3(g.tv + 9 * t + 3 * i);
    d3 n = ld3(g.nrm + 3 * t);
    double A = g.area[t];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) X[i][j] = 0.0;
    for (int q = 0; q < 7; ++q) {
        double l0, l1, l2, w;
        rule7_d(q, l0, l1, l2, w);
        d3 rq = l0 * v[0] + l1 * v[1] + l2 * v[2];
        d3 f[3];
        for (int i = 0; i < 3; ++i) f[i] = (g.tri_coef[3 * t + i] / (2.0 * A)) * (rq - v[i]);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) X[i][j] += w * A * dot(f[i], cross(n, f[j]));
    }
}

// Gradient of the absorbed power P = Re(xJ^H X xM) = x^H H x, H = (1/2)[[0, X], [X^T, 0]]
// (X real), with respect to conj(x): out = H x = (1/2) [X xM ; X^T xJ].  One thread per
// edge gathers the contributions of its two triangles (no atomics); grid.y = rhs.
__global__ void k_pabs_grad(GeomDev g, const c128* __restrict__ x, c128* __restrict__ out) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (m >= g.ne) return;
    const c128* xr = x + (int64_t)r * 2 * g.ne;
    c128 gJ = mk<double>(0, 0), gM = gJ;
    for (int s = 0; s < 2; ++s) {
        const int t = g.edge_tri[2 * m + s], li = g.edge_loc[2 * m + s];
        double X[3][3];
        twisted_gram_local(g, t, X);
        for (int j = 0; j < 3; ++j) {
            const int e = g.tri_edge[3 * t + j];
            gJ = gJ + X[li][j] * xr[g.ne + e];
            gM = gM + X[j][li] * xr[e];
        }
    }
    c128* o = out + (int64_t)r * 2 * g.ne;
    o[m] = 0.5 * gJ;
    o[g.ne + m] = 0.5 * gM;
}

cudaError_t power_abs_grad(GeomDev g, const c128* x, int nrhs, c128* out, cudaStream_t st) {
    dim3 grid((g.ne + 127) / 128, nrhs);
    k_pabs_grad<<<grid, 128, 0, st>>>(g, x, out);
    return cudaGetLastError();
}

cudaError_t power_abs(GeomDev g, const c128* x, int nrhs, double* per_tri, double* partial, int npart,
                      cudaStream_t st) {
    (void)npart;
    dim3 grid((g.nt + 255) / 256, nrhs);
    k_pabs<<<grid, 256, 0, st>>>(g, x, per_tri, partial);
    return cudaGetLastError();
}

// scattered power: one CTA per direction (theta_i, phi_j); grid.y = right-hand side
__global__ void k_psca(GeomDev g, const c128* __restrict__ x, double* __restrict__ partial, int nphi,
                       const double* __restrict__ ct, const double* __restrict__ wt) {
    __shared__ double sh[32];
    int dir = blockIdx.x;
    int r = blockIdx.y;
    int it = dir / nphi, ip = dir % nphi;
    double cth = ct[it], sth = sqrt(fmax(0.0, 1.0 - cth * cth));
    double phi = 2.0 * BEM_PI * ip / nphi;
    d3 rh = D3(sth * cos(phi), sth * sin(phi), cth);
    const c128* xr = x + (int64_t)r * 2 * g.ne;
    c128 N[3], L[3];
    for (int d = 0; d < 3; ++d) N[d] = L[d] = mk<double>(0, 0);
    for (int e = threadIdx.x; e < 7 * g.nt; e += blockDim.x) {
        int t = e / 7, q = e % 7;
        d3 v[3];
        for (int i = 0; i < 3; ++i) v[i] = ld3(g.tv + 9 * t + 3 * i);
        double A = g.area[t];
        double l0, l1, l2, w;
        rule7_d(q, l0, l1, l2, w);
        d3 rq = l0 * v[0] + l1 * v[1] + l2 * v[2];
        c128 J[3], M[3];
        for (int d = 0; d < 3; ++d) J[d] = M[d] = mk<double>(0, 0);
        for (int i = 0; i < 3; ++i) {
            d3 f = (g.tri_coef[3 * t + i] / (2.0 * A)) * (rq - v[i]);
            c128 xj = xr[g.tri_edge[3 * t + i]], xm = xr[g.ne + g.tri_edge[3 * t + i]];
            J[0] = J[0] + f.x * xj; J[1] = J[1] + f.y * xj; J[2] = J[2] + f.z * xj;
            M[0] = M[0] + f.x * xm; M[1] = M[1] + f.y * xm; M[2] = M[2] + f.z * xm;
        }
        double sn, cs;
        sincos(g.k0 * dot(rh, rq), &sn, &cs);
        c128 ph = (w * A) * mk<double>(cs, sn);
        for (int d = 0; d < 3; ++d) {
            N[d] = N[d] + ph * J[d];
            L[d] = L[d] + ph * M[d];
        }
    }
    double vals[12] = {N[0].re, N[0].im, N[1].re, N[1].im, N[2].re, N[2].im,
                       L[0].re, L[0].im, L[1].re, L[1].im, L[2].re, L[2].im};
    __shared__ double tot[12];
    for (int k = 0; k < 12; ++k) {
        double s = block_sum_d(vals[k], sh);
        if (threadIdx.x == 0) tot[k] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        c128 Nt[3] = {mk<double>(tot[0], tot[1]), mk<double>(tot[2], tot[3]), mk<double>(tot[4], tot[5])};
        c128 Lt[3] = {mk<double>(tot[6], tot[7]), mk<double>(tot[8], tot[9]), mk<double>(tot[10], tot[11])};
        c128 rn = rh.x * Nt[0] + rh.y * Nt[1] + rh.z * Nt[2];
        c128 Ntr[3] = {Nt[0] - rh.x * rn, Nt[1] - rh.y * rn, Nt[2] - rh.z * rn};
        c128 rxL[3] = {rh.y * Lt[2] - rh.z * Lt[1], rh.z * Lt[0] - rh.x * Lt[2], rh.x * Lt[1] - rh.y * Lt[0]};
        double e2 = 0.0;
        for (int d = 0; d < 3; ++d) e2 += cabs2(rxL[d] - Ntr[d]);
        e2 *= (g.k0 / (4.0 * BEM_PI)) * (g.k0 / (4.0 * BEM_PI));
        partial[(int64_t)r * gridDim.x + dir] = wt[it] * (2.0 * BEM_PI / nphi) * e2;
    }
}

cudaError_t power_sca(GeomDev g, const c128* x, int nrhs, double* partial, int ntheta, int nphi, const double* ct,
                      const double* wt, cudaStream_t st) {
    dim3 grid(ntheta * nphi, nrhs);
    k_psca<<<grid, 256, 0, st>>>(g, x, partial, nphi, ct, wt);
    return cudaGetLastError();
}

// Re(a_J^H b_J + b_M^H a_M) partial sums (grid.y = rhs)
__global__ void k_pext(const c128* __restrict__ a, const c128* __restrict__ b, int64_t ne,
                       double* __restrict__ partial) {
    __shared__ double sh[32];
    int r = blockIdx.y;
    const c128* ar = a + (int64_t)r * 2 * ne;
    const c128* br = b + (int64_t)r * 2 * ne;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ne; i += (int64_t)gridDim.x * blockDim.x) {
        c128 aj = ar[i], bj = br[i], am = ar[ne + i], bm = br[ne + i];
        s += aj.re * bj.re + aj.im * bj.im;  // Re(conj(aJ) bJ)
        s += bm.re * am.re + bm.im * am.im;  // Re(conj(bM) aM)
    }
    double t = block_sum_d(s, sh);
    if (threadIdx.x == 0) partial[(int64_t)r * gridDim.x + blockIdx.x] = t;
}

cudaError_t dot_real_parts(const c128* a, const c128* b, int64_t n, int nrhs, double* partial, int npart,
                           cudaStream_t st) {
    dim3 grid(npart, nrhs);
    k_pext<<<grid, 256, 0, st>>>(a, b, n, partial);
    return cudaGetLastError();
}

}  // namespace bem
