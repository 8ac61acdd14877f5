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

// Scattered power, in two kernels.  k_psca_points writes, once per call, every
// quadrature point r_q (7 per triangle) and the weighted currents w_q A_t J(r_q),
// w_q A_t M(r_q) of each right-hand side (6 complex values).  k_psca_dirs then takes
// one direction (theta_i, phi_j) per CTA and PSCA_RB right-hand sides per grid.y,
// forms each point's phase e^{j k0 rhat.r_q} once for all of them, and accumulates
// N and L; the far-field magnitude follows in thread 0.  FP64 throughout.
constexpr int PSCA_T = 256;
constexpr int PSCA_RB = 4;

__global__ void __launch_bounds__(PSCA_T) k_psca_points(GeomDev g, const c128* __restrict__ x, int r0, int nr,
                                                        double* __restrict__ pts, c128* __restrict__ cur) {
    const int64_t Q = 7 * (int64_t)g.nt;
    const int64_t q = (int64_t)blockIdx.x * PSCA_T + threadIdx.x;
    const int rr = blockIdx.y;
    if (q >= Q || rr >= nr) return;
    const int t = (int)(q / 7), iq = (int)(q % 7);
    d3 v[3];
    for (int i = 0; i < 3; ++i) v[i] = ld3(g.tv + 9 * t + 3 * i);
    const double A = g.area[t];
    double l0, l1, l2, w;
    rule7_d(iq, l0, l1, l2, w);
    const d3 rq = l0 * v[0] + l1 * v[1] + l2 * v[2];
    if (rr == 0) {
        pts[q] = rq.x;
        pts[Q + q] = rq.y;
        pts[2 * Q + q] = rq.z;
    }
    const c128* xr = x + (int64_t)(r0 + rr) * 2 * g.ne;
    c128 J[3], M[3];
    for (int d = 0; d < 3; ++d) J[d] = M[d] = mk<double>(0, 0);
    for (int i = 0; i < 3; ++i) {
        d3 f = (g.tri_coef[3 * t + i] / (2.0 * A)) * (rq - v[i]);
        c128 xj = xr[g.tri_edge[3 * t + i]], xm = xr[g.ne + g.tri_edge[3 * t + i]];
        J[0] = J[0] + f.x * xj; J[1] = J[1] + f.y * xj; J[2] = J[2] + f.z * xj;
        M[0] = M[0] + f.x * xm; M[1] = M[1] + f.y * xm; M[2] = M[2] + f.z * xm;
    }
    const double wA = w * A;
    c128* cr = cur + (int64_t)rr * 6 * Q;
    for (int d = 0; d < 3; ++d) {
        cr[d * Q + q] = wA * J[d];
        cr[(3 + d) * Q + q] = wA * M[d];
    }
}

__global__ void __launch_bounds__(PSCA_T) k_psca_dirs(const double* __restrict__ pts, const c128* __restrict__ cur,
                                                      int64_t Q, double k0, int nr, int r0, int nphi,
                                                      const double* __restrict__ ct, const double* __restrict__ wt,
                                                      double* __restrict__ partial) {
    __shared__ double sh[PSCA_T / 32][12 * PSCA_RB];
    const int dir = blockIdx.x;
    const int rb = blockIdx.y * PSCA_RB;
    const int nb = min(PSCA_RB, nr - rb);
    const int it = dir / nphi, ip = dir % nphi;
    const double cth = ct[it], sth = sqrt(fmax(0.0, 1.0 - cth * cth));
    const double phi = 2.0 * BEM_PI * ip / nphi;
    const d3 rh = D3(sth * cos(phi), sth * sin(phi), cth);
    double acc[PSCA_RB][12];
#pragma unroll
    for (int u = 0; u < PSCA_RB; ++u)
#pragma unroll
        for (int c = 0; c < 12; ++c) acc[u][c] = 0.0;
    for (int64_t q = threadIdx.x; q < Q; q += PSCA_T) {
        double sn, cs;
        sincos(k0 * (rh.x * pts[q] + rh.y * pts[Q + q] + rh.z * pts[2 * Q + q]), &sn, &cs);
#pragma unroll
        for (int u = 0; u < PSCA_RB; ++u) {
            if (u >= nb) break;
            const c128* cr = cur + (int64_t)(rb + u) * 6 * Q + q;
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const c128 v = cr[(int64_t)c * Q];
                acc[u][2 * c] += cs * v.re - sn * v.im;
                acc[u][2 * c + 1] += cs * v.im + sn * v.re;
            }
        }
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int u = 0; u < PSCA_RB; ++u)
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            double v = acc[u][c];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (l == 0) sh[w][12 * u + c] = v;
        }
    __syncthreads();
    if (threadIdx.x >= nb) return;
    const int u = threadIdx.x;
    double tot[12];
    for (int c = 0; c < 12; ++c) {
        double s = 0.0;
        for (int k = 0; k < PSCA_T / 32; ++k) s += sh[k][12 * u + c];
        tot[c] = s;
    }
    const c128 Nt[3] = {mk<double>(tot[0], tot[1]), mk<double>(tot[2], tot[3]), mk<double>(tot[4], tot[5])};
    const c128 Lt[3] = {mk<double>(tot[6], tot[7]), mk<double>(tot[8], tot[9]), mk<double>(tot[10], tot[11])};
    const c128 rn = rh.x * Nt[0] + rh.y * Nt[1] + rh.z * Nt[2];
    const c128 Ntr[3] = {Nt[0] - rh.x * rn, Nt[1] - rh.y * rn, Nt[2] - rh.z * rn};
    const c128 rxL[3] = {rh.y * Lt[2] - rh.z * Lt[1], rh.z * Lt[0] - rh.x * Lt[2], rh.x * Lt[1] - rh.y * Lt[0]};
    double e2 = 0.0;
    for (int d = 0; d < 3; ++d) e2 += cabs2(rxL[d] - Ntr[d]);
    e2 *= (k0 / (4.0 * BEM_PI)) * (k0 / (4.0 * BEM_PI));
    partial[(int64_t)(r0 + rb + u) * gridDim.x + dir] = wt[it] * (2.0 * BEM_PI / nphi) * e2;
}

size_t power_sca_scratch(GeomDev g, int nrhs) {
    const int64_t Q = 7 * (int64_t)g.nt;
    const int chunk = std::min(nrhs, PSCA_CHUNK);
    return sizeof(double) * 3 * Q + sizeof(c128) * 6 * Q * chunk;
}

cudaError_t power_sca(GeomDev g, const c128* x, int nrhs, double* partial, int ntheta, int nphi, const double* ct,
                      const double* wt, void* scratch, cudaStream_t st) {
    const int64_t Q = 7 * (int64_t)g.nt;
    double* pts = (double*)scratch;
    c128* cur = (c128*)(pts + 3 * Q);
    for (int r0 = 0; r0 < nrhs; r0 += PSCA_CHUNK) {
        const int nr = std::min(PSCA_CHUNK, nrhs - r0);
        k_psca_points<<<dim3((unsigned)((Q + PSCA_T - 1) / PSCA_T), nr), PSCA_T, 0, st>>>(g, x, r0, nr, pts, cur);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_psca_dirs<<<dim3(ntheta * nphi, (nr + PSCA_RB - 1) / PSCA_RB), PSCA_T, 0, st>>>(
            pts, cur, Q, g.k0, nr, r0, nphi, ct, wt, partial);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
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
