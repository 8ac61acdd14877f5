// Bilinear forms of the interior operators for the gradient of the absorbed power
// with respect to the interior permittivity eps_r (the "dG/dk pass").
//
// The interior wavenumber k1 = k0 sqrt(eps_r mu_r) and impedance ratio
// eta_r = sqrt(mu_r / eps_r) enter the blocks A = T^0 + eta_r T^1, B = K0 + K1,
// C = T^0 + T^1 / eta_r; with lambda the adjoint solution, the gradient needs
// lambda^H (dZ/d eps_r) x, i.e. the six forms
//     lJ^H T^1 xJ,  lM^H T^1 xM,  lJ^H T^1' xJ,  lM^H T^1' xM,  lJ^H K1' xM,  lM^H K1' xJ
// (' = d/dk at k1).  They are summed over all triangle pairs, O(nt^2), in FP64:
// singular pairs from the FP64 tables (values, and their exact k-derivatives from
// k_sing_dvalues), all others by the 7 x 7-point rule differentiated under the sum
//     dG/dk = -j e^{-jkR}/(4 pi),   dg/dk = -k G,
// which is the exact derivative of the stored regular entries.  No operator data
// is used, so the forms are those of the uncompressed discretisation.
#include "common.cuh"
#include "geom.cuh"

namespace bem {

#define FORMS_THREADS 128

// local 3 x 3 matrices of T^_1, dT^_1/dk and dK_1/dk of a regular pair (a, b)
__device__ void regular_dk(const GeomDev& g, int a, int b, c128 T[3][3], c128 dT[3][3], c128 dK[3][3]) {
    const c128 k = g.k1;
    const c128 z0 = mk<double>(0, 0);
    d3 va[3], vb[3];
    const d3 oa = ld3(g.cen + 3 * a);
    for (int i = 0; i < 3; ++i) {
        va[i] = ld3(g.tv + 9 * a + 3 * i) - oa;
        vb[i] = ld3(g.tv + 9 * b + 3 * i) - oa;
    }
    const double Aa = g.area[a], Ab = g.area[b];
    c128 SGff[3][3], SGkff[3][3], SgK[3][3], SG = z0, SGk = z0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) SGff[i][j] = SGkff[i][j] = SgK[i][j] = z0;
    for (int p = 0; p < 7; ++p) {
        double l0, l1, l2, wpp;
        rule7_d(p, l0, l1, l2, wpp);
        const d3 pa = l0 * va[0] + l1 * va[1] + l2 * va[2];
        for (int q = 0; q < 7; ++q) {
            double m0, m1, m2, wq;
            rule7_d(q, m0, m1, m2, wq);
            const d3 pb = m0 * vb[0] + m1 * vb[1] + m2 * vb[2];
            const d3 d = pa - pb;
            const double R = sqrt(dot(d, d));
            const double W = wpp * Aa * wq * Ab / (4.0 * BEM_PI);
            double sn, cs;
            sincos(k.re * R, &sn, &cs);
            const double am = exp(k.im * R) * W;
            const c128 e = mk<double>(am * cs, -am * sn);  // W e^{-jkR}/(4 pi)
            const c128 G = (1.0 / R) * e;                   // W G
            const c128 Gk = mk<double>(e.im, -e.re);        // W dG/dk = -j W e^{-jkR}/(4 pi)
            const c128 gk = -1.0 * (k * G);                 // W dg/dk = -k W G
            SG = SG + G;
            SGk = SGk + Gk;
            for (int j = 0; j < 3; ++j) {
                const d3 wb = pb - vb[j];
                const d3 cr = cross(d, wb);
                for (int i = 0; i < 3; ++i) {
                    const d3 ua = pa - va[i];
                    const double ff = dot(ua, wb), kk = dot(ua, cr);
                    SGff[i][j] = SGff[i][j] + ff * G;
                    SGkff[i][j] = SGkff[i][j] + ff * Gk;
                    SgK[i][j] = SgK[i][j] + kk * gk;
                }
            }
        }
    }
    const c128 j1 = mk<double>(0.0, 1.0);
    const c128 jk = mk<double>(-k.im, k.re);
    const c128 j_over_k = cdiv(j1, k);
    const c128 j_over_k2 = cdiv(j1, k * k);
    const double AA = Aa * Ab;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            const double cc = g.tri_coef[3 * a + i] * g.tri_coef[3 * b + j];
            T[i][j] = cc * (jk * ((1.0 / (4.0 * AA)) * SGff[i][j]) - j_over_k * ((1.0 / AA) * SG));
            dT[i][j] = cc * (j1 * ((1.0 / (4.0 * AA)) * SGff[i][j]) + jk * ((1.0 / (4.0 * AA)) * SGkff[i][j]) +
                             j_over_k2 * ((1.0 / AA) * SG) - j_over_k * ((1.0 / AA) * SGk));
            dK[i][j] = (cc / (4.0 * AA)) * SgK[i][j];
        }
}

// One CTA per test triangle a, threads over source triangles b; per-a partial sums
// of the six forms at partial[f * nt + a].
__global__ void __launch_bounds__(FORMS_THREADS) k_interior_forms(GeomDev g, const c128* __restrict__ dvals,
                                                                  const c128* __restrict__ x,
                                                                  const c128* __restrict__ lam,
                                                                  c128* __restrict__ partial) {
    __shared__ double sh[FORMS_THREADS / 32][12];
    const int a = blockIdx.x;
    const int ne = g.ne;
    c128 lJ[3], lM[3];
    for (int i = 0; i < 3; ++i) {
        const int e = g.tri_edge[3 * a + i];
        lJ[i] = cconj(lam[e]);
        lM[i] = cconj(lam[ne + e]);
    }
    c128 acc[6];
    for (int f = 0; f < 6; ++f) acc[f] = mk<double>(0, 0);
    for (int b = threadIdx.x; b < g.nt; b += blockDim.x) {
        c128 xJ[3], xM[3];
        for (int j = 0; j < 3; ++j) {
            const int e = g.tri_edge[3 * b + j];
            xJ[j] = x[e];
            xM[j] = x[ne + e];
        }
        c128 T[3][3], dT[3][3], dK[3][3];
        const int slot = find_singular(g, a, b);
        if (slot >= 0) {
            const c128* v = g.sing_val + (int64_t)slot * 36;
            const c128* dv = dvals + (int64_t)slot * 18;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    T[i][j] = v[18 + 3 * i + j];
                    dT[i][j] = dv[3 * i + j];
                    dK[i][j] = dv[9 + 3 * i + j];
                }
        } else {
            regular_dk(g, a, b, T, dT, dK);
        }
        for (int i = 0; i < 3; ++i) {
            c128 tJ = mk<double>(0, 0), tM = tJ, dJ = tJ, dM = tJ, kJ = tJ, kM = tJ;
            for (int j = 0; j < 3; ++j) {
                tJ = tJ + T[i][j] * xJ[j];
                tM = tM + T[i][j] * xM[j];
                dJ = dJ + dT[i][j] * xJ[j];
                dM = dM + dT[i][j] * xM[j];
                kJ = kJ + dK[i][j] * xM[j];
                kM = kM + dK[i][j] * xJ[j];
            }
            acc[0] = acc[0] + lJ[i] * tJ;
            acc[1] = acc[1] + lM[i] * tM;
            acc[2] = acc[2] + lJ[i] * dJ;
            acc[3] = acc[3] + lM[i] * dM;
            acc[4] = acc[4] + lJ[i] * kJ;
            acc[5] = acc[5] + lM[i] * kM;
        }
    }
    // block sum in a fixed order
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int f = 0; f < 6; ++f)
        for (int o = 16; o > 0; o >>= 1) {
            acc[f].re += __shfl_xor_sync(0xffffffffu, acc[f].re, o);
            acc[f].im += __shfl_xor_sync(0xffffffffu, acc[f].im, o);
        }
    if (l == 0)
        for (int f = 0; f < 6; ++f) {
            sh[w][2 * f] = acc[f].re;
            sh[w][2 * f + 1] = acc[f].im;
        }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int f = threadIdx.x;
        c128 s = mk<double>(0, 0);
        for (int q = 0; q < FORMS_THREADS / 32; ++q) s = s + mk<double>(sh[q][2 * f], sh[q][2 * f + 1]);
        partial[(int64_t)f * gridDim.x + a] = s;
    }
}

cudaError_t interior_forms(GeomDev g, const c128* dvals, const c128* x, const c128* lam, c128* partial, c128* out,
                           cudaStream_t st) {
    if (g.nt <= 0) return cudaErrorInvalidValue;
    k_interior_forms<<<g.nt, FORMS_THREADS, 0, st>>>(g, dvals, x, lam, partial);
    BEM_CUDA_TRY(cudaGetLastError());
    return kv_reduce_partials(partial, g.nt, 6, out, st);
}

}  // namespace bem
