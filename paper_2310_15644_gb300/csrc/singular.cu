// Singular and near-singular triangle pairs, integrated in FP64 with singularity
// extraction.
//
// The single- and double-layer operators of Sec. II (Eqs. 1-3) have kernels that
// blow up as R -> 0; the double layer is a Cauchy principal value.  For a pair of
// triangles that share a vertex, or whose centroids are closer than twice the
// larger longest edge, the leading terms of the small-R expansion
//     G = 1/(4 pi R) - k^2 R/(8 pi) + G_s,
//     grad G = [-1/(4 pi R^3) - k^2/(8 pi R) + g_s] (r - r'),
// are integrated over the source triangle in closed form (line integrals of R^q
// along its edges plus the solid angle it subtends), and the smooth remainders
// G_s, g_s (Taylor series below |k| R = 1) by the 7-point rule.  The outer
// integral over the test triangle uses the 7-point rule.  Each pair yields the
// 3 x 3 local matrices of T^_k and K_k at k0 and k1, stored once and gathered by
// every operator entry that involves the pair.
#include "common.cuh"
#include "geom.cuh"

namespace bem {

__device__ __forceinline__ c128 expmjkr(c128 k, double R) {
    // e^{-j k R} = e^{Im(k) R} (cos(Re(k) R) - j sin(Re(k) R))
    double s, c;
    sincos(k.re * R, &s, &c);
    double a = exp(k.im * R);
    return mk<double>(a * c, -a * s);
}

// G_k - 1/(4 pi R) + k^2 R / (8 pi)
__device__ c128 smooth_G(c128 k, double R) {
    double x = sqrt(cabs2(k)) * R;
    if (x < 1.0) {
        c128 mjk = mk<double>(k.im, -k.re);  // -j k
        c128 z = R * mjk;
        c128 term = (1.0 / 6.0) * (z * z);
        c128 sum = mk<double>(1.0, 0.0) + term;
        for (int n = 4; n < 30; ++n) {
            term = (1.0 / n) * (term * z);
            sum = sum + term;
        }
        return (1.0 / (4.0 * BEM_PI)) * (mjk * sum);
    }
    c128 e = expmjkr(k, R) - mk<double>(1.0, 0.0);
    c128 k2 = k * k;
    return (1.0 / (4.0 * BEM_PI * R)) * e + (R / (8.0 * BEM_PI)) * k2;
}

// g_k + 1/(4 pi R^3) + k^2/(8 pi R), with grad G = g (r - r')
__device__ c128 smooth_g(c128 k, double R) {
    double x = sqrt(cabs2(k)) * R;
    c128 mjk = mk<double>(k.im, -k.re);
    if (x < 1.0) {
        c128 z = R * mjk;
        c128 base = mk<double>(1.0 / 6.0, 0.0);  // z^{n-3}/n! at n = 3
        c128 sum = 2.0 * base;
        for (int n = 4; n < 30; ++n) {
            base = (1.0 / n) * (base * z);
            sum = sum + (double)(n - 1) * base;
        }
        c128 mjk3 = mjk * mjk * mjk;
        return (1.0 / (4.0 * BEM_PI)) * (mjk3 * sum);
    }
    c128 e = expmjkr(k, R);
    c128 jkR = mk<double>(-k.im * R, k.re * R);
    c128 one_jkR = mk<double>(1.0, 0.0) + jkR;
    c128 kR = R * k;
    c128 num = mk<double>(1.0, 0.0) - one_jkR * e + 0.5 * (kR * kR);
    return (1.0 / (4.0 * BEM_PI * R * R * R)) * num;
}

struct Analytic {
    double S_m1, S_1;
    d3 V_m1, V_1, G_m3, G_1, rho;
};

// closed-form integrals over a flat triangle tv with unit normal n, for point r
__device__ Analytic triangle_integrals(d3 r, const d3* tv, d3 n, bool inplane) {
    Analytic o;
    double h = inplane ? 0.0 : dot(n, r - tv[0]);
    d3 rho = r - h * n;
    double ah = fabs(h);
    double s_m1 = 0.0, sum_t_i1 = 0.0, omega = 0.0;
    d3 v_m1 = D3(0, 0, 0), v_1 = D3(0, 0, 0), g_in = D3(0, 0, 0);
    for (int i = 0; i < 3; ++i) {
        d3 va = tv[i], vb = tv[(i + 1) % 3];
        d3 e = vb - va;
        d3 lhat = (1.0 / sqrt(dot(e, e))) * e;
        d3 mhat = cross(lhat, n);
        double lm = dot(va - rho, lhat);
        double lp = dot(vb - rho, lhat);
        double t = dot(va - rho, mhat);
        double r0sq = t * t + h * h;
        double rm = sqrt(lm * lm + r0sq), rp = sqrt(lp * lp + r0sq);
        double im1;
        if (lm >= 0.0)
            im1 = log((rp + lp) / (rm + lm));
        else if (lp <= 0.0)
            im1 = log((rm - lm) / (rp - lp));
        else
            im1 = log((rp + lp) * (rm - lm) / r0sq);
        double i1 = 0.5 * (lp * rp - lm * rm + r0sq * im1);
        double i3 = 0.25 * (lp * rp * rp * rp - lm * rm * rm * rm) + 0.75 * r0sq * i1;
        if (t != 0.0) s_m1 += t * im1;
        sum_t_i1 += t * i1;
        if (r0sq + ah * fmin(rp, rm) > 0.0)
            omega += atan(t * lp / (r0sq + ah * rp)) - atan(t * lm / (r0sq + ah * rm));
        v_m1 = v_m1 + i1 * mhat;
        v_1 = v_1 + (i3 / 3.0) * mhat;
        g_in = g_in - im1 * mhat;
    }
    s_m1 -= ah * omega;
    o.S_m1 = s_m1;
    o.S_1 = (h * h * s_m1 + sum_t_i1) / 3.0;
    o.V_m1 = v_m1;
    o.V_1 = v_1;
    double sg = (h > 0.0) ? 1.0 : ((h < 0.0) ? -1.0 : 0.0);
    o.G_m3 = g_in - (sg * omega) * n;
    o.G_1 = D3(0, 0, 0) - v_m1 + (h * s_m1) * n;
    o.rho = rho;
    return o;
}

// ---------------------------------------------------------------------------
// partner search: shared vertex, or centroid distance < 2 * max(longest edge)
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool is_singular(const GeomDev& g, int a, int b) {
    const int* va = g.tvid + 3 * a;
    const int* vb = g.tvid + 3 * b;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (va[i] == vb[j]) return true;
    double dx = __dsub_rn(g.cen[3 * a], g.cen[3 * b]);
    double dy = __dsub_rn(g.cen[3 * a + 1], g.cen[3 * b + 1]);
    double dz = __dsub_rn(g.cen[3 * a + 2], g.cen[3 * b + 2]);
    double d = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
    return d < 2.0 * fmax(g.diam[a], g.diam[b]);
}

// Visit the triangles of the 27 cells around triangle a's cell.
template <typename F>
__device__ __forceinline__ void for_each_neighbour(const SingGrid& G, int a, F f) {
    const int cid = G.tri_cell[a];
    const int cx0 = cid % G.nx, cy0 = (cid / G.nx) % G.ny, cz0 = cid / (G.nx * G.ny);
    for (int dz = -1; dz <= 1; ++dz) {
        const int cz = cz0 + dz;
        if (cz < 0 || cz >= G.nz) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            const int cy = cy0 + dy;
            if (cy < 0 || cy >= G.ny) continue;
            for (int dx = -1; dx <= 1; ++dx) {
                const int cx = cx0 + dx;
                if (cx < 0 || cx >= G.nx) continue;
                const int cell = (cz * G.ny + cy) * G.nx + cx;
                for (int k = G.cell_start[cell]; k < G.cell_start[cell + 1]; ++k) f(G.cell_tri[k]);
            }
        }
    }
}

__global__ void k_sing_count(GeomDev g, SingGrid G, int* counts) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= g.nt) return;
    int c = 0;
    for_each_neighbour(G, a, [&](int b) { c += is_singular(g, a, b); });
    counts[a] = c;
}

// partners of a, ascending (insertion sort of the short list)
__global__ void k_sing_fill(GeomDev g, SingGrid G, const int* ptr, int* partners) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= g.nt) return;
    const int o = ptr[a];
    int n = 0;
    for_each_neighbour(G, a, [&](int b) {
        if (is_singular(g, a, b)) {
            int k = n++;
            while (k > 0 && partners[o + k - 1] > b) {
                partners[o + k] = partners[o + k - 1];
                --k;
            }
            partners[o + k] = b;
        }
    });
}

cudaError_t singular_count(GeomDev g, SingGrid G, int* counts, cudaStream_t st) {
    k_sing_count<<<(g.nt + 127) / 128, 128, 0, st>>>(g, G, counts);
    return cudaGetLastError();
}
cudaError_t singular_fill(GeomDev g, SingGrid G, const int* ptr, int* partners, cudaStream_t st) {
    k_sing_fill<<<(g.nt + 127) / 128, 128, 0, st>>>(g, G, ptr, partners);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// local matrices of a singular pair: one warp per pair, lane = 8*kidx + p
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_sing_values(GeomDev g, int npairs, const int* __restrict__ pair_a,
                                                     c128* __restrict__ vals) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= npairs) return;
    int a = pair_a[warp];
    int b = g.sing_b[warp];
    int kidx = lane >> 3, p = lane & 7;
    bool act = (kidx < 2) && (p < 7);
    c128 k = (kidx == 0) ? mk<double>(g.k0, 0.0) : g.k1;

    d3 va[3], vb[3];
    for (int i = 0; i < 3; ++i) {
        va[i] = ld3(g.tv + 9 * a + 3 * i);
        vb[i] = ld3(g.tv + 9 * b + 3 * i);
    }
    double Aa = g.area[a], Ab = g.area[b];
    d3 nb = ld3(g.nrm + 3 * b);

    c128 Iff[3][3], Ik[3][3], I0 = mk<double>(0, 0);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Iff[i][j] = Ik[i][j] = mk<double>(0, 0);

    if (act) {
        double l0, l1, l2, wp;
        rule7_d(p, l0, l1, l2, wp);
        wp *= Aa;
        d3 r = l0 * va[0] + l1 * va[1] + l2 * va[2];
        Analytic an = triangle_integrals(r, vb, nb, a == b);
        z3 F[3];
        c128 Phi = mk<double>(0, 0), S0 = mk<double>(0, 0);
        z3 S1 = Z3(mk<double>(0, 0), mk<double>(0, 0), mk<double>(0, 0));
        for (int j = 0; j < 3; ++j) F[j] = S1;
        for (int q = 0; q < 7; ++q) {
            double m0, m1, m2, wq;
            rule7_d(q, m0, m1, m2, wq);
            wq *= Ab;
            d3 rq = m0 * vb[0] + m1 * vb[1] + m2 * vb[2];
            d3 d = r - rq;
            double R = sqrt(dot(d, d));
            c128 Gs = wq * smooth_G(k, R);
            c128 gs = wq * smooth_g(k, R);
            for (int j = 0; j < 3; ++j) F[j] = zadd(F[j], zscale(Gs, rq - vb[j]));
            Phi = Phi + Gs;
            S0 = S0 + gs;
            S1 = zadd(S1, zscale(gs, rq));
        }
        c128 k2 = k * k;
        c128 c1 = mk<double>(1.0 / (4.0 * BEM_PI), 0.0);
        c128 c2 = (-1.0 / (8.0 * BEM_PI)) * k2;
        for (int j = 0; j < 3; ++j) {
            d3 rv = an.rho - vb[j];
            F[j] = zadd(F[j], zscale(c1, an.V_m1 + an.S_m1 * rv));
            F[j] = zadd(F[j], zscale(c2, an.V_1 + an.S_1 * rv));
        }
        Phi = Phi + an.S_m1 * c1 + an.S_1 * c2;
        z3 gvec = zadd(zscale(c1, an.G_m3), zscale(c2, an.G_1));
        for (int j = 0; j < 3; ++j) {
            z3 inner = zsub(S1, zscale(S0, vb[j]));            // S1 - v_j S0
            z3 H = zadd(rzcross(r, inner), zrcross(S1, vb[j]));  // r x (S1 - v_j S0) + S1 x v_j
            H = zadd(H, zrcross(gvec, r - vb[j]));              // + gvec x (r - v_j)
            for (int i = 0; i < 3; ++i) {
                d3 u = r - va[i];
                Iff[i][j] = wp * zdot(u, F[j]);
                Ik[i][j] = wp * zdot(u, H);
            }
        }
        I0 = wp * Phi;
    }
    // sum over the 7 outer points of each wavenumber (8-lane groups)
    for (int o = 4; o > 0; o >>= 1) {
        I0.re += __shfl_xor_sync(0xffffffffu, I0.re, o);
        I0.im += __shfl_xor_sync(0xffffffffu, I0.im, o);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                Iff[i][j].re += __shfl_xor_sync(0xffffffffu, Iff[i][j].re, o);
                Iff[i][j].im += __shfl_xor_sync(0xffffffffu, Iff[i][j].im, o);
                Ik[i][j].re += __shfl_xor_sync(0xffffffffu, Ik[i][j].re, o);
                Ik[i][j].im += __shfl_xor_sync(0xffffffffu, Ik[i][j].im, o);
            }
    }
    if ((lane == 0 || lane == 8)) {
        c128 jk = mk<double>(-k.im, k.re);
        c128 j_over_k = cdiv(mk<double>(0.0, 1.0), k);
        double AA = Aa * Ab;
        c128* out = vals + (int64_t)warp * 36 + kidx * 18;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double cc = g.tri_coef[3 * a + i] * g.tri_coef[3 * b + j];
                c128 t = jk * ((1.0 / (4.0 * AA)) * Iff[i][j]) - j_over_k * ((1.0 / AA) * I0);
                out[3 * i + j] = cc * t;
                out[9 + 3 * i + j] = (cc / (4.0 * AA)) * Ik[i][j];
            }
    }
}

// ---------------------------------------------------------------------------
// k-derivatives of the singular-pair local matrices (gradient with respect to the
// interior permittivity).  The extraction splits G = 1/(4 pi R) - k^2 R/(8 pi) + G_s and
// g = -1/(4 pi R^3) - k^2/(8 pi R) + g_s; differentiating the same split,
//   dG/dk = -k R/(4 pi) + dG_s/dk,   dG_s/dk = -j e^{-jkR}/(4 pi) + k R/(4 pi),
//   dg/dk = -k/(4 pi R) + dg_s/dk,   dg_s/dk = -k (e^{-jkR} - 1)/(4 pi R),
// so the analytic parts only keep their R (resp. grad R) integrals, with factor
// -k/(4 pi), and the smooth parts are integrated by the same 7 x 7 rule.  This is
// the exact derivative of the stored T^_k and K_k of the pair.
// ---------------------------------------------------------------------------
__device__ c128 smooth_dG(c128 k, double R) {
    c128 e = expmjkr(k, R);
    c128 mje = mk<double>(e.im, -e.re);  // -j e
    return (1.0 / (4.0 * BEM_PI)) * (mje + R * k);
}

__device__ c128 smooth_dg(c128 k, double R) {
    double x = sqrt(cabs2(k)) * R;
    const c128 mjk = mk<double>(k.im, -k.re);  // -j k
    c128 em1_R;                                // (e^{-jkR} - 1) / R
    if (x < 1.0) {
        // (e^z - 1) / R = -j k sum_{n>=1} z^{n-1} / n!, z = -j k R: finite at R = 0
        // (the coincident outer and inner points of a self pair)
        c128 z = R * mjk;
        c128 term = mk<double>(1.0, 0.0), sum = term;
        for (int n = 2; n < 30; ++n) {
            term = (1.0 / n) * (term * z);
            sum = sum + term;
        }
        em1_R = mjk * sum;
    } else {
        em1_R = (1.0 / R) * (expmjkr(k, R) - mk<double>(1.0, 0.0));
    }
    return (-1.0 / (4.0 * BEM_PI)) * (k * em1_R);
}

// dT^_1/dk and dK_1/dk (k = k1) of every singular pair: 18 complex per pair, the
// same [i][j] layout and coefficients as the values table.  One warp per pair,
// lanes 0..6 = outer points.
__global__ void __launch_bounds__(128) k_sing_dvalues(GeomDev g, int npairs, const int* __restrict__ pair_a,
                                                      c128* __restrict__ dvals) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= npairs) return;
    int a = pair_a[warp];
    int b = g.sing_b[warp];
    const int p = lane;
    const bool act = p < 7;
    const c128 k = g.k1;
    d3 va[3], vb[3];
    for (int i = 0; i < 3; ++i) {
        va[i] = ld3(g.tv + 9 * a + 3 * i);
        vb[i] = ld3(g.tv + 9 * b + 3 * i);
    }
    double Aa = g.area[a], Ab = g.area[b];
    d3 nb = ld3(g.nrm + 3 * b);
    const c128 z0 = mk<double>(0, 0);
    c128 Iff[3][3], dIff[3][3], dIk[3][3], I0 = z0, dI0 = z0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Iff[i][j] = dIff[i][j] = dIk[i][j] = z0;
    if (act) {
        double l0, l1, l2, wp;
        rule7_d(p, l0, l1, l2, wp);
        wp *= Aa;
        d3 r = l0 * va[0] + l1 * va[1] + l2 * va[2];
        Analytic an = triangle_integrals(r, vb, nb, a == b);
        z3 F[3], dF[3];
        z3 zz = Z3(z0, z0, z0);
        c128 Phi = z0, dPhi = z0, dS0 = z0;
        z3 dS1 = zz;
        for (int j = 0; j < 3; ++j) F[j] = dF[j] = zz;
        for (int q = 0; q < 7; ++q) {
            double m0, m1, m2, wq;
            rule7_d(q, m0, m1, m2, wq);
            wq *= Ab;
            d3 rq = m0 * vb[0] + m1 * vb[1] + m2 * vb[2];
            d3 d = r - rq;
            double R = sqrt(dot(d, d));
            c128 Gs = wq * smooth_G(k, R);
            c128 dGs = wq * smooth_dG(k, R);
            c128 dgs = wq * smooth_dg(k, R);
            for (int j = 0; j < 3; ++j) {
                F[j] = zadd(F[j], zscale(Gs, rq - vb[j]));
                dF[j] = zadd(dF[j], zscale(dGs, rq - vb[j]));
            }
            Phi = Phi + Gs;
            dPhi = dPhi + dGs;
            dS0 = dS0 + dgs;
            dS1 = zadd(dS1, zscale(dgs, rq));
        }
        const c128 c1 = mk<double>(1.0 / (4.0 * BEM_PI), 0.0);
        const c128 c2 = (-1.0 / (8.0 * BEM_PI)) * (k * k);
        const c128 dc2 = (-1.0 / (4.0 * BEM_PI)) * k;
        for (int j = 0; j < 3; ++j) {
            d3 rv = an.rho - vb[j];
            F[j] = zadd(F[j], zscale(c1, an.V_m1 + an.S_m1 * rv));
            F[j] = zadd(F[j], zscale(c2, an.V_1 + an.S_1 * rv));
            dF[j] = zadd(dF[j], zscale(dc2, an.V_1 + an.S_1 * rv));
        }
        Phi = Phi + an.S_m1 * c1 + an.S_1 * c2;
        dPhi = dPhi + an.S_1 * dc2;
        z3 dgvec = zscale(dc2, an.G_1);
        for (int j = 0; j < 3; ++j) {
            z3 inner = zsub(dS1, zscale(dS0, vb[j]));
            z3 H = zadd(rzcross(r, inner), zrcross(dS1, vb[j]));
            H = zadd(H, zrcross(dgvec, r - vb[j]));
            for (int i = 0; i < 3; ++i) {
                d3 u = r - va[i];
                Iff[i][j] = wp * zdot(u, F[j]);
                dIff[i][j] = wp * zdot(u, dF[j]);
                dIk[i][j] = wp * zdot(u, H);
            }
        }
        I0 = wp * Phi;
        dI0 = wp * dPhi;
    }
    for (int o = 4; o > 0; o >>= 1) {
        const unsigned m = 0xffffffffu;
        I0.re += __shfl_xor_sync(m, I0.re, o);
        I0.im += __shfl_xor_sync(m, I0.im, o);
        dI0.re += __shfl_xor_sync(m, dI0.re, o);
        dI0.im += __shfl_xor_sync(m, dI0.im, o);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                Iff[i][j].re += __shfl_xor_sync(m, Iff[i][j].re, o);
                Iff[i][j].im += __shfl_xor_sync(m, Iff[i][j].im, o);
                dIff[i][j].re += __shfl_xor_sync(m, dIff[i][j].re, o);
                dIff[i][j].im += __shfl_xor_sync(m, dIff[i][j].im, o);
                dIk[i][j].re += __shfl_xor_sync(m, dIk[i][j].re, o);
                dIk[i][j].im += __shfl_xor_sync(m, dIk[i][j].im, o);
            }
    }
    if (lane == 0) {
        // T^ = jk/(4AA') Iff - (j/k)/(AA') I0, so
        // dT^/dk = j/(4AA') Iff + jk/(4AA') dIff + j/(k^2 AA') I0 - (j/k)/(AA') dI0
        const c128 j1 = mk<double>(0.0, 1.0);
        const c128 jk = mk<double>(-k.im, k.re);
        const c128 j_over_k = cdiv(j1, k);
        const c128 j_over_k2 = cdiv(j1, k * k);
        const double AA = Aa * Ab;
        c128* out = dvals + (int64_t)warp * 18;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double cc = g.tri_coef[3 * a + i] * g.tri_coef[3 * b + j];
                c128 t = j1 * ((1.0 / (4.0 * AA)) * Iff[i][j]) + jk * ((1.0 / (4.0 * AA)) * dIff[i][j]) +
                         j_over_k2 * ((1.0 / AA) * I0) - j_over_k * ((1.0 / AA) * dI0);
                out[3 * i + j] = cc * t;
                out[9 + 3 * i + j] = (cc / (4.0 * AA)) * dIk[i][j];
            }
    }
}

cudaError_t singular_dvalues(GeomDev g, int npairs, const int* pair_a, c128* dvals, cudaStream_t st) {
    if (npairs <= 0) return cudaSuccess;
    const int warps_per_block = 4;
    const int blocks = (npairs + warps_per_block - 1) / warps_per_block;
    k_sing_dvalues<<<blocks, 32 * warps_per_block, 0, st>>>(g, npairs, pair_a, dvals);
    return cudaGetLastError();
}

cudaError_t singular_values(GeomDev g, int npairs, const int* pair_a, c128* vals, cudaStream_t st) {
    if (npairs <= 0) return cudaSuccess;
    int warps_per_block = 4;
    int blocks = (npairs + warps_per_block - 1) / warps_per_block;
    k_sing_values<<<blocks, 32 * warps_per_block, 0, st>>>(g, npairs, pair_a, vals);
    return cudaGetLastError();
}

}  // namespace bem
