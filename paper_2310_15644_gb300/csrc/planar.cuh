// Two-dimensional (z-invariant) Galerkin operators of the paper's own setting:
// the single-layer, double-layer and hypersingular operators of Eqs. 1-4 with the
// kernel G_k(R) = -(j/4) H0^(2)(k R) (Eq. 5), tested and expanded with hat
// functions on a closed polygon (Sec. III, Eq. 8).  Host-and-device functions in
// FP64: the Hankel functions of orders 0 and 1, the kernels' static parts
// integrated over a straight segment in closed form, and the 2 x 2 local
// matrices of one segment pair.
#pragma once

#include "common.cuh"

namespace bem2d {

#define P2_HD __host__ __device__ __forceinline__

constexpr double P2_PI = 3.14159265358979323846;
constexpr double P2_TWO_PI = 6.28318530717958647692;
constexpr double P2_EULER = 0.57721566490153286061;
constexpr double P2_SERIES_X = 1.0;     // |k R| below which the kernel remainders use power series
constexpr double P2_HANKEL_SWITCH = 12.0;  // |z| from which the Hankel asymptotic expansion is used

P2_HD c128 cexp2(c128 z) {
    const double e = exp(z.re);
    return mk<double>(e * cos(z.im), e * sin(z.im));
}
P2_HD c128 clog2(c128 z) { return mk<double>(log(hypot(z.re, z.im)), atan2(z.im, z.re)); }
P2_HD c128 csqrt2(c128 z) {
    const double r = hypot(z.re, z.im);
    const double a = sqrt(fmax(0.0, 0.5 * (r + z.re)));
    const double b = copysign(sqrt(fmax(0.0, 0.5 * (r - z.re))), z.im);
    return mk<double>(a, b);
}
P2_HD double cabs2d(c128 z) { return hypot(z.re, z.im); }
P2_HD c128 mul_j(c128 z) { return mk<double>(-z.im, z.re); }       // j z
P2_HD c128 mul_mj(c128 z) { return mk<double>(z.im, -z.re); }      // -j z

// Gauss-Legendre rules on [0, 1]: node i and weight of the 10- and 20-point rules
P2_HD void gl10(int i, double& x, double& w) {
    switch (i) {
        case 0: x = 0.013046735741414128; w = 0.033335672154344069; break;
        case 1: x = 0.067468316655507732; w = 0.074725674575290196; break;
        case 2: x = 0.16029521585048778; w = 0.10954318125799101; break;
        case 3: x = 0.28330230293537639; w = 0.13463335965499826; break;
        case 4: x = 0.42556283050918442; w = 0.14776211235737641; break;
        case 5: x = 0.57443716949081558; w = 0.14776211235737641; break;
        case 6: x = 0.71669769706462361; w = 0.13463335965499826; break;
        case 7: x = 0.83970478414951222; w = 0.10954318125799101; break;
        case 8: x = 0.93253168334449232; w = 0.074725674575290196; break;
        default: x = 0.98695326425858587; w = 0.033335672154344069; break;
    }
}
P2_HD void gl20(int i, double& x, double& w) {
    switch (i) {
        case 0: x = 0.0034357004074525022; w = 0.0088070035695754466; break;
        case 1: x = 0.018014036361043095; w = 0.020300714900193223; break;
        case 2: x = 0.043882785874337027; w = 0.031336024167054395; break;
        case 3: x = 0.080441514088890609; w = 0.041638370788352357; break;
        case 4: x = 0.1268340467699246; w = 0.050965059908620353; break;
        case 5: x = 0.18197315963674249; w = 0.059097265980759303; break;
        case 6: x = 0.24456649902458644; w = 0.065844319224588443; break;
        case 7: x = 0.31314695564229023; w = 0.071048054659191201; break;
        case 8: x = 0.38610707442917747; w = 0.07458649323630212; break;
        case 9: x = 0.46173673943325133; w = 0.076376693565363141; break;
        case 10: x = 0.53826326056674867; w = 0.076376693565363141; break;
        case 11: x = 0.61389292557082253; w = 0.07458649323630212; break;
        case 12: x = 0.68685304435770977; w = 0.071048054659191201; break;
        case 13: x = 0.75543350097541362; w = 0.065844319224588443; break;
        case 14: x = 0.81802684036325757; w = 0.059097265980759303; break;
        case 15: x = 0.8731659532300754; w = 0.050965059908620353; break;
        case 16: x = 0.91955848591110945; w = 0.041638370788352357; break;
        case 17: x = 0.95611721412566297; w = 0.031336024167054395; break;
        case 18: x = 0.98198596363895696; w = 0.020300714900193223; break;
        default: x = 0.99656429959254744; w = 0.0088070035695754466; break;
    }
}

// H0^(2)(z) and H1^(2)(z) for z != 0 with Im z <= 0 (complex wavenumbers of lossy
// media, and the complexified k~ of the Calderon form).
//   |z| < 12: ascending series of J0, J1, Y0, Y1 (Abramowitz and Stegun 9.1.10,
//     9.1.11, 9.1.13), H^(2) = J - j Y;
//   |z| >= 12: Hankel's expansion H_nu^(2)(z) ~ sqrt(2/(pi z)) e^{-j(z - nu pi/2 - pi/4)}
//     sum_k (-j)^k a_k(nu) / z^k, a_k(nu) = prod_{i<=k} (4 nu^2 - (2i-1)^2) / (k! 8^k)
//     (A&S 9.2.8), summed while the terms decrease (relative error about e^{-2|z|}).
P2_HD void hankel2_01(c128 z, c128& h0, c128& h1) {
    const double az = cabs2d(z);
    if (az < P2_HANKEL_SWITCH) {
        const c128 h = 0.5 * z;
        const c128 q = h * h;
        const c128 mq = mk<double>(-q.re, -q.im);
        const c128 lnh = clog2(h) + mk<double>(P2_EULER, 0.0);
        c128 t = mk<double>(1.0, 0.0), J0 = t, S0 = mk<double>(0.0, 0.0);
        c128 u = t, sU = t, sH = mk<double>(1.0, 0.0);   // H_0 + H_1 = 1 for m = 0
        double Hm = 0.0;
        // unrolled, so the divisions by the index are constants; the terms fall
        // monotonically once m > |z| / 2, and below 1e-18 they no longer move the
        // O(1) sums
#pragma unroll
        for (int m = 1; m < 48; ++m) {
            t = (1.0 / ((double)m * m)) * (t * mq);
            u = (1.0 / ((double)m * (m + 1))) * (u * mq);
            const double Hm1 = Hm + 1.0 / m;                 // H_m
            const double Hm2 = Hm1 + 1.0 / (m + 1);          // H_{m+1}
            J0 = J0 + t;
            S0 = S0 - Hm1 * t;
            sU = sU + u;
            sH = sH + (Hm1 + Hm2) * u;
            Hm = Hm1;
            if (2 * m > (int)az + 2 && cabs2(t) + cabs2(u) < 1e-36) break;
        }
        const c128 J1 = h * sU;
        const c128 Y0 = (2.0 / P2_PI) * (lnh * J0 + S0);
        const c128 Y1 = (2.0 / P2_PI) * (lnh * J1) - (2.0 / P2_PI) * cdiv(mk<double>(1.0, 0.0), z) -
                        (1.0 / P2_PI) * (h * sH);
        h0 = J0 + mul_mj(Y0);
        h1 = J1 + mul_mj(Y1);
        return;
    }
    const c128 zi = cdiv(mk<double>(1.0, 0.0), z);
    const c128 pref = csqrt2((2.0 / P2_PI) * zi);
    for (int nu = 0; nu < 2; ++nu) {
        const double mu = 4.0 * nu * nu;
        c128 term = mk<double>(1.0, 0.0), sum = term;
        double prev = 1.0;
        for (int kk = 1; kk < 40; ++kk) {
            const double c = (mu - (2.0 * kk - 1.0) * (2.0 * kk - 1.0)) / (8.0 * kk);
            term = c * mul_mj(term * zi);
            const double at = cabs2d(term);
            if (at >= prev || at < 1e-17) break;
            sum = sum + term;
            prev = at;
        }
        // e^{-j w}, w = z - nu pi/2 - pi/4
        const c128 w = z - mk<double>(0.5 * P2_PI * nu + 0.25 * P2_PI, 0.0);
        const c128 ph = cexp2(mul_mj(w));
        const c128 hv = pref * ph * sum;
        if (nu == 0)
            h0 = hv;
        else
            h1 = hv;
    }
}

// Gr_k(R) = G_k(R) + ln(R)/(2 pi), continuous at R = 0; power series for |k R| < 1
// (the logarithm cancels analytically), Hankel functions above.
P2_HD c128 green_rem(c128 k, double R) {
    const c128 x = R * k;
    if (cabs2d(x) < P2_SERIES_X) {
        const c128 q = 0.25 * (x * x);
        const c128 mq = mk<double>(-q.re, -q.im);
        c128 t = mk<double>(1.0, 0.0), J0 = t, S = mk<double>(0.0, 0.0);
        double Hm = 0.0;
#pragma unroll
        for (int m = 1; m < 24; ++m) {
            t = (1.0 / ((double)m * m)) * (t * mq);
            Hm += 1.0 / m;
            J0 = J0 + t;
            S = S - Hm * t;
            if (cabs2(t) < 1e-36) break;  // |x| < 1: the terms fall from the first
        }
        const double lnR = R > 0.0 ? log(R) : 0.0;
        const c128 lk = clog2(0.5 * k) + mk<double>(P2_EULER, 0.0);
        const c128 bracket = lk * J0 + lnR * (J0 - mk<double>(1.0, 0.0)) + S;
        return mul_mj(0.25 * J0) - (1.0 / P2_TWO_PI) * bracket;
    }
    c128 h0, h1;
    hankel2_01(x, h0, h1);
    return mul_mj(0.25 * h0) + mk<double>(log(R) / P2_TWO_PI, 0.0);
}

// Ar_k(R) = A_k(R) - 1/(2 pi R^2), d_n' G_k = A_k(R) ((r - r').n'), A_k = -(j k/(4R)) H1^(2)(k R); R > 0
P2_HD c128 dgreen_rem(c128 k, double R) {
    const c128 x = R * k;
    if (cabs2d(x) < P2_SERIES_X) {
        const c128 q = 0.25 * (x * x);
        const c128 mq = mk<double>(-q.re, -q.im);
        c128 t = mk<double>(1.0, 0.0), sT = t, sH = t;   // T_0 = 1, H_0 + H_1 = 1
        double Hm = 0.0;
#pragma unroll
        for (int m = 1; m < 24; ++m) {
            t = (1.0 / ((double)m * (m + 1))) * (t * mq);
            const double Hm1 = Hm + 1.0 / m, Hm2 = Hm1 + 1.0 / (m + 1);
            sT = sT + t;
            sH = sH + (Hm1 + Hm2) * t;
            Hm = Hm1;
            if (cabs2(t) < 1e-36) break;
        }
        const c128 k2 = k * k;
        const c128 lx = clog2(0.5 * x) + mk<double>(P2_EULER, 0.0);
        return mul_mj(0.125 * (k2 * sT)) - (1.0 / (4.0 * P2_PI)) * (k2 * (lx * sT)) +
               (1.0 / (8.0 * P2_PI)) * (k2 * sH);
    }
    c128 h0, h1;
    hankel2_01(x, h0, h1);
    return (1.0 / R) * mul_mj(0.25 * (k * h1)) - mk<double>(1.0 / (P2_TWO_PI * R * R), 0.0);
}

// Both remainders at one distance (R > 0), sharing one Hankel evaluation above the
// series range: gr = Gr_k(R), ar = Ar_k(R)
P2_HD void kernel_rems(c128 k, double R, c128& gr, c128& ar) {
    const c128 x = R * k;
    if (cabs2d(x) < P2_SERIES_X) {
        gr = green_rem(k, R);
        ar = dgreen_rem(k, R);
        return;
    }
    c128 h0, h1;
    hankel2_01(x, h0, h1);
    gr = mul_mj(0.25 * h0) + mk<double>(log(R) / P2_TWO_PI, 0.0);
    ar = (1.0 / R) * mul_mj(0.25 * (k * h1)) - mk<double>(1.0 / (P2_TWO_PI * R * R), 0.0);
}

// Closed forms over a straight source segment of length L for a target at local
// coordinates (u along the segment from its start, v along its outward normal):
//   log moments  m0 = int_0^L ln R dt,  m1 = int_0^L t ln R dt,
//   angle moments e0 = int_0^L v/R^2 dt, e1 = int_0^L t v/R^2 dt (0 on the segment's line).
P2_HD void log_moments(double u, double v, double L, double& m0, double& m1) {
    double F[2], G[2];
    const double s[2] = {L - u, -u};
    for (int i = 0; i < 2; ++i) {
        const double Q = s[i] * s[i] + v * v;
        const double lnr = Q > 0.0 ? 0.5 * log(Q) : 0.0;
        const double at = v != 0.0 ? v * atan(s[i] / v) : 0.0;
        F[i] = s[i] * lnr - s[i] + at;
        G[i] = 0.5 * Q * lnr - 0.25 * s[i] * s[i] + u * F[i];
    }
    m0 = F[0] - F[1];
    m1 = G[0] - G[1];
}

P2_HD void angle_moments(double u, double v, double L, double& e0, double& e1) {
    if (v == 0.0) {
        e0 = e1 = 0.0;
        return;
    }
    double A[2], B[2];
    const double s[2] = {L - u, -u};
    for (int i = 0; i < 2; ++i) {
        const double Q = s[i] * s[i] + v * v;
        A[i] = atan(s[i] / v);
        B[i] = 0.5 * v * (Q > 0.0 ? log(Q) : 0.0) + u * A[i];
    }
    e0 = A[0] - A[1];
    e1 = B[0] - B[1];
}

// Local 2 x 2 matrices S_ab[p][q] = int_a int_b phi_p G phi_q and
// D_ab[p][q] = int_a int_b phi_p d_n'G phi_q of test segment a = (pa, ta, La) and
// source segment b = (pb, tb, nb, Lb), phi_0 = 1 - t/L, phi_1 = t/L.
// mode 0: 10-point outer rule; 1 / 2: 20-point rule graded by u = s^2 toward the
// end / start of segment a (the vertex shared with b).  The static parts go in
// closed form over b, the remainders on the 10-point inner rule.
P2_HD void pair_local(const double pa[2], const double ta[2], double La, const double pb[2], const double tb[2],
                      const double nb[2], double Lb, int mode, c128 k, c128 S[2][2], c128 D[2][2]) {
    for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 2; ++q) S[p][q] = D[p][q] = mk<double>(0.0, 0.0);
    const int no = mode == 0 ? 10 : 20;
    for (int o = 0; o < no; ++o) {
        double ua, wa;
        if (mode == 0) {
            gl10(o, ua, wa);
        } else {
            double s, w;
            gl20(mode == 1 ? no - 1 - o : o, s, w);
            ua = s * s;
            wa = 2.0 * s * w;
            if (mode == 1) ua = 1.0 - ua;
        }
        const double r0 = pa[0] + ua * La * ta[0], r1 = pa[1] + ua * La * ta[1];
        const double d0 = r0 - pb[0], d1 = r1 - pb[1];
        const double u = d0 * tb[0] + d1 * tb[1];
        const double v = d0 * nb[0] + d1 * nb[1];
        double m0, m1, e0, e1;
        log_moments(u, v, Lb, m0, m1);
        angle_moments(u, v, Lb, e0, e1);
        c128 Sq[2], Dq[2];
        Sq[0] = mk<double>(-(m0 - m1 / Lb) / P2_TWO_PI, 0.0);
        Sq[1] = mk<double>(-(m1 / Lb) / P2_TWO_PI, 0.0);
        Dq[0] = mk<double>((e0 - e1 / Lb) / P2_TWO_PI, 0.0);
        Dq[1] = mk<double>((e1 / Lb) / P2_TWO_PI, 0.0);
        for (int i = 0; i < 10; ++i) {
            double xi, wi;
            gl10(i, xi, wi);
            const double q0 = pb[0] + xi * Lb * tb[0], q1 = pb[1] + xi * Lb * tb[1];
            const double dx = r0 - q0, dy = r1 - q1;
            const double R = sqrt(dx * dx + dy * dy);
            const double vv = dx * nb[0] + dy * nb[1];
            const double W = wi * Lb;
            c128 g0, a0;
            kernel_rems(k, R, g0, a0);
            const c128 gr = W * g0;
            const c128 ar = (W * vv) * a0;
            Sq[0] = Sq[0] + (1.0 - xi) * gr;
            Sq[1] = Sq[1] + xi * gr;
            Dq[0] = Dq[0] + (1.0 - xi) * ar;
            Dq[1] = Dq[1] + xi * ar;
        }
        const double Wo = wa * La;
        const double ph[2] = {1.0 - ua, ua};
        for (int p = 0; p < 2; ++p)
            for (int q = 0; q < 2; ++q) {
                S[p][q] = S[p][q] + (Wo * ph[p]) * Sq[q];
                D[p][q] = D[p][q] + (Wo * ph[p]) * Dq[q];
            }
    }
}

// ---------------------------------------------------------------------------
// Well-separated segment pairs: the kernel is smooth over both segments, so S and
// D are integrated directly on the 5 x 5 Gauss-Legendre product rule (no static
// split).  With the midpoints at least P2_FAR_FACTOR segment lengths apart, the
// nearest singularity of ln R lies about 11 half-lengths from either segment, and
// the 5-point rule's error is below (22)^-10 ~ 4e-14 of the integrand's size.
// ---------------------------------------------------------------------------
constexpr double P2_FAR_FACTOR = 6.0;
constexpr double P2_ASYM_F = 8.0;  // |k R| from which the FP32 form uses Hankel's expansion
#define P2_FORM_FP64 0             // every kernel evaluation in FP64
#define P2_FORM_FP32 1             // far pairs with |k R| >= P2_ASYM_F evaluated in FP32

// 5-point Gauss-Legendre rule on [0, 1] (nodes (1 + t)/2 of the roots t = 0,
// +-sqrt(5 -+ 2 sqrt(10/7)) / 3; weights 64/225, (322 +- 13 sqrt 70)/1800)
P2_HD void gl5(int i, double& x, double& w) {
    switch (i) {
        case 0: x = 0.046910077030668004; w = 0.11846344252809454; break;
        case 1: x = 0.23076534494715845; w = 0.23931433524968323; break;
        case 2: x = 0.5; w = 0.28444444444444444; break;
        case 3: x = 0.76923465505284155; w = 0.23931433524968323; break;
        default: x = 0.95308992296933200; w = 0.11846344252809454; break;
    }
}

P2_HD c64 csqrt_f(c64 z) {
    const float r = hypotf(z.re, z.im);
    const float a = sqrtf(fmaxf(0.0f, 0.5f * (r + z.re)));
    const float b = copysignf(sqrtf(fmaxf(0.0f, 0.5f * (r - z.re))), z.im);
    return mk<float>(a, b);
}

// Hankel's expansion (A&S 9.2.8) of H0^(2)(z), H1^(2)(z) in FP32 for |z| >= P2_ASYM_F,
// where its smallest term is below FP32 rounding.  The phase factor
// eph = e^{-j z} comes in from the caller, which forms it from an FP64 phase per
// pair times an FP32 phase of the small offset (so large k R loses no phase).
P2_HD void hankel2_01_asym_f(c64 z, c64 eph, c64& h0, c64& h1) {
    const c64 zi = cdiv(mk<float>(1.0f, 0.0f), z);
    const c64 pref = csqrt_f((float)(2.0 / P2_PI) * zi);
    const float c45 = 0.70710678118654752f;
    for (int nu = 0; nu < 2; ++nu) {
        const float mu = 4.0f * nu * nu;
        c64 term = mk<float>(1.0f, 0.0f), sum = term;
        float prev = 1.0f;
        for (int kk = 1; kk < 24; ++kk) {
            const float c = (mu - (2.0f * kk - 1.0f) * (2.0f * kk - 1.0f)) / (8.0f * kk);
            const c64 tz = term * zi;
            term = mk<float>(c * tz.im, -c * tz.re);  // c (-j) term / z
            const float at = hypotf(term.re, term.im);
            if (at >= prev || at < 3e-8f) break;
            sum = sum + term;
            prev = at;
        }
        // e^{-j (z - nu pi/2 - pi/4)} = e^{-j z} e^{j pi/4} j^nu
        const c64 rot = nu == 0 ? mk<float>(c45, c45) : mk<float>(-c45, c45);
        const c64 hv = pref * ((eph * rot) * sum);
        if (nu == 0)
            h0 = hv;
        else
            h1 = hv;
    }
}

// S_ab and D_ab of a well-separated pair (as pair_local) on the 5 x 5 rule.  form
// P2_FORM_FP32: offsets, distances and, where |k R| >= P2_ASYM_F, the Hankel
// functions in FP32; R = R0 + dR with R0 the midpoint distance (FP64) and dR from
// the small offsets, so the phase e^{-j k R} = e^{-j k R0} e^{-j k dR} stays exact
// to FP32 rounding of dR.
P2_HD void far_pair_local(const double pa[2], const double ta[2], double La, const double pb[2],
                          const double tb[2], const double nb[2], double Lb, c128 k, int form, c128 S[2][2],
                          c128 D[2][2]) {
    const double D0[2] = {(pa[0] + 0.5 * La * ta[0]) - (pb[0] + 0.5 * Lb * tb[0]),
                          (pa[1] + 0.5 * La * ta[1]) - (pb[1] + 0.5 * Lb * tb[1])};
    const double R0 = sqrt(D0[0] * D0[0] + D0[1] * D0[1]);
    for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 2; ++q) S[p][q] = D[p][q] = mk<double>(0.0, 0.0);
    if (form == P2_FORM_FP32) {
        const c128 e0d = cexp2(mul_mj(R0 * k));  // e^{-j k R0}
        const c64 e0 = mk<float>((float)e0d.re, (float)e0d.im);
        const c64 kf = mk<float>((float)k.re, (float)k.im);
        const float d0x = (float)D0[0], d0y = (float)D0[1], r0 = (float)R0;
        const float dnb = (float)(D0[0] * nb[0] + D0[1] * nb[1]);
        c64 Sf[2][2], Df[2][2];
        for (int p = 0; p < 2; ++p)
            for (int q = 0; q < 2; ++q) Sf[p][q] = Df[p][q] = mk<float>(0.0f, 0.0f);
        for (int i = 0; i < 5; ++i) {
            double xa, wa;
            gl5(i, xa, wa);
            const float oa = (float)((xa - 0.5) * La);
            for (int j = 0; j < 5; ++j) {
                double xb, wb;
                gl5(j, xb, wb);
                const float ob = (float)((xb - 0.5) * Lb);
                const float dx = oa * (float)ta[0] - ob * (float)tb[0];
                const float dy = oa * (float)ta[1] - ob * (float)tb[1];
                const float cross = 2.0f * (d0x * dx + d0y * dy) + (dx * dx + dy * dy);
                const float R = sqrtf(r0 * r0 + cross);
                const float dR = cross / (R + r0);
                const c64 z = R * kf;
                c64 h0, h1;
                if (hypotf(z.re, z.im) >= (float)P2_ASYM_F) {
                    // e^{-j k dR} = e^{-j Re(k) dR} e^{Im(k) dR}
                    float sn, cs;
                    sincosf(kf.re * dR, &sn, &cs);
                    const float m = expf(kf.im * dR);
                    const c64 eph = e0 * mk<float>(m * cs, -m * sn);
                    hankel2_01_asym_f(z, eph, h0, h1);
                } else {
                    c128 g0, g1;
                    hankel2_01((double)R * k, g0, g1);
                    h0 = mk<float>((float)g0.re, (float)g0.im);
                    h1 = mk<float>((float)g1.re, (float)g1.im);
                }
                const float vv = dnb + (dx * (float)nb[0] + dy * (float)nb[1]);
                const float W = (float)(wa * wb * La * Lb);
                const c64 G = mk<float>(0.25f * h0.im, -0.25f * h0.re);           // -(j/4) H0
                const c64 kh = kf * h1;
                const c64 A = mk<float>(0.25f * kh.im / R, -0.25f * kh.re / R);   // -(j k / (4R)) H1
                const float ph[2] = {(float)(1.0 - xa), (float)xa}, qh[2] = {(float)(1.0 - xb), (float)xb};
                for (int p = 0; p < 2; ++p)
                    for (int q = 0; q < 2; ++q) {
                        const float f = W * ph[p] * qh[q];
                        Sf[p][q] = Sf[p][q] + f * G;
                        Df[p][q] = Df[p][q] + (f * vv) * A;
                    }
            }
        }
        for (int p = 0; p < 2; ++p)
            for (int q = 0; q < 2; ++q) {
                S[p][q] = mk<double>(Sf[p][q].re, Sf[p][q].im);
                D[p][q] = mk<double>(Df[p][q].re, Df[p][q].im);
            }
        return;
    }
    for (int i = 0; i < 5; ++i) {
        double xa, wa;
        gl5(i, xa, wa);
        const double r0 = pa[0] + xa * La * ta[0], r1 = pa[1] + xa * La * ta[1];
        for (int j = 0; j < 5; ++j) {
            double xb, wb;
            gl5(j, xb, wb);
            const double dx = r0 - (pb[0] + xb * Lb * tb[0]), dy = r1 - (pb[1] + xb * Lb * tb[1]);
            const double R = sqrt(dx * dx + dy * dy);
            c128 h0, h1;
            hankel2_01(R * k, h0, h1);
            const double vv = dx * nb[0] + dy * nb[1];
            const double W = wa * wb * La * Lb;
            const c128 G = mul_mj(0.25 * h0);
            const c128 A = (1.0 / R) * mul_mj(0.25 * (k * h1));
            const double ph[2] = {1.0 - xa, xa}, qh[2] = {1.0 - xb, xb};
            for (int p = 0; p < 2; ++p)
                for (int q = 0; q < 2; ++q) {
                    const double f = W * ph[p] * qh[q];
                    S[p][q] = S[p][q] + f * G;
                    D[p][q] = D[p][q] + (f * vv) * A;
                }
        }
    }
}

// S of a segment of length L with itself: the logarithm over both copies in closed
// form (L^2 (ln L / 4 + K_pq), K = [[-7/16, -5/16], [-5/16, -7/16]] on the unit
// square) and the remainder on the 10 x 10 product rule (D vanishes there).
P2_HD void self_local(double L, c128 k, c128 S[2][2]) {
    const double K[2][2] = {{-7.0 / 16.0, -5.0 / 16.0}, {-5.0 / 16.0, -7.0 / 16.0}};
    for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 2; ++q) S[p][q] = mk<double>(-(L * L) * (0.25 * log(L) + K[p][q]) / P2_TWO_PI, 0.0);
    for (int i = 0; i < 10; ++i) {
        double xi, wi;
        gl10(i, xi, wi);
        for (int j = 0; j < 10; ++j) {
            double xj, wj;
            gl10(j, xj, wj);
            const c128 g = (wi * wj * L * L) * green_rem(k, fabs(xi - xj) * L);
            const double pi_[2] = {1.0 - xi, xi}, pj[2] = {1.0 - xj, xj};
            for (int p = 0; p < 2; ++p)
                for (int q = 0; q < 2; ++q) S[p][q] = S[p][q] + (pi_[p] * pj[q]) * g;
        }
    }
}

// Local matrices of the segment pair (a, b) as the operator kernels compute them.
// rel 0: the same segment; 1: b follows a; 2: b precedes a; 3: any other pair, on
// the 5 x 5 rule when well separated, else as pair_local.
P2_HD void local_matrices(const double pa[2], const double ta[2], double La, const double pb[2],
                          const double tb[2], const double nb[2], double Lb, int rel, c128 k, int form,
                          c128 S[2][2], c128 D[2][2]) {
    if (rel == 0) {
        self_local(La, k, S);
        for (int p = 0; p < 2; ++p)
            for (int q = 0; q < 2; ++q) D[p][q] = mk<double>(0.0, 0.0);
        return;
    }
    if (rel == 3) {
        const double mx = (pa[0] + 0.5 * La * ta[0]) - (pb[0] + 0.5 * Lb * tb[0]);
        const double my = (pa[1] + 0.5 * La * ta[1]) - (pb[1] + 0.5 * Lb * tb[1]);
        const double lim = P2_FAR_FACTOR * fmax(La, Lb);
        if (mx * mx + my * my >= lim * lim) {
            far_pair_local(pa, ta, La, pb, tb, nb, Lb, k, form, S, D);
            return;
        }
    }
    pair_local(pa, ta, La, pb, tb, nb, Lb, rel == 3 ? 0 : rel, k, S, D);
}

}  // namespace bem2d
