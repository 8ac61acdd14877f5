// Test harness: the host instantiation of the two-dimensional operator functions
// of the library (csrc/planar.cuh), exported for the CPU tests, which compare them
// with the oracle.  Built by tests/test_planar_host.py; no GPU needed.
#include "../../paper_2310_15644_gb300/csrc/planar.cuh"

using namespace bem2d;

extern "C" void h2_hankel01(double zr, double zi, double* out) {
    c128 h0, h1;
    hankel2_01(mk<double>(zr, zi), h0, h1);
    out[0] = h0.re;
    out[1] = h0.im;
    out[2] = h1.re;
    out[3] = h1.im;
}

extern "C" void h2_green_rem(double kr, double ki, double R, double* out) {
    c128 g = green_rem(mk<double>(kr, ki), R);
    out[0] = g.re;
    out[1] = g.im;
}

extern "C" void h2_dgreen_rem(double kr, double ki, double R, double* out) {
    c128 g = dgreen_rem(mk<double>(kr, ki), R);
    out[0] = g.re;
    out[1] = g.im;
}

// full matrices by the kernels' per-pair functions and summation order (host loop)
// Hankel's expansion in FP32 at z = zr + j zi (|z| >= 8), its phase e^{-j z} from FP64
extern "C" void h2_hankel01_asym_f(double zr, double zi, double* out) {
    const c128 eph = cexp2(mul_mj(mk<double>(zr, zi)));
    c64 h0, h1;
    hankel2_01_asym_f(mk<float>((float)zr, (float)zi), mk<float>((float)eph.re, (float)eph.im), h0, h1);
    out[0] = h0.re;
    out[1] = h0.im;
    out[2] = h1.re;
    out[3] = h1.im;
}

extern "C" void h2_operators(const double* verts, int n, double kr, double ki, int form, double* S, double* D,
                             double* N) {
    const c128 k = mk<double>(kr, ki);
    std::vector<double> P(2 * n), T(2 * n), Nn(2 * n), L(n);
    for (int e = 0; e < n; ++e) {
        const int f = (e + 1) % n;
        const double dx = verts[2 * f] - verts[2 * e], dy = verts[2 * f + 1] - verts[2 * e + 1];
        L[e] = std::sqrt(dx * dx + dy * dy);
        P[2 * e] = verts[2 * e];
        P[2 * e + 1] = verts[2 * e + 1];
        T[2 * e] = dx / L[e];
        T[2 * e + 1] = dy / L[e];
        Nn[2 * e] = T[2 * e + 1];
        Nn[2 * e + 1] = -T[2 * e];
    }
    std::vector<c128> locS((size_t)n * n * 4), locD((size_t)n * n * 4);
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
            c128 s[2][2], d[2][2];
            const int rel = a == b ? 0 : (b == (a + 1) % n ? 1 : (b == (a + n - 1) % n ? 2 : 3));
            local_matrices(&P[2 * a], &T[2 * a], L[a], &P[2 * b], &T[2 * b], &Nn[2 * b], L[b], rel, k, form, s, d);
            for (int p = 0; p < 2; ++p)
                for (int q = 0; q < 2; ++q) {
                    locS[((size_t)a * n + b) * 4 + 2 * p + q] = s[p][q];
                    locD[((size_t)a * n + b) * 4 + 2 * p + q] = d[p][q];
                }
        }
    const c128 k2 = k * k;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            c128 s = mk<double>(0, 0), d = s, nn = s;
            for (int p = 0; p < 2; ++p) {
                const int a = (i - p + n) % n;
                for (int q = 0; q < 2; ++q) {
                    const int b = (j - q + n) % n;
                    const size_t base = ((size_t)a * n + b) * 4;
                    const c128 v = locS[base + 2 * p + q];
                    s = s + v;
                    d = d + locD[base + 2 * p + q];
                    const c128 tot = (locS[base] + locS[base + 1]) + (locS[base + 2] + locS[base + 3]);
                    const double sg = (p == q ? 1.0 : -1.0) / (L[a] * L[b]);
                    const double nab = Nn[2 * a] * Nn[2 * b] + Nn[2 * a + 1] * Nn[2 * b + 1];
                    nn = nn + sg * tot - nab * (k2 * v);
                }
            }
            const size_t o = 2 * ((size_t)i * n + j);
            S[o] = s.re;
            S[o + 1] = s.im;
            D[o] = d.re;
            D[o + 1] = d.im;
            N[o] = nn.re;
            N[o + 1] = nn.im;
        }
}
