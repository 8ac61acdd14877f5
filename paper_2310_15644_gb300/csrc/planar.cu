// The paper's own two-dimensional operators on the GPU (see planar.cuh): the dense
// Galerkin matrices S, D, D* = D^T and N of Eqs. 1-4 for a closed polygon, in FP64
// (or with the well-separated pairs' Hankel functions in FP32).
// One thread per segment pair computes its 2 x 2 local matrices; a second kernel
// sums the four segment pairs that meet at each vertex pair in a fixed order (no
// atomics, reproducible), applying the Maue identity for N:
//   N_ab[p][q] = s_p s_q / (La Lb) sum_{p'q'} S_ab[p'][q'] - k^2 (n_a . n_b) S_ab[p][q],
//   s = (-1, +1) (derivatives of the two hat functions along the curve).
#include "common.cuh"
#include <cstdio>

#include "planar.cuh"

using namespace bem2d;

namespace {

struct Seg {
    double p[2], t[2], n[2], L;
};

__global__ void k_planar_local(const Seg* __restrict__ seg, int n, c128 k, int form, c128* __restrict__ locS,
                               c128* __restrict__ locD) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * n) return;
    const int a = (int)(idx / n), b = (int)(idx % n);
    c128 S[2][2], D[2][2];
    const int rel = a == b ? 0 : (b == (a + 1) % n ? 1 : (b == (a + n - 1) % n ? 2 : 3));
    local_matrices(seg[a].p, seg[a].t, seg[a].L, seg[b].p, seg[b].t, seg[b].n, seg[b].L, rel, k, form, S, D);
    for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 2; ++q) {
            locS[idx * 4 + 2 * p + q] = S[p][q];
            locD[idx * 4 + 2 * p + q] = D[p][q];
        }
}

// entry (i, j): segment pairs (a, b) = (i - p, j - q), p, q in {0, 1}; row-major outputs
__global__ void k_planar_assemble(const Seg* __restrict__ seg, int n, c128 k, const c128* __restrict__ locS,
                                  const c128* __restrict__ locD, c128* __restrict__ S, c128* __restrict__ D,
                                  c128* __restrict__ N) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * n) return;
    const int i = (int)(idx / n), j = (int)(idx % n);
    const c128 k2 = k * k;
    c128 s = mk<double>(0.0, 0.0), d = s, nn = s;
    for (int p = 0; p < 2; ++p) {
        const int a = (i - p + n) % n;
        for (int q = 0; q < 2; ++q) {
            const int b = (j - q + n) % n;
            const int64_t base = ((int64_t)a * n + b) * 4;
            const c128 v = locS[base + 2 * p + q];
            s = s + v;
            d = d + locD[base + 2 * p + q];
            const c128 tot = (locS[base] + locS[base + 1]) + (locS[base + 2] + locS[base + 3]);
            const double sg = (p == q ? 1.0 : -1.0) / (seg[a].L * seg[b].L);
            const double nab = seg[a].n[0] * seg[b].n[0] + seg[a].n[1] * seg[b].n[1];
            nn = nn + sg * tot - nab * (k2 * v);
        }
    }
    if (S) S[idx] = s;
    if (D) D[idx] = d;
    if (N) N[idx] = nn;
}

// Row 0 only (circulant operators of a regular polygon): the local matrices of the
// segment pairs (a, b) with a in {0, n - 1} (ai = 0, 1) and every b, then row 0.
__global__ void k_planar_local_row0(const Seg* __restrict__ seg, int n, c128 k, int form, c128* __restrict__ locS,
                                    c128* __restrict__ locD) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 2 * n) return;
    const int ai = idx / n, b = idx % n;
    const int a = ai == 0 ? 0 : n - 1;
    c128 S[2][2], D[2][2];
    const int rel = a == b ? 0 : (b == (a + 1) % n ? 1 : (b == (a + n - 1) % n ? 2 : 3));
    local_matrices(seg[a].p, seg[a].t, seg[a].L, seg[b].p, seg[b].t, seg[b].n, seg[b].L, rel, k, form, S, D);
    for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 2; ++q) {
            locS[(int64_t)idx * 4 + 2 * p + q] = S[p][q];
            locD[(int64_t)idx * 4 + 2 * p + q] = D[p][q];
        }
}

__global__ void k_planar_row0(const Seg* __restrict__ seg, int n, c128 k, const c128* __restrict__ locS,
                              const c128* __restrict__ locD, c128* __restrict__ S, c128* __restrict__ D,
                              c128* __restrict__ N) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const c128 k2 = k * k;
    c128 s = mk<double>(0.0, 0.0), d = s, nn = s;
    for (int p = 0; p < 2; ++p) {
        const int a = p == 0 ? 0 : n - 1;  // (0 - p) mod n, stored as ai = p
        for (int q = 0; q < 2; ++q) {
            const int b = (j - q + n) % n;
            const int64_t base = ((int64_t)p * n + b) * 4;
            const c128 v = locS[base + 2 * p + q];
            s = s + v;
            d = d + locD[base + 2 * p + q];
            const c128 tot = (locS[base] + locS[base + 1]) + (locS[base + 2] + locS[base + 3]);
            const double sg = (p == q ? 1.0 : -1.0) / (seg[a].L * seg[b].L);
            const double nab = seg[a].n[0] * seg[b].n[0] + seg[a].n[1] * seg[b].n[1];
            nn = nn + sg * tot - nab * (k2 * v);
        }
    }
    if (S) S[j] = s;
    if (D) D[j] = d;
    if (N) N[j] = nn;
}

}  // namespace

void bem_ctx_set_error(bem_ctx* c, const char* msg);

static bem_status planar_operators_impl(bem_ctx* ctx, const double* verts, int n, bem_c128 k, int fp32, void* S,
                                        void* D, void* N, void* stream, bool row0);

// row 0 of S, D, N (device complex128 vectors of n, each may be NULL) with the same
// quadrature as bem_planar_operators: the whole operators when they are circulant
bem_status planar_operators_row0(bem_ctx* ctx, const double* verts, int n, bem_c128 k, int fp32, void* S, void* D,
                                 void* N, void* stream);

extern "C" bem_status bem_planar_operators(bem_ctx* ctx, const double* verts, int n, bem_c128 k, int fp32, void* S,
                                           void* D, void* N, void* stream) {
    return planar_operators_impl(ctx, verts, n, k, fp32, S, D, N, stream, false);
}

bem_status planar_operators_row0(bem_ctx* ctx, const double* verts, int n, bem_c128 k, int fp32, void* S, void* D,
                                 void* N, void* stream) {
    return planar_operators_impl(ctx, verts, n, k, fp32, S, D, N, stream, true);
}

static bem_status planar_operators_impl(bem_ctx* ctx, const double* verts, int n, bem_c128 k, int fp32, void* S,
                                        void* D, void* N, void* stream, bool row0) {
    auto fail = [&](bem_status s, const char* msg) {
        if (ctx) bem_ctx_set_error(ctx, msg);
        return s;
    };
    if (!verts || n < 3)
        return fail(BEM_EINVAL, "bem_planar_operators: a closed polygon needs at least 3 vertices");
    if (n > 46340) return fail(BEM_EINVAL, "bem_planar_operators: more than 46340 vertices");
    if (!(k.re > 0.0) || k.im > 0.0 || !std::isfinite(k.re) || !std::isfinite(k.im))
        return fail(BEM_EINVAL, "bem_planar_operators: need Re k > 0 and Im k <= 0 (e^{+jwt})");
    if (fp32 != 0 && fp32 != 1) return fail(BEM_EINVAL, "bem_planar_operators: fp32 must be 0 or 1");
    std::vector<Seg> seg(n);
    double area2 = 0.0;
    for (int e = 0; e < n; ++e) {
        const int f = (e + 1) % n;
        const double dx = verts[2 * f] - verts[2 * e], dy = verts[2 * f + 1] - verts[2 * e + 1];
        const double L = std::sqrt(dx * dx + dy * dy);
        if (!(L > 0.0) || !std::isfinite(L))
            return fail(BEM_EINVAL, "bem_planar_operators: zero-length segment");
        Seg& s = seg[e];
        s.p[0] = verts[2 * e];
        s.p[1] = verts[2 * e + 1];
        s.t[0] = dx / L;
        s.t[1] = dy / L;
        s.n[0] = s.t[1];
        s.n[1] = -s.t[0];
        s.L = L;
        area2 += verts[2 * e] * verts[2 * f + 1] - verts[2 * f] * verts[2 * e + 1];
    }
    if (!(area2 > 0.0)) return fail(BEM_EINVAL, "bem_planar_operators: vertices must run counter-clockwise");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nn = row0 ? 2 * (int64_t)n : (int64_t)n * n;  // segment pairs computed
    Seg* d_seg = nullptr;
    c128 *locS = nullptr, *locD = nullptr;
    {
        // the two per-pair scratch arrays (64 n^2 bytes each) are the binding limit: refuse up front
        size_t fr = 0, tot = 0;
        const size_t need = 2 * sizeof(c128) * 4 * (size_t)nn + sizeof(Seg) * (size_t)n;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && need > fr) {
            char buf[200];
            snprintf(buf, sizeof buf, "bem_planar_operators: n = %d needs %zu bytes of scratch, %zu bytes free", n,
                     need, fr);
            return fail(BEM_ENOMEM, buf);
        }
    }
    cudaError_t e = cudaMalloc(&d_seg, sizeof(Seg) * n);
    if (e == cudaSuccess) e = cudaMalloc(&locS, sizeof(c128) * 4 * nn);
    if (e == cudaSuccess) e = cudaMalloc(&locD, sizeof(c128) * 4 * nn);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_seg, seg.data(), sizeof(Seg) * n, cudaMemcpyHostToDevice, st);
    const unsigned blocks = (unsigned)((nn + 127) / 128);
    const c128 kk = mk<double>(k.re, k.im);
    const int form = fp32 ? P2_FORM_FP32 : P2_FORM_FP64;
    if (e == cudaSuccess) {
        if (row0)
            k_planar_local_row0<<<blocks, 128, 0, st>>>(d_seg, n, kk, form, locS, locD);
        else
            k_planar_local<<<blocks, 128, 0, st>>>(d_seg, n, kk, form, locS, locD);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        if (row0)
            k_planar_row0<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(d_seg, n, kk, locS, locD, (c128*)S, (c128*)D,
                                                                        (c128*)N);
        else
            k_planar_assemble<<<blocks, 128, 0, st>>>(d_seg, n, kk, locS, locD, (c128*)S, (c128*)D, (c128*)N);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_seg);
    cudaFree(locS);
    cudaFree(locD);
    if (e != cudaSuccess)
        return fail(e == cudaErrorMemoryAllocation ? BEM_ENOMEM : BEM_ECUDA, cudaGetErrorString(e));
    return BEM_OK;
}
