// Calderon preconditioner of the PMCHWT operator: the 3-D counterpart of the
// Calderon-preconditioned CFIE of Sec. III, where the single layer is composed with
// the hypersingular operator through the inverse Gram matrix so that the product is
// the identity plus a compact operator.
//
// The PMCHWT operator Z is composed with itself.  The second factor is discretised
// with Buffa-Christiansen (BC) functions on the barycentric refinement of the mesh,
// div-conforming functions close to n x RWG that pair with the RWG functions through
// a well-conditioned mixed Gram matrix G[m, e] = int (n x f_m) . g_e dS.  The
// preconditioner is
//
//     P = -Gb^-T Cb^T Z_fine Cb Gb^-1,   Gb = diag(G, G), Cb = diag(C, C),
//
// with C the BC functions written in the RWG basis of the refined mesh and Z_fine
// the PMCHWT operator of that mesh (assembled and compressed like Z itself).  The
// solver applies it on the right: Z P y = b, x = P y.
//
// This file holds the host construction (refinement, C, G, the Chebyshev plan for
// G^-1) and the device kernels (sparse products, Chebyshev steps).
//
// Constructions (FP64 on the host):
//   * refinement: coarse triangle t with corners (v0, v1, v2) gives fine triangles
//     6t + 2i = (v_i, m(v_i, v_i+1), g_t) and 6t + 2i + 1 = (v_i, g_t, m(v_i-1, v_i));
//     fine vertices are the coarse vertices, then the edge midpoints (edge order),
//     then the centroids (triangle order), so fine triangle f lies in the dual cell
//     of its first vertex and in coarse triangle f / 6.
//   * BC function of coarse edge e, traversed a -> b by its T+: flux l_e / 2 from
//     the cell of a into the cell of b through each fine edge (m_e, g_T+-), charge
//     l_e / N on each of the N fine triangles of the two cells (source at a, sink
//     at b), and the radial fluxes of least norm, which in closed form are
//     -+ l_e (1/2 - i / N) counter-clockwise across the i-th radial fine edge of
//     the cell counted around the vertex from (v, m_e) (0 on that edge).
//   * G by the three-point edge-midpoint rule on every fine triangle, exact for
//     the quadratic integrand (n x f_m) . phi_k.
//   * G^-1 by a fixed number of Chebyshev steps on D^-1 G (D = diag G), whose
//     eigenvalues are real to a few 1e-3 and lie in a fixed interval under
//     refinement: the interval comes from power iterations, the step count from a
//     host run on a pseudo-random vector (to the caller's target).  A fixed polynomial keeps the
//     preconditioner linear, so GMRES sees one fixed operator.
#include "common.cuh"

#include <cstdio>
#include <utility>

namespace bem {
namespace cald {

void refine(const MeshTables& c, std::vector<double>& fv, std::vector<int>& ft) {
    const int64_t nv = c.nv, ne = c.ne, nt = c.nt;
    fv.assign((size_t)3 * (nv + ne + nt), 0.0);
    std::copy(c.verts, c.verts + 3 * nv, fv.begin());
    for (int64_t e = 0; e < ne; ++e)
        for (int d = 0; d < 3; ++d)
            fv[3 * (nv + e) + d] = (c.verts[3 * c.edge_v[2 * e] + d] + c.verts[3 * c.edge_v[2 * e + 1] + d]) * 0.5;
    for (int64_t t = 0; t < nt; ++t)
        for (int d = 0; d < 3; ++d) {
            const double s = (c.verts[3 * c.tris[3 * t] + d] + c.verts[3 * c.tris[3 * t + 1] + d]) +
                             c.verts[3 * c.tris[3 * t + 2] + d];
            fv[3 * (nv + ne + t) + d] = s / 3.0;
        }
    ft.resize((size_t)18 * nt);
    for (int64_t t = 0; t < nt; ++t) {
        const int g = (int)(nv + ne + t);
        for (int i = 0; i < 3; ++i) {
            const int v = c.tris[3 * t + i];
            const int m_next = (int)nv + c.tri_edge[3 * t + (i + 2) % 3];  // edge (v_i, v_i+1)
            const int m_prev = (int)nv + c.tri_edge[3 * t + (i + 1) % 3];  // edge (v_i-1, v_i)
            int* f = &ft[18 * t + 6 * i];
            f[0] = v, f[1] = m_next, f[2] = g;
            f[3] = v, f[4] = g, f[5] = m_prev;
        }
    }
}

namespace {

// fine edge joining vertices a and b (edges are numbered in lexicographic order)
int find_edge(const MeshTables& f, int a, int b) {
    const int lo = std::min(a, b), hi = std::max(a, b);
    int64_t l = 0, h = f.ne;
    while (l < h) {
        const int64_t mid = (l + h) / 2;
        const int x = f.edge_v[2 * mid], y = f.edge_v[2 * mid + 1];
        if (x < lo || (x == lo && y < hi))
            l = mid + 1;
        else
            h = mid;
    }
    return (l < f.ne && f.edge_v[2 * l] == lo && f.edge_v[2 * l + 1] == hi) ? (int)l : -1;
}

int corner_of(const MeshTables& m, int t, int v) {
    for (int j = 0; j < 3; ++j)
        if (m.tris[3 * t + j] == v) return j;
    return -1;
}

double edge_len(const MeshTables& m, int e) {
    return std::fabs(m.tri_coef[3 * m.edge_tri[2 * e] + m.edge_loc[2 * e]]);
}

struct Trip {
    int r, c;
    double v;
};

Csr from_triplets(std::vector<Trip>& t, int64_t rows, int64_t cols) {
    std::sort(t.begin(), t.end(), [](const Trip& a, const Trip& b) { return a.r != b.r ? a.r < b.r : a.c < b.c; });
    Csr m;
    m.rows = rows;
    m.cols = cols;
    m.ptr.assign(rows + 1, 0);
    for (size_t i = 0; i < t.size();) {
        size_t j = i;
        double s = 0;
        while (j < t.size() && t[j].r == t[i].r && t[j].c == t[i].c) s += t[j++].v;
        m.col.push_back(t[i].c);
        m.val.push_back(s);
        m.ptr[t[i].r + 1]++;
        i = j;
    }
    for (int64_t r = 0; r < rows; ++r) m.ptr[r + 1] += m.ptr[r];
    return m;
}

}  // namespace

bool bc_matrix(const MeshTables& c, const MeshTables& f, Csr& C, std::string& err) {
    const int nv = (int)c.nv, ne = (int)c.ne;
    std::vector<Trip> trip;
    trip.reserve((size_t)30 * ne);
    auto other_tri = [&](int E, int T) { return c.edge_tri[2 * E] == T ? c.edge_tri[2 * E + 1] : c.edge_tri[2 * E]; };
    char buf[160];
    for (int e = 0; e < ne; ++e) {
        const int tp = c.edge_tri[2 * e], tm = c.edge_tri[2 * e + 1], ip = c.edge_loc[2 * e];
        const int a = c.tris[3 * tp + (ip + 1) % 3], b = c.tris[3 * tp + (ip + 2) % 3];  // T+ runs a -> b
        const double le = edge_len(c, e);
        const int m = nv + e;
        // the two cell-boundary fine edges at the midpoint: l_e / 2 each, from the cell of a to that of b
        for (int T : {tp, tm}) {
            const int k = find_edge(f, m, nv + ne + T);
            if (k < 0) {
                snprintf(buf, sizeof buf, "refinement: no fine edge (midpoint of %d, centroid of %d)", e, T);
                err = buf;
                return false;
            }
            const int fp = f.edge_tri[2 * k];
            const int cell = f.tris[3 * fp];
            if (cell != a && cell != b) {
                err = "refinement: fine edge at a midpoint outside the two cells";
                return false;
            }
            trip.push_back({k, e, (cell == a ? 0.5 : -0.5) * le / edge_len(f, k)});
        }
        // radial fluxes of the two cells (source a: -, sink b: +, counter-clockwise)
        const int ends[2] = {a, b};
        const int start[2] = {tp, tm};  // the triangle in which v is followed by the other end
        for (int side = 0; side < 2; ++side) {
            const int v = ends[side];
            const double sigma = side == 0 ? -1.0 : 1.0;
            std::vector<int> rad, ccw;
            int T = start[side];
            int j = corner_of(c, T, v);
            if (j < 0 || c.tri_edge[3 * T + (j + 2) % 3] != e) {
                err = "refinement: inconsistent orientation around a vertex";
                return false;
            }
            for (int guard = 0;; ++guard) {
                if (guard > 2 * c.nt) {
                    err = "refinement: the triangles around a vertex do not close";
                    return false;
                }
                rad.push_back(find_edge(f, v, nv + c.tri_edge[3 * T + (j + 2) % 3]));  // (v, m_next)
                ccw.push_back(6 * T + 2 * j);
                rad.push_back(find_edge(f, v, nv + ne + T));  // (v, g_T)
                ccw.push_back(6 * T + 2 * j + 1);
                const int Eprev = c.tri_edge[3 * T + (j + 1) % 3];  // (v_prev, v): shared with the next triangle
                T = other_tri(Eprev, T);
                j = corner_of(c, T, v);
                if (j < 0) {
                    err = "refinement: broken fan around a vertex";
                    return false;
                }
                if (c.tri_edge[3 * T + (j + 2) % 3] == e) break;  // back at (v, m_e)
            }
            const int N = (int)rad.size();
            for (int i = 1; i < N; ++i) {
                const int k = rad[i];
                if (k < 0 || (f.edge_tri[2 * k] != ccw[i] && f.edge_tri[2 * k + 1] != ccw[i])) {
                    err = "refinement: radial fine edge not found";
                    return false;
                }
                const double flux = sigma * le * (0.5 - (double)i / N);
                const double s = f.edge_tri[2 * k + 1] == ccw[i] ? 1.0 : -1.0;  // T- on the counter-clockwise side
                trip.push_back({k, e, s * flux / edge_len(f, k)});
            }
        }
    }
    C = from_triplets(trip, f.ne, c.ne);
    return true;
}

Csr transpose(const Csr& a) {
    std::vector<Trip> t;
    t.reserve(a.val.size());
    for (int64_t r = 0; r < a.rows; ++r)
        for (int p = a.ptr[r]; p < a.ptr[r + 1]; ++p) t.push_back({a.col[p], (int)r, a.val[p]});
    return from_triplets(t, a.cols, a.rows);
}

void mixed_gram(const MeshTables& c, const MeshTables& f, const Csr& C, Csr& G) {
    std::vector<Trip> trip;
    trip.reserve((size_t)f.nt * 9 * 8);
    for (int64_t tau = 0; tau < f.nt; ++tau) {
        const int64_t T = tau / 6;
        const double* n = c.nrm + 3 * T;
        const double* P[3];
        for (int q = 0; q < 3; ++q) P[q] = f.verts + 3 * f.tris[3 * tau + q];
        double M[3][3];  // edge midpoints of the fine triangle
        for (int q = 0; q < 3; ++q)
            for (int d = 0; d < 3; ++d) M[q][d] = 0.5 * (P[(q + 1) % 3][d] + P[(q + 2) % 3][d]);
        for (int s = 0; s < 3; ++s) {
            const int m = c.tri_edge[3 * T + s];
            const double cm = c.tri_coef[3 * T + s] / (2.0 * c.area[T]);
            const double* p = c.verts + 3 * c.tris[3 * T + s];
            double rot[3][3];  // n x f_m at the three midpoints
            for (int q = 0; q < 3; ++q) {
                const double fm[3] = {cm * (M[q][0] - p[0]), cm * (M[q][1] - p[1]), cm * (M[q][2] - p[2])};
                rot[q][0] = n[1] * fm[2] - n[2] * fm[1];
                rot[q][1] = n[2] * fm[0] - n[0] * fm[2];
                rot[q][2] = n[0] * fm[1] - n[1] * fm[0];
            }
            for (int r = 0; r < 3; ++r) {
                const int k = f.tri_edge[3 * tau + r];
                const double ck = f.tri_coef[3 * tau + r] / (2.0 * f.area[tau]);
                const double* pk = P[r];
                double I = 0;
                for (int q = 0; q < 3; ++q)
                    I += rot[q][0] * ck * (M[q][0] - pk[0]) + rot[q][1] * ck * (M[q][1] - pk[1]) +
                         rot[q][2] * ck * (M[q][2] - pk[2]);
                I *= f.area[tau] / 3.0;
                for (int pp = C.ptr[k]; pp < C.ptr[k + 1]; ++pp) trip.push_back({m, C.col[pp], I * C.val[pp]});
            }
        }
    }
    G = from_triplets(trip, c.ne, c.ne);
}

namespace {

void spmv_host(const Csr& a, const std::vector<double>& dinv, const std::vector<double>& x, std::vector<double>& y) {
    for (int64_t r = 0; r < a.rows; ++r) {
        double s = 0;
        for (int p = a.ptr[r]; p < a.ptr[r + 1]; ++p) s += a.val[p] * x[a.col[p]];
        y[r] = dinv[r] * s;
    }
}

double norm2(const std::vector<double>& x) {
    double s = 0;
    for (double v : x) s += v * v;
    return std::sqrt(s);
}

// deterministic pseudo-random vector in [-1, 1) (64-bit linear congruential generator)
std::vector<double> lcg_vector(int64_t n, uint64_t seed) {
    std::vector<double> x(n);
    uint64_t s = seed;
    for (int64_t i = 0; i < n; ++i) {
        s = s * 6364136223846793005ULL + 1442695040888963407ULL;
        x[i] = (double)(s >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    }
    return x;
}

void make_coefficients(ChebPlan& p, int steps) {
    const double theta = 0.5 * (p.lmax + p.lmin), delta = 0.5 * (p.lmax - p.lmin), sigma = theta / delta;
    p.theta = theta;
    p.steps = steps;
    p.c1.assign(std::max(steps - 1, 0), 0.0);
    p.c2.assign(std::max(steps - 1, 0), 0.0);
    double rho = 1.0 / sigma;
    for (int k = 0; k + 1 < steps; ++k) {
        const double rn = 1.0 / (2.0 * sigma - rho);
        p.c1[k] = rn * rho;
        p.c2[k] = 2.0 * rn / delta;
        rho = rn;
    }
}

// relative residual |D^-1 (b - G x)| / |D^-1 b| after each of up to max_steps updates
std::vector<double> chebyshev_host(const Csr& G, const std::vector<double>& dinv, const ChebPlan& p,
                                   const std::vector<double>& b) {
    const int64_t n = G.rows;
    std::vector<double> r(n), x(n), d(n), ad(n), out;
    for (int64_t i = 0; i < n; ++i) r[i] = dinv[i] * b[i];
    const double r0 = norm2(r);
    for (int64_t i = 0; i < n; ++i) {
        d[i] = r[i] / p.theta;
        x[i] = d[i];
    }
    for (int k = 0;; ++k) {
        spmv_host(G, dinv, d, ad);
        for (int64_t i = 0; i < n; ++i) r[i] -= ad[i];
        out.push_back(norm2(r) / r0);  // residual of x after k + 1 updates
        if (k + 1 >= p.steps) break;
        for (int64_t i = 0; i < n; ++i) {
            d[i] = p.c1[k] * d[i] + p.c2[k] * r[i];
            x[i] += d[i];
        }
    }
    return out;
}

}  // namespace

bool chebyshev_plan(const Csr& G, double target, int max_steps, ChebPlan& plan, std::string& err) {
    const int64_t n = G.rows;
    std::vector<double> dinv(n, 0.0);
    for (int64_t r = 0; r < n; ++r) {
        for (int p = G.ptr[r]; p < G.ptr[r + 1]; ++p)
            if (G.col[p] == r) dinv[r] = 1.0 / G.val[p];
        if (!(dinv[r] > 0) || !std::isfinite(dinv[r])) {
            err = "mixed Gram matrix: non-positive diagonal entry";
            return false;
        }
    }
    // largest eigenvalue of D^-1 G: power iteration
    std::vector<double> x = lcg_vector(n, 12345), y(n);
    double hi = 0;
    for (int it = 0; it < 100; ++it) {
        spmv_host(G, dinv, x, y);
        hi = norm2(y) / norm2(x);
        const double s = 1.0 / norm2(y);
        for (int64_t i = 0; i < n; ++i) x[i] = y[i] * s;
    }
    hi *= 1.05;
    // smallest: power iteration on hi I - D^-1 G
    x = lcg_vector(n, 777);
    double mu = 0;
    for (int it = 0; it < 200; ++it) {
        spmv_host(G, dinv, x, y);
        for (int64_t i = 0; i < n; ++i) y[i] = hi * x[i] - y[i];
        mu = norm2(y) / norm2(x);
        const double s = 1.0 / norm2(y);
        for (int64_t i = 0; i < n; ++i) x[i] = y[i] * s;
    }
    double lo = hi - mu;
    if (!(lo > 0)) {
        err = "mixed Gram matrix: D^-1 G is not definite (Chebyshev interval reaches 0)";
        return false;
    }
    lo *= 0.85;
    const std::vector<double> b = lcg_vector(n, 4242);
    for (int attempt = 0; attempt < 5; ++attempt, lo *= 0.7) {
        plan.lmin = lo;
        plan.lmax = hi;
        make_coefficients(plan, max_steps);
        const std::vector<double> res = chebyshev_host(G, dinv, plan, b);
        for (int k = 0; k < (int)res.size(); ++k)
            if (res[k] <= target) {
                make_coefficients(plan, k + 1);
                plan.reduction = res[k];
                return true;
            }
    }
    err = "mixed Gram matrix: the Chebyshev iteration does not reach its tolerance";
    return false;
}

// ---------------------------------------------------------------------------
// device: sparse products and Chebyshev steps on nblk blocks.  A thread takes one
// row for BCH consecutive blocks (grid.y = blocks / BCH), so each matrix row is
// read once per BCH blocks; the blocks' vectors are gathered from L2.
// ---------------------------------------------------------------------------
namespace {

constexpr int CT = 256;

template <typename R, int BCH>
__global__ void __launch_bounds__(CT) k_csr_apply(const int* __restrict__ ptr, const int* __restrict__ col,
                                                 const R* __restrict__ val, int64_t rows,
                                                 const cx<R>* __restrict__ x, int64_t xs, cx<R>* __restrict__ y,
                                                 int64_t ys, int nblk, R scale) {
    const int64_t r = (int64_t)blockIdx.x * CT + threadIdx.x;
    if (r >= rows) return;
    const int b0 = blockIdx.y * BCH;
    const int nb = min(BCH, nblk - b0);
    cx<R> s[BCH];
#pragma unroll
    for (int u = 0; u < BCH; ++u) s[u] = mk<R>(0, 0);
    for (int p = ptr[r]; p < ptr[r + 1]; ++p) {
        const R a = val[p];
        const cx<R>* xc = x + (int64_t)b0 * xs + col[p];
#pragma unroll
        for (int u = 0; u < BCH; ++u)
            if (u < nb) {
                const cx<R> v = xc[(int64_t)u * xs];
                s[u].re += a * v.re;
                s[u].im += a * v.im;
            }
    }
#pragma unroll
    for (int u = 0; u < BCH; ++u)
        if (u < nb) y[(int64_t)(b0 + u) * ys + r] = scale * s[u];
}

// r = D^-1 b, d0 = r / theta, x = d0 (the first update); one thread per entry
template <typename R>
__global__ void __launch_bounds__(CT) k_cheb_init(const R* __restrict__ dinv, int64_t n, R inv_theta,
                                                 const cx<R>* __restrict__ b, cx<R>* __restrict__ x,
                                                 cx<R>* __restrict__ r, cx<R>* __restrict__ d0) {
    const int64_t i = (int64_t)blockIdx.x * CT + threadIdx.x;
    if (i >= n) return;
    const int64_t o = (int64_t)blockIdx.y * n + i;
    const cx<R> ri = dinv[i] * b[o];
    r[o] = ri;
    const cx<R> di = inv_theta * ri;
    d0[o] = di;
    x[o] = di;
}

// r -= D^-1 A d; d' = c1 d + c2 r; x += d'
template <typename R, int BCH>
__global__ void __launch_bounds__(CT) k_cheb_step(const int* __restrict__ ptr, const int* __restrict__ col,
                                                 const R* __restrict__ val, const R* __restrict__ dinv, int64_t n,
                                                 const cx<R>* __restrict__ d, cx<R>* __restrict__ dn,
                                                 cx<R>* __restrict__ r, cx<R>* __restrict__ x, int nblk, R c1,
                                                 R c2) {
    const int64_t i = (int64_t)blockIdx.x * CT + threadIdx.x;
    if (i >= n) return;
    const int b0 = blockIdx.y * BCH;
    const int nb = min(BCH, nblk - b0);
    cx<R> s[BCH];
#pragma unroll
    for (int u = 0; u < BCH; ++u) s[u] = mk<R>(0, 0);
    for (int p = ptr[i]; p < ptr[i + 1]; ++p) {
        const R a = val[p];
        const cx<R>* dc = d + (int64_t)b0 * n + col[p];
#pragma unroll
        for (int u = 0; u < BCH; ++u)
            if (u < nb) {
                const cx<R> v = dc[(int64_t)u * n];
                s[u].re += a * v.re;
                s[u].im += a * v.im;
            }
    }
    const R di = dinv[i];
#pragma unroll
    for (int u = 0; u < BCH; ++u)
        if (u < nb) {
            const int64_t o = (int64_t)(b0 + u) * n + i;
            const cx<R> ri = r[o] - di * s[u];
            r[o] = ri;
            const cx<R> dv = c1 * d[o] + c2 * ri;
            dn[o] = dv;
            x[o] = x[o] + dv;
        }
}

constexpr int BCH_MANY = 8;  // blocks per thread for many right-hand sides
constexpr int BCH_FEW = 2;   // one right-hand side: its J and M blocks

}  // namespace

template <typename R>
cudaError_t csr_apply(const int* ptr, const int* col, const R* val, int64_t rows, const cx<R>* x, int64_t xs,
                      cx<R>* y, int64_t ys, int nblk, R scale, cudaStream_t st) {
    if (rows <= 0 || nblk <= 0) return cudaSuccess;
    const int bch = nblk >= BCH_MANY ? BCH_MANY : BCH_FEW;
    const int gy = (nblk + bch - 1) / bch;
    if (gy > 65535) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((rows + CT - 1) / CT), (unsigned)gy);
    if (bch == BCH_MANY)
        k_csr_apply<R, BCH_MANY><<<grid, CT, 0, st>>>(ptr, col, val, rows, x, xs, y, ys, nblk, scale);
    else
        k_csr_apply<R, BCH_FEW><<<grid, CT, 0, st>>>(ptr, col, val, rows, x, xs, y, ys, nblk, scale);
    return cudaGetLastError();
}

template <typename R>
cudaError_t chebyshev_solve(const int* ptr, const int* col, const R* val, const R* dinv, int64_t n,
                            const ChebPlan& p, const cx<R>* b, cx<R>* x, cx<R>* r, cx<R>* d0, cx<R>* d1, int nblk,
                            cudaStream_t st) {
    if (n <= 0 || nblk <= 0) return cudaSuccess;
    if (nblk > 65535 || p.steps < 1) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((n + CT - 1) / CT), (unsigned)nblk);
    k_cheb_init<R><<<grid, CT, 0, st>>>(dinv, n, (R)(1.0 / p.theta), b, x, r, d0);
    cudaError_t e = cudaGetLastError();
    const int bch = nblk >= BCH_MANY ? BCH_MANY : BCH_FEW;
    dim3 sgrid(grid.x, (unsigned)((nblk + bch - 1) / bch));
    for (int k = 0; k + 1 < p.steps && e == cudaSuccess; ++k) {
        const cx<R>* d = (k & 1) ? d1 : d0;
        cx<R>* dn = (k & 1) ? d0 : d1;
        if (bch == BCH_MANY)
            k_cheb_step<R, BCH_MANY><<<sgrid, CT, 0, st>>>(ptr, col, val, dinv, n, d, dn, r, x, nblk, (R)p.c1[k],
                                                            (R)p.c2[k]);
        else
            k_cheb_step<R, BCH_FEW><<<sgrid, CT, 0, st>>>(ptr, col, val, dinv, n, d, dn, r, x, nblk, (R)p.c1[k],
                                                           (R)p.c2[k]);
        e = cudaGetLastError();
    }
    return e;
}

template cudaError_t csr_apply<float>(const int*, const int*, const float*, int64_t, const c64*, int64_t, c64*,
                                      int64_t, int, float, cudaStream_t);
template cudaError_t csr_apply<double>(const int*, const int*, const double*, int64_t, const c128*, int64_t, c128*,
                                       int64_t, int, double, cudaStream_t);
template cudaError_t chebyshev_solve<float>(const int*, const int*, const float*, const float*, int64_t,
                                            const ChebPlan&, const c64*, c64*, c64*, c64*, c64*, int, cudaStream_t);
template cudaError_t chebyshev_solve<double>(const int*, const int*, const double*, const double*, int64_t,
                                             const ChebPlan&, const c128*, c128*, c128*, c128*, c128*, int,
                                             cudaStream_t);

}  // namespace cald
}  // namespace bem
