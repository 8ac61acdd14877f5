// libbem C interface: context, mesh -> RWG table, operator assembly, product,
// solve and powers.  Host code orchestrates; every step on the data runs in the
// kernels of the other translation units.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <map>
#include <tuple>
#include <numeric>

#include "common.cuh"

namespace bem {

// allocations left before the injected failures of bem_debug_fail_alloc_after (< 0: off)
static long long g_alloc_left = -1;

cudaError_t dalloc(DevBuf& b, size_t bytes) {
    dfree(b);
    if (bytes == 0) return cudaSuccess;
    if (g_alloc_left == 0) return cudaErrorMemoryAllocation;
    if (g_alloc_left > 0) --g_alloc_left;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        b.p = nullptr;
        return e;
    }
    b.bytes = bytes;
    return cudaSuccess;
}

}  // namespace bem

extern "C" void bem_debug_fail_alloc_after(long long after) { bem::g_alloc_left = after < 0 ? -1 : after; }

namespace bem {

void dfree(DevBuf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

}  // namespace bem

using namespace bem;

namespace {

// Work schedule of the rows kernel, for the forward or the adjoint product
struct RowsPlan {
    int64_t near_stride = 0;           // complex elements per operator array of the dense items
    int nslot = 0, pmax = 1;           // rows-kernel CTAs; most slots of one leaf
    DevBuf d_work_ptr, d_work_item, d_near_c0, d_near_n, d_near_off, d_pieces, d_ypart, d_arrive;
    DevBuf d_leaf_parts, d_slot_order, d_slot_leaf, d_slot_part;
    // host copies (schedules built from this one, e.g. the tensor-core product's)
    std::vector<int> h_wptr, h_witem, h_nc0, h_nn;
    std::vector<int64_t> h_noff, h_scost;
    std::vector<PieceDesc> h_pieces;
};

static void release_rows_plan(RowsPlan& r) {
    r.h_wptr.clear();
    r.h_witem.clear();
    r.h_nc0.clear();
    r.h_nn.clear();
    r.h_noff.clear();
    r.h_scost.clear();
    r.h_pieces.clear();
    DevBuf* plan[] = {&r.d_work_ptr,   &r.d_work_item, &r.d_near_c0,  &r.d_near_n,     &r.d_near_off,
                      &r.d_pieces,     &r.d_ypart,     &r.d_arrive,   &r.d_leaf_parts,
                      &r.d_slot_order, &r.d_slot_leaf, &r.d_slot_part};
    for (DevBuf* b : plan) dfree(*b);
    r.near_stride = 0;
    r.nslot = 0;
    r.pmax = 1;
}

struct Operator {
    bool built = false;
    // product plan of this precision: dense items (leaf row x column range) and far pieces
    std::vector<BlockDesc> items;      // dense items sorted by (r0, c0); rows are one leaf
    std::vector<BlockDesc> far_desc;   // blocks stored as factors (partition far blocks, or their splits)
    int64_t n_far_split = 0;           // far blocks split because their rank passed the cap
    int64_t n_far_dense = 0;           // partition far blocks stored densely (rank above break-even)
    int row_target = BEM_ROW_TARGET_CTAS;  // rows-kernel slots aimed at (bem_autotune may change it)
    RowsPlan fwd;         // rows kernel of Z x (items by row leaf)
    RowsPlan adj;         // rows kernel of Z^H x (transposed items, by column leaf); built on first use
    bool adj_built = false;
    DevBuf near;          // 3 * fwd.near_stride complex
    DevBuf nearT;         // transposed dense items, 3 * adj.near_stride complex (adjoint)
    DevBuf arena;         // low-rank factors
    DevBuf arena_bf16;    // BF16 copy of the factors (complex64 operator, BEM_PREC_BF16F)
    int64_t arena_len = 0;
    DevBuf far_rec;       // FarRec[nfar]
    DevBuf far_order;     // int2[nvhx]: V^H x units
    DevBuf xp, t;         // product workspace
    int64_t t_len = 0;
    int nvhx = 0;                      // units of the V^H x kernel
    int64_t factor_entries[3] = {0, 0, 0};
    int max_rank = 0;
    std::vector<FarRec> recs;
    // tensor-core product (complex64 operator, passes of 64 vectors); built on first use
    bool tc_built = false;
    RowsPlan tcp;                      // rows schedule with BEM_TC_ROW_TARGET slots
    DevBuf tc_tasks, tc_pairs, tc_xp, tc_t, tc_ypart, tc_vcta, tc_wcopy, tc_cta_slot_ptr, tc_cta_slots, tc_rec_ptr,
        tc_recs;
    int tc_ntask = 0;
};

struct GmresWork {  // the CG-type solvers' inner right-hand side and iterate
    int dtype = -1;
    int64_t n = 0;
    DevBuf xin, rin;
};

// workspace of the batched GMRES (gmres.cu): basis, iterate, right-hand sides and
// the per-right-hand-side Hessenberg state for nrhs columns of n
struct BgsWork {
    int dtype = -1, nrhs = 0, m = 0, chunk = 0, nblk = 0;
    int npart_cap = 0;  // partial norms per right-hand side that npart holds
    int64_t n = 0;
    DevBuf V, x, b, cplx, dbl, ints, part, npart;
    DevBuf zr, rr, cn;         // refinement: Z x and b - Z x (complex128), column norms
    int* host_active = nullptr;  // mapped host memory
    int* dev_active = nullptr;
};

}  // namespace

struct bem_ctx {
    bem_options opt;
    std::string err;
    // mesh and RWG table (host)
    int64_t nv = 0, nt = 0, ne = 0;
    std::vector<double> verts;
    std::vector<int> tris;
    std::vector<int> edge_v, edge_tri, edge_loc, tri_edge;
    std::vector<double> tri_coef, area, nrm, cen, diam, tv, mid;
    bool has_mesh = false, has_media = false;
    double k0 = 0;
    c128 eps{1, 0}, mu{1, 0}, k1{0, 0}, eta_r{1, 0};
    // device geometry
    DevBuf d_tv, d_area, d_nrm, d_cen, d_diam, d_tvid, d_tri_edge, d_tri_coef, d_edge_tri, d_edge_loc, d_mid;
    DevBuf d_sing_ptr, d_sing_b, d_sing_val;
    int64_t n_sing = 0;
    // cluster tree and partition
    std::vector<int> node_lo, node_hi, node_child0;
    std::vector<int64_t> perm;
    std::vector<int> leaf_lo, leaf_m;
    std::vector<BlockDesc> near_blocks, far_blocks;  // sorted by (r0, c0)
    DevBuf d_perm;
    // product plan (precision independent part)
    DevBuf d_leaf_r0, d_leaf_m, d_pos_leaf_lo, d_pos_leaf_m;
    DevBuf d_trif;
    Operator op[2];
    bool assembled = false;
    double assemble_ms = 0;
    double phase_ms[BEM_PHASES] = {0, 0, 0, 0, 0};
    // reductions and small transfers
    DevBuf d_part, d_red, d_tmp_in, d_one, d_gl;
    GmresWork gw;
    BgsWork bw;
    struct {
        int dtype = -1;
        int64_t n = 0;
        DevBuf v[8];
    } cgw;  // vectors of the CG-type solvers
    // kernel timing of bem_matvec
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;   // created once, reused
    size_t ev_used = 0;
    // one medium only (k1): the operator of one region of a layered body
    bool single = false;
    // layered body (bem_set_regions): one single-medium context per region, on the
    // region's boundary; edges[e] is the edge of this context that boundary edge e is,
    // sign[e] = +1 if the region lies on the normal side of that edge's surface
    struct Region {
        bem_ctx* sub = nullptr;
        std::vector<int> edges;
        std::vector<signed char> sign;
        DevBuf d_edges, d_sign;
    };
    std::vector<Region> regions;
    bool near_only = false;       // drop the far blocks (near-field refined operator of a preconditioner)
    int num_sms = 0;              // persistent CTAs of the tensor-core kernels
    int64_t tc_passes = 0;        // tensor-core operator passes since the last assembly
    int* tc_err_host = nullptr;   // set by a tensor-core kernel whose bounded wait ran out (mapped host memory)
    int* tc_err_dev = nullptr;
    DevBuf d_rx, d_ry;   // one region's operand and product
    DevBuf d_xext;       // the currents of the exterior boundary (powers)
    DevBuf d_far;        // quadrature points and weighted currents of the scattered power
    // Calderon preconditioner (BEM_PRECOND_CALDERON): refined-mesh context, sparse
    // matrices (host copies and FP32/FP64 device copies), Chebyshev plan, work
    struct Calderon {
        bem_ctx* fine = nullptr;
        cald::Csr C, Ct, G, Gt;
        cald::ChebPlan plan;
        DevBuf ptr[4], col[4], val32[4], val64[4];  // C, C^T, G, G^T
        DevBuf dinv32, dinv64;
        DevBuf u, r, d0, d1, vf, wf, py;
        double ms = 0;
        bool host = false;   // refinement, C, G and the plan (host only)
        bool built = false;  // plus the refined operator and the device copies
    } cal;
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
static bem_status fail(bem_ctx* c, bem_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

static bem_status cuda_fail(bem_ctx* c, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(c, e == cudaErrorMemoryAllocation ? BEM_ENOMEM : BEM_ECUDA, m);
}

#define CK(expr)                                            \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) return cuda_fail(c, _e, #expr); \
    } while (0)

// Kernels over right-hand sides put them on grid.y, whose limit is 65535
static std::string nrhs_msg(const char* fn, int nrhs) {
    char buf[160];
    snprintf(buf, sizeof buf, "%s: %d right-hand sides in one call; at most %d", fn, nrhs, BEM_MAX_NRHS);
    return buf;
}

template <typename T>
static cudaError_t upload(DevBuf& b, const std::vector<T>& v, cudaStream_t st) {
    cudaError_t e = dalloc(b, v.size() * sizeof(T));
    if (e != cudaSuccess || v.empty()) return e;
    e = cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

static cudaError_t ensure(DevBuf& b, size_t bytes) {
    if (b.bytes >= bytes && b.p) return cudaSuccess;
    return dalloc(b, bytes);
}

// internal product dtype: complex128 vectors, complex64 operator, FP64 sums
#define DT_C64_IN_FP64 100
static int esize_of(int dtype) { return (dtype == BEM_C128 || dtype == DT_C64_IN_FP64) ? 16 : 8; }
// element type of the vectors of a product dtype
static int vec_dtype(int dtype) { return (dtype == BEM_C64_BF16F || dtype == BEM_C64_TC) ? BEM_C64 : dtype; }

static GeomDev geom_view(const bem_ctx* c) {
    GeomDev g;
    g.nt = (int)c->nt;
    g.ne = (int)c->ne;
    g.tv = (const double*)c->d_tv.p;
    g.area = (const double*)c->d_area.p;
    g.nrm = (const double*)c->d_nrm.p;
    g.cen = (const double*)c->d_cen.p;
    g.diam = (const double*)c->d_diam.p;
    g.tvid = (const int*)c->d_tvid.p;
    g.tri_edge = (const int*)c->d_tri_edge.p;
    g.tri_coef = (const double*)c->d_tri_coef.p;
    g.edge_tri = (const int*)c->d_edge_tri.p;
    g.edge_loc = (const int*)c->d_edge_loc.p;
    g.sing_ptr = (const int*)c->d_sing_ptr.p;
    g.sing_b = (const int*)c->d_sing_b.p;
    g.sing_val = (const c128*)c->d_sing_val.p;
    g.trif = (const TriF*)c->d_trif.p;
    g.k0 = c->k0;
    g.k1 = c->k1;
    g.eta_r = c->eta_r;
    MediaConst<double> md;
    md.k0 = c->k0;
    md.k1r = c->k1.re;
    md.k1i = c->k1.im;
    md.jk0 = mk<double>(0.0, c->k0);
    md.jk1 = mk<double>(-c->k1.im, c->k1.re);
    md.jok0 = mk<double>(0.0, 1.0 / c->k0);
    md.jok1 = cdiv(mk<double>(0.0, 1.0), c->k1);
    md.er = c->eta_r;
    md.ie = cdiv(mk<double>(1.0, 0.0), c->eta_r);
    md.w0 = c->single ? 0.0 : 1.0;
    g.md = md;
    auto f = [](c128 z) { return mk<float>((float)z.re, (float)z.im); };
    g.mf.k0 = (float)md.k0;
    g.mf.k1r = (float)md.k1r;
    g.mf.k1i = (float)md.k1i;
    g.mf.jk0 = f(md.jk0);
    g.mf.jk1 = f(md.jk1);
    g.mf.jok0 = f(md.jok0);
    g.mf.jok1 = f(md.jok1);
    g.mf.er = f(md.er);
    g.mf.ie = f(md.ie);
    g.mf.w0 = (float)md.w0;
    return g;
}

static c128 csqrt_principal(c128 z) {
    double r = std::sqrt(z.re * z.re + z.im * z.im);
    double a = std::sqrt(std::max(0.0, 0.5 * (r + z.re)));
    double b = std::sqrt(std::max(0.0, 0.5 * (r - z.re)));
    if (z.im < 0) b = -b;
    return mk<double>(a, b);
}

static void release_operator(Operator& o) {
    release_rows_plan(o.fwd);
    release_rows_plan(o.adj);
    release_rows_plan(o.tcp);
    DevBuf* tcb[] = {&o.tc_tasks, &o.tc_pairs, &o.tc_xp, &o.tc_t, &o.tc_ypart, &o.tc_vcta, &o.tc_wcopy,
                     &o.tc_cta_slot_ptr, &o.tc_cta_slots, &o.tc_rec_ptr, &o.tc_recs};
    for (DevBuf* b : tcb) dfree(*b);
    o.tc_built = false;
    o.tc_ntask = 0;
    o.row_target = BEM_ROW_TARGET_CTAS;
    o.adj_built = false;
    dfree(o.nearT);
    o.items.clear();
    o.far_desc.clear();
    o.n_far_dense = 0;
    o.n_far_split = 0;
    dfree(o.near);
    dfree(o.arena);
    dfree(o.arena_bf16);
    o.arena_len = 0;
    dfree(o.far_rec);
    dfree(o.far_order);
    dfree(o.xp);
    dfree(o.t);
    o.built = false;
    o.t_len = 0;
    o.recs.clear();
    o.max_rank = 0;
    for (int i = 0; i < 3; ++i) o.factor_entries[i] = 0;
}

extern "C" void bem_destroy(bem_ctx* c);

static void release_calderon(bem_ctx* c) {
    auto& K = c->cal;
    if (K.fine) bem_destroy(K.fine);
    K.fine = nullptr;
    for (int i = 0; i < 4; ++i) {
        dfree(K.ptr[i]);
        dfree(K.col[i]);
        dfree(K.val32[i]);
        dfree(K.val64[i]);
    }
    DevBuf* w[] = {&K.dinv32, &K.dinv64, &K.u, &K.r, &K.d0, &K.d1, &K.vf, &K.wf, &K.py};
    for (DevBuf* b : w) dfree(*b);
    K.C = K.Ct = K.G = K.Gt = cald::Csr();
    K.plan = cald::ChebPlan();
    K.ms = 0;
    K.host = false;
    K.built = false;
}

static void invalidate(bem_ctx* c) {
    c->assembled = false;
    c->tc_passes = 0;
    for (int i = 0; i < 2; ++i) release_operator(c->op[i]);
    release_calderon(c);
}

// back to one body: drop the regions' contexts
static void clear_regions(bem_ctx* c) {
    for (auto& r : c->regions) {
        bem_destroy(r.sub);
        dfree(r.d_edges);
        dfree(r.d_sign);
    }
    c->regions.clear();
    dfree(c->d_rx);
    dfree(c->d_ry);
    dfree(c->d_xext);
}

static bool layered(const bem_ctx* c) { return !c->regions.empty(); }

// ---------------------------------------------------------------------------
// options, context
// ---------------------------------------------------------------------------
extern "C" void bem_default_options(bem_options* o) {
    if (!o) return;
    o->precision = BEM_PREC_C64;
    o->leaf_size = 64;
    o->eta = 2.0;
    o->aca_tol = 1e-4;
    o->aca_max_rank = 96;
    o->gmres_restart = 50;
    o->maxit = 1000;
    o->tol = 1e-6;
    o->refine_tol = 0.0;
    o->refine_maxit = 10;
    o->solver = BEM_SOLVER_GMRES;
    o->aca_recompress = 1;
    o->preconditioner = BEM_PRECOND_NONE;
    o->precond_aca_tol = 3e-2;
    o->precond_near_only = 0;
}

extern "C" bem_status bem_create(const bem_options* opt, bem_ctx** out) {
    if (!out) return BEM_EINVAL;
    *out = nullptr;
    bem_options o;
    bem_default_options(&o);
    if (opt) o = *opt;
    if (o.leaf_size < 2 || o.leaf_size > BEM_MAX_LEAF || (o.precision & 7) == 0 || (o.precision & ~7) != 0 ||
        o.aca_tol <= 0 || o.aca_max_rank < 1 || o.aca_max_rank > 128 || o.gmres_restart < 1 || o.gmres_restart > 200 || o.maxit < 1 ||
        o.tol <= 0 || o.refine_tol < 0 || o.refine_maxit < 1 || o.solver < BEM_SOLVER_GMRES ||
        o.solver > BEM_SOLVER_CGNR || o.aca_recompress < 0 || o.aca_recompress > 1 ||
        o.preconditioner < BEM_PRECOND_NONE || o.preconditioner > BEM_PRECOND_CALDERON ||
        !(o.precond_aca_tol > 0) || !(o.precond_aca_tol < 1) || o.precond_near_only < 0 || o.precond_near_only > 1)
        return BEM_EINVAL;
    bem_ctx* c = new (std::nothrow) bem_ctx();
    if (!c) return BEM_ENOMEM;
    c->opt = o;
    *out = c;
    return BEM_OK;
}

extern "C" void bem_destroy(bem_ctx* c) {
    if (!c) return;
    invalidate(c);
    clear_regions(c);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    DevBuf* bufs[] = {&c->d_tv, &c->d_area, &c->d_nrm, &c->d_cen, &c->d_diam, &c->d_tvid, &c->d_tri_edge,
                      &c->d_tri_coef, &c->d_edge_tri, &c->d_edge_loc, &c->d_mid, &c->d_sing_ptr, &c->d_sing_b,
                      &c->d_sing_val, &c->d_perm, &c->d_leaf_r0, &c->d_leaf_m, &c->d_pos_leaf_lo,
                      &c->d_pos_leaf_m, &c->d_part, &c->d_trif,
                      &c->d_red, &c->d_tmp_in, &c->d_one, &c->d_gl,
                      &c->gw.xin, &c->gw.rin, &c->cgw.v[0],
                      &c->cgw.v[1], &c->cgw.v[2], &c->cgw.v[3], &c->cgw.v[4], &c->cgw.v[5], &c->cgw.v[6],
                      &c->cgw.v[7], &c->bw.V, &c->bw.x, &c->bw.b, &c->bw.cplx, &c->bw.dbl, &c->bw.ints,
                      &c->bw.part, &c->bw.npart, &c->bw.zr, &c->bw.rr, &c->bw.cn, &c->d_far};
    for (DevBuf* b : bufs) dfree(*b);
    if (c->tc_err_host) cudaFreeHost(c->tc_err_host);
    if (c->bw.host_active) cudaFreeHost(c->bw.host_active);
    delete c;
}

extern "C" const char* bem_last_error(const bem_ctx* c) { return c ? c->err.c_str() : "null context"; }

extern "C" int64_t bem_num_edges(const bem_ctx* c) { return (c && c->has_mesh) ? c->ne : -1; }
extern "C" int64_t bem_num_unknowns(const bem_ctx* c) { return (c && c->has_mesh) ? 2 * c->ne : -1; }

// ---------------------------------------------------------------------------
// mesh -> RWG table (same conventions as the problem statement in bem.h)
// ---------------------------------------------------------------------------
extern "C" bem_status bem_set_mesh(bem_ctx* c, const double* verts, int64_t nv, const int32_t* tris, int64_t nt) {
    if (!c) return BEM_EINVAL;
    if (!verts || !tris || nv <= 0 || nt <= 0) return fail(c, BEM_EINVAL, "empty mesh");
    if (nt > (1 << 29) || nv > (1 << 30)) return fail(c, BEM_EINVAL, "mesh too large");
    invalidate(c);
    if (layered(c)) c->has_media = false;  // the regions belonged to the old mesh
    clear_regions(c);
    c->has_mesh = false;
    for (int64_t t = 0; t < nt; ++t)
        for (int i = 0; i < 3; ++i) {
            int v = tris[3 * t + i];
            if (v < 0 || v >= nv) return fail(c, BEM_EINVAL, "triangle index out of range");
        }
    std::vector<double> tv(9 * nt), area(nt), nrm(3 * nt), cen(3 * nt), diam(nt);
    for (int64_t t = 0; t < nt; ++t) {
        int a = tris[3 * t], b = tris[3 * t + 1], d = tris[3 * t + 2];
        if (a == b || b == d || a == d) return fail(c, BEM_EINVAL, "degenerate triangle (repeated vertex)");
        const double* p[3] = {verts + 3 * a, verts + 3 * b, verts + 3 * d};
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) tv[9 * t + 3 * i + k] = p[i][k];
        double e1[3], e2[3];
        for (int k = 0; k < 3; ++k) {
            e1[k] = p[1][k] - p[0][k];
            e2[k] = p[2][k] - p[0][k];
        }
        double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        double dbl = std::sqrt((cr[0] * cr[0] + cr[1] * cr[1]) + cr[2] * cr[2]);
        double lmax2 = 0.0, lmax = 0.0;
        for (int i = 0; i < 3; ++i) {
            const double* u = p[(i + 1) % 3];
            const double* v = p[(i + 2) % 3];
            double dx = u[0] - v[0], dy = u[1] - v[1], dz = u[2] - v[2];
            double s2 = (dx * dx + dy * dy) + dz * dz;
            lmax2 = std::max(lmax2, s2);
            lmax = std::max(lmax, std::sqrt(s2));
        }
        if (!(dbl > 1e-12 * lmax2)) return fail(c, BEM_EINVAL, "zero-area triangle");
        area[t] = 0.5 * dbl;
        for (int k = 0; k < 3; ++k) {
            nrm[3 * t + k] = cr[k] / dbl;
            cen[3 * t + k] = ((p[0][k] + p[1][k]) + p[2][k]) / 3.0;
        }
        diam[t] = lmax;
    }
    // half edges: (min, max, tri, local vertex opposite, direction)
    struct HE {
        int lo, hi, t, i, fwd;
    };
    std::vector<HE> he(3 * nt);
    for (int64_t t = 0; t < nt; ++t)
        for (int i = 0; i < 3; ++i) {
            int a = tris[3 * t + (i + 1) % 3], b = tris[3 * t + (i + 2) % 3];
            he[3 * t + i] = {std::min(a, b), std::max(a, b), (int)t, i, a < b ? 1 : 0};
        }
    std::sort(he.begin(), he.end(), [](const HE& x, const HE& y) {
        if (x.lo != y.lo) return x.lo < y.lo;
        if (x.hi != y.hi) return x.hi < y.hi;
        return x.t < y.t;
    });
    std::vector<int> edge_v, edge_tri, edge_loc;
    std::vector<int> tri_edge(3 * nt, -1);
    std::vector<double> tri_coef(3 * nt, 0.0);
    size_t k = 0;
    while (k < he.size()) {
        size_t j = k;
        while (j < he.size() && he[j].lo == he[k].lo && he[j].hi == he[k].hi) ++j;
        if (j - k != 2) return fail(c, BEM_EINVAL, "edge not shared by exactly two triangles (mesh not closed two-manifold)");
        HE a = he[k], b = he[k + 1];
        if (a.fwd == b.fwd) return fail(c, BEM_EINVAL, "inconsistent triangle orientation");
        if (a.t == b.t) return fail(c, BEM_EINVAL, "edge used twice by one triangle");
        if (b.t < a.t) std::swap(a, b);
        int e = (int)edge_v.size() / 2;
        edge_v.push_back(a.lo);
        edge_v.push_back(a.hi);
        edge_tri.push_back(a.t);
        edge_tri.push_back(b.t);
        edge_loc.push_back(a.i);
        edge_loc.push_back(b.i);
        const double* pa = verts + 3 * a.lo;
        const double* pb = verts + 3 * a.hi;
        double dx = pb[0] - pa[0], dy = pb[1] - pa[1], dz = pb[2] - pa[2];
        double len = std::sqrt((dx * dx + dy * dy) + dz * dz);
        tri_edge[3 * a.t + a.i] = e;
        tri_coef[3 * a.t + a.i] = len;
        tri_edge[3 * b.t + b.i] = e;
        tri_coef[3 * b.t + b.i] = -len;
        k = j;
    }
    int64_t ne = (int64_t)edge_v.size() / 2;
    std::vector<double> mid(3 * ne);
    for (int64_t e = 0; e < ne; ++e)
        for (int d = 0; d < 3; ++d) mid[3 * e + d] = (verts[3 * edge_v[2 * e] + d] + verts[3 * edge_v[2 * e + 1] + d]) * 0.5;
    c->nv = nv;
    c->nt = nt;
    c->ne = ne;
    c->verts.assign(verts, verts + 3 * nv);
    c->tris.assign(tris, tris + 3 * nt);
    c->edge_v.swap(edge_v);
    c->edge_tri.swap(edge_tri);
    c->edge_loc.swap(edge_loc);
    c->tri_edge.swap(tri_edge);
    c->tri_coef.swap(tri_coef);
    c->area.swap(area);
    c->nrm.swap(nrm);
    c->cen.swap(cen);
    c->diam.swap(diam);
    c->tv.swap(tv);
    c->mid.swap(mid);
    c->has_mesh = true;
    c->err.clear();
    return BEM_OK;
}

extern "C" bem_status bem_set_media(bem_ctx* c, double k0, bem_c128 eps_r, bem_c128 mu_r) {
    if (!c) return BEM_EINVAL;
    if (!(k0 > 0) || !std::isfinite(k0)) return fail(c, BEM_EINVAL, "k0 must be positive");
    if (eps_r.im > 0 || mu_r.im > 0) return fail(c, BEM_EINVAL, "Im eps_r and Im mu_r must be <= 0 (e^{+jwt})");
    if (eps_r.re == 0 && eps_r.im == 0) return fail(c, BEM_EINVAL, "eps_r must be nonzero");
    if (mu_r.re == 0 && mu_r.im == 0) return fail(c, BEM_EINVAL, "mu_r must be nonzero");
    invalidate(c);
    clear_regions(c);
    c->k0 = k0;
    c->eps = mk<double>(eps_r.re, eps_r.im);
    c->mu = mk<double>(mu_r.re, mu_r.im);
    c->k1 = k0 * csqrt_principal(c->eps * c->mu);
    c->eta_r = csqrt_principal(cdiv(c->mu, c->eps));
    c->has_media = true;
    c->err.clear();
    return BEM_OK;
}

// Layered body: surfaces between homogeneous regions (see bem.h).  Host only: the
// regions' boundary meshes, their edge maps and signs, and one context per region
// holding that region's medium alone.
extern "C" bem_status bem_set_regions(bem_ctx* c, double k0, int nreg, const bem_c128* eps_r, const bem_c128* mu_r,
                                      const int32_t* tri_regions) {
    if (!c) return BEM_EINVAL;
    if (!c->has_mesh) return fail(c, BEM_ESTATE, "bem_set_regions needs bem_set_mesh");
    if (!(k0 > 0) || !std::isfinite(k0)) return fail(c, BEM_EINVAL, "k0 must be positive");
    if (nreg < 2 || nreg > 4096 || !eps_r || !mu_r || !tri_regions) return fail(c, BEM_EINVAL, "bad arguments");
    for (int r = 1; r < nreg; ++r) {
        if (!std::isfinite(eps_r[r].re) || !std::isfinite(eps_r[r].im) || !std::isfinite(mu_r[r].re) ||
            !std::isfinite(mu_r[r].im))
            return fail(c, BEM_EINVAL, "eps_r and mu_r must be finite");
        if (eps_r[r].im > 0 || mu_r[r].im > 0)
            return fail(c, BEM_EINVAL, "Im eps_r and Im mu_r must be <= 0 (e^{+jwt})");
        if ((eps_r[r].re == 0 && eps_r[r].im == 0) || (mu_r[r].re == 0 && mu_r[r].im == 0))
            return fail(c, BEM_EINVAL, "eps_r and mu_r must be nonzero");
    }
    const int64_t nt = c->nt, ne = c->ne;
    for (int64_t t = 0; t < nt; ++t) {
        const int o = tri_regions[2 * t], i = tri_regions[2 * t + 1];
        if (o < 0 || o >= nreg || i < 0 || i >= nreg) return fail(c, BEM_EINVAL, "region index out of range");
        if (o == i) return fail(c, BEM_EINVAL, "a triangle must separate two different regions");
        if (i == 0) return fail(c, BEM_EINVAL, "normals of the surfaces bounding region 0 must point into it");
    }
    for (int64_t e = 0; e < ne; ++e) {
        const int a = c->edge_tri[2 * e], b = c->edge_tri[2 * e + 1];
        if (tri_regions[2 * a] != tri_regions[2 * b] || tri_regions[2 * a + 1] != tri_regions[2 * b + 1])
            return fail(c, BEM_EINVAL, "the two triangles of an edge bound different regions");
    }
    {
        std::vector<char> bounded(nreg, 0);
        for (int64_t t = 0; t < nt; ++t) bounded[tri_regions[2 * t]] = bounded[tri_regions[2 * t + 1]] = 1;
        for (int r = 0; r < nreg; ++r)
            if (!bounded[r]) return fail(c, BEM_EINVAL, "region " + std::to_string(r) + " has no boundary");
    }
    invalidate(c);
    clear_regions(c);
    c->has_media = false;
    c->regions.resize(nreg);
    std::vector<int> newid(c->nv);
    for (int r = 0; r < nreg; ++r) {
        bem_ctx::Region& R = c->regions[r];
        std::vector<int> tsel;
        for (int64_t t = 0; t < nt; ++t)
            if (tri_regions[2 * t] == r || tri_regions[2 * t + 1] == r) tsel.push_back((int)t);
        if (tsel.empty()) {
            clear_regions(c);
            return fail(c, BEM_EINVAL, "region " + std::to_string(r) + " has no boundary");
        }
        // vertices of the boundary, renumbered in increasing order (so the boundary's
        // edges keep the body's relative order and T+ / T- roles)
        std::fill(newid.begin(), newid.end(), -1);
        for (int t : tsel)
            for (int k = 0; k < 3; ++k) newid[c->tris[3 * t + k]] = 0;
        std::vector<int> vsel;
        for (int64_t v = 0; v < c->nv; ++v)
            if (newid[v] == 0) {
                newid[v] = (int)vsel.size();
                vsel.push_back((int)v);
            }
        std::vector<double> sv(3 * vsel.size());
        for (size_t v = 0; v < vsel.size(); ++v)
            for (int d = 0; d < 3; ++d) sv[3 * v + d] = c->verts[3 * (size_t)vsel[v] + d];
        std::vector<int32_t> stris(3 * tsel.size());
        for (size_t t = 0; t < tsel.size(); ++t)
            for (int k = 0; k < 3; ++k) stris[3 * t + k] = newid[c->tris[3 * (size_t)tsel[t] + k]];
        bem_status s = bem_create(&c->opt, &R.sub);
        if (s == BEM_OK) {
            s = bem_set_mesh(R.sub, sv.data(), (int64_t)vsel.size(), stris.data(), (int64_t)tsel.size());
            if (s != BEM_OK) c->err = "region " + std::to_string(r) + ": " + R.sub->err;
        } else {
            c->err = "region context";
        }
        if (s != BEM_OK) {
            clear_regions(c);
            return s;
        }
        bem_ctx* q = R.sub;
        // the region's medium alone, in the k1 slot (region 0: free space)
        q->k0 = k0;
        q->eps = r == 0 ? mk<double>(1, 0) : mk<double>(eps_r[r].re, eps_r[r].im);
        q->mu = r == 0 ? mk<double>(1, 0) : mk<double>(mu_r[r].re, mu_r[r].im);
        q->k1 = k0 * csqrt_principal(q->eps * q->mu);
        q->eta_r = csqrt_principal(cdiv(q->mu, q->eps));
        q->single = true;
        q->has_media = true;
        // boundary edge -> body edge: the body's edges are sorted by (min, max) vertex
        R.edges.resize(q->ne);
        R.sign.resize(q->ne);
        for (int64_t e = 0; e < q->ne; ++e) {
            const int lo = vsel[q->edge_v[2 * e]], hi = vsel[q->edge_v[2 * e + 1]];
            int64_t a = 0, b = ne;
            while (a < b) {
                const int64_t m = (a + b) / 2;
                const int ml = c->edge_v[2 * m], mh = c->edge_v[2 * m + 1];
                if (ml < lo || (ml == lo && mh < hi))
                    a = m + 1;
                else
                    b = m;
            }
            if (a >= ne || c->edge_v[2 * a] != lo || c->edge_v[2 * a + 1] != hi) {
                clear_regions(c);
                return fail(c, BEM_EINVAL, "boundary edge not found in the mesh");
            }
            R.edges[e] = (int)a;
            const int tb = tsel[q->edge_tri[2 * e]];
            R.sign[e] = tri_regions[2 * tb] == r ? 1 : -1;
        }
    }
    c->k0 = k0;
    c->eps = mk<double>(1, 0);
    c->mu = mk<double>(1, 0);
    c->k1 = mk<double>(k0, 0);
    c->eta_r = mk<double>(1, 0);
    c->has_media = true;
    c->err.clear();
    return BEM_OK;
}

extern "C" bem_status bem_region_boundary(const bem_ctx* cc, int r, int64_t* n_edges, int32_t* edges, int8_t* sign) {
    bem_ctx* c = const_cast<bem_ctx*>(cc);
    if (!c || !n_edges) return BEM_EINVAL;
    if (!layered(c)) return fail(c, BEM_ESTATE, "not a layered context (bem_set_regions)");
    if (r < 0 || r >= (int)c->regions.size()) return fail(c, BEM_EINVAL, "region index out of range");
    const bem_ctx::Region& R = c->regions[r];
    *n_edges = (int64_t)R.edges.size();
    for (size_t e = 0; e < R.edges.size(); ++e) {
        if (edges) edges[e] = R.edges[e];
        if (sign) sign[e] = R.sign[e];
    }
    return BEM_OK;
}

extern "C" bem_status bem_debye_eps(double f, const double* params, bem_c128* out) {
    if (!out || !(f >= 0) || !std::isfinite(f)) return BEM_EINVAL;
    double einf = 3.0, es = 60.0, e2 = 3.6, t1 = 10e-12, t2 = 0.2e-12;
    if (params) {
        einf = params[0];
        es = params[1];
        e2 = params[2];
        t1 = params[3];
        t2 = params[4];
    }
    double w = 2.0 * BEM_PI * f;
    c128 a = cdiv(mk<double>(es - e2, 0.0), mk<double>(1.0, w * t1));
    c128 b = cdiv(mk<double>(e2 - einf, 0.0), mk<double>(1.0, w * t2));
    out->re = einf + a.re + b.re;
    out->im = a.im + b.im;
    return BEM_OK;
}

extern "C" bem_status bem_edges(const bem_ctx* c, int32_t* out) {
    if (!c || !out) return BEM_EINVAL;
    if (!c->has_mesh) return BEM_ESTATE;
    for (int64_t e = 0; e < c->ne; ++e) {
        out[4 * e] = c->edge_v[2 * e];
        out[4 * e + 1] = c->edge_v[2 * e + 1];
        out[4 * e + 2] = c->edge_tri[2 * e];
        out[4 * e + 3] = c->edge_tri[2 * e + 1];
    }
    return BEM_OK;
}

// ---------------------------------------------------------------------------
// assembly
// ---------------------------------------------------------------------------
static bem_status upload_geometry(bem_ctx* c, cudaStream_t st) {
    std::vector<int> tvid(c->tris.begin(), c->tris.end());
    CK(upload(c->d_tv, c->tv, st));
    CK(upload(c->d_area, c->area, st));
    CK(upload(c->d_nrm, c->nrm, st));
    CK(upload(c->d_cen, c->cen, st));
    CK(upload(c->d_diam, c->diam, st));
    CK(upload(c->d_tvid, tvid, st));
    CK(upload(c->d_tri_edge, c->tri_edge, st));
    CK(upload(c->d_tri_coef, c->tri_coef, st));
    CK(upload(c->d_edge_tri, c->edge_tri, st));
    CK(upload(c->d_edge_loc, c->edge_loc, st));
    CK(upload(c->d_mid, c->mid, st));
    // FP32 triangle records
    std::vector<TriF> tf(c->nt);
    for (int64_t a = 0; a < c->nt; ++a) {
        TriF& r = tf[a];
        const double* cc = &c->cen[3 * a];
        float hi[3], lo[3];
        for (int d = 0; d < 3; ++d) {
            hi[d] = (float)cc[d];
            lo[d] = (float)(cc[d] - (double)hi[d]);
        }
        r.c_hi = make_float4(hi[0], hi[1], hi[2], (float)c->area[a]);
        r.c_lo = make_float4(lo[0], lo[1], lo[2], (float)c->diam[a]);
        for (int v = 0; v < 3; ++v) {
            const double* p = &c->tv[9 * a + 3 * v];
            r.v[v] = make_float4((float)(p[0] - cc[0]), (float)(p[1] - cc[1]), (float)(p[2] - cc[2]), 0.f);
        }
        r.coef = make_float4((float)c->tri_coef[3 * a], (float)c->tri_coef[3 * a + 1], (float)c->tri_coef[3 * a + 2],
                             (float)(1.0 / c->area[a]));
    }
    CK(upload(c->d_trif, tf, st));
    return BEM_OK;
}

static bem_status build_tree(bem_ctx* c, cudaStream_t st) {
    const int N = (int)c->ne, leaf = c->opt.leaf_size;
    // node ranges depend on sizes only: breadth-first layout
    std::vector<int> lo, hi, child0, level;
    lo.push_back(0);
    hi.push_back(N);
    child0.push_back(-1);
    level.push_back(0);
    for (size_t i = 0; i < lo.size(); ++i) {
        int sz = hi[i] - lo[i];
        if (sz > leaf) {
            child0[i] = (int)lo.size();
            int midp = lo[i] + sz / 2;
            lo.push_back(lo[i]);
            hi.push_back(midp);
            child0.push_back(-1);
            level.push_back(level[i] + 1);
            lo.push_back(midp);
            hi.push_back(hi[i]);
            child0.push_back(-1);
            level.push_back(level[i] + 1);
        }
    }
    const int nn = (int)lo.size();
    DevBuf d_lo, d_hi, d_child0, d_bbmin, d_bbmax, d_pos, d_split, d_perm2;
    struct Guard {
        DevBuf* b[8];
        ~Guard() {
            for (DevBuf* x : b) dfree(*x);
        }
    } guard{{&d_lo, &d_hi, &d_child0, &d_bbmin, &d_bbmax, &d_pos, &d_split, &d_perm2}};
    CK(upload(d_lo, lo, st));
    CK(upload(d_hi, hi, st));
    CK(upload(d_child0, child0, st));
    CK(dalloc(d_bbmin, sizeof(double) * 3 * nn));
    CK(dalloc(d_bbmax, sizeof(double) * 3 * nn));
    std::vector<int64_t> perm(N);
    std::iota(perm.begin(), perm.end(), 0);
    CK(upload(c->d_perm, perm, st));
    CK(dalloc(d_perm2, sizeof(int64_t) * N));
    CK(dalloc(d_pos, sizeof(int) * N));
    CK(dalloc(d_split, sizeof(int) * nn));
    const double* pts = (const double*)c->d_mid.p;
    int maxlev = *std::max_element(level.begin(), level.end());
    for (int L = 0; L <= maxlev; ++L) {
        int ls = (int)(std::find(level.begin(), level.end(), L) - level.begin());
        int le = ls;
        while (le < nn && level[le] == L) ++le;
        bool any = false;
        std::vector<int> pos(N, -1), split(le - ls, 0);
        for (int i = ls; i < le; ++i) {
            split[i - ls] = child0[i] >= 0;
            any |= child0[i] >= 0;
            for (int k = lo[i]; k < hi[i]; ++k) pos[k] = i - ls;
        }
        if (!any) break;
        CK(cudaMemcpyAsync(d_pos.p, pos.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(d_split.p, split.data(), sizeof(int) * split.size(), cudaMemcpyHostToDevice, st));
        CK(tree_bbox_level(pts, (const int64_t*)c->d_perm.p, (const int*)d_lo.p + ls, (const int*)d_hi.p + ls,
                           le - ls, (double*)d_bbmin.p + 3 * ls, (double*)d_bbmax.p + 3 * ls, st));
        CK(tree_split_level(pts, (const int64_t*)c->d_perm.p, (int64_t*)d_perm2.p, (const int*)d_lo.p + ls,
                            (const int*)d_hi.p + ls, (const double*)d_bbmin.p + 3 * ls,
                            (const double*)d_bbmax.p + 3 * ls, (const int*)d_split.p, le - ls, (const int*)d_pos.p, N,
                            st));
        std::swap(c->d_perm, d_perm2);
        CK(cudaStreamSynchronize(st));
    }
    CK(tree_bbox_level(pts, (const int64_t*)c->d_perm.p, (const int*)d_lo.p, (const int*)d_hi.p, nn,
                       (double*)d_bbmin.p, (double*)d_bbmax.p, st));
    CK(cudaMemcpyAsync(perm.data(), c->d_perm.p, sizeof(int64_t) * N, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    c->perm.swap(perm);
    c->node_lo = lo;
    c->node_hi = hi;
    c->node_child0 = child0;
    c->leaf_lo.clear();
    c->leaf_m.clear();
    for (int i = 0; i < nn; ++i)
        if (child0[i] < 0) {
            c->leaf_lo.push_back(lo[i]);
            c->leaf_m.push_back(hi[i] - lo[i]);
        }
    {
        std::vector<size_t> idx(c->leaf_lo.size());
        std::iota(idx.begin(), idx.end(), 0);
        std::sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return c->leaf_lo[a] < c->leaf_lo[b]; });
        std::vector<int> l2, m2;
        for (size_t i : idx) {
            l2.push_back(c->leaf_lo[i]);
            m2.push_back(c->leaf_m[i]);
        }
        c->leaf_lo.swap(l2);
        c->leaf_m.swap(m2);
    }
    // block tree, level by level on the device
    DevBuf d_cand, d_next, d_kind, d_counts, d_offs, d_tot, d_nearl, d_farl;
    struct Guard2 {
        DevBuf* b[8];
        ~Guard2() {
            for (DevBuf* x : b) dfree(*x);
        }
    } guard2{{&d_cand, &d_next, &d_kind, &d_counts, &d_offs, &d_tot, &d_nearl, &d_farl}};
    std::vector<int> cand0 = {0, 0};
    CK(upload(d_cand, cand0, st));
    CK(dalloc(d_tot, sizeof(int) * 3));
    int ncand = 1;
    std::vector<BlockDesc> nearv, farv;
    const double eta = c->opt.eta;
    while (ncand > 0) {
        CK(ensure(d_kind, sizeof(int) * ncand));
        CK(ensure(d_counts, sizeof(int) * 3 * ncand));
        CK(ensure(d_offs, sizeof(int) * 3 * ncand));
        CK(tree_block_level((const int*)d_cand.p, ncand, (const int*)d_lo.p, (const int*)d_hi.p,
                            (const int*)d_child0.p, (const double*)d_bbmin.p, (const double*)d_bbmax.p, eta,
                            (int*)d_kind.p, (int*)d_counts.p, st));
        for (int q = 0; q < 3; ++q)
            CK(scan_exclusive((const int*)d_counts.p + q * ncand, (int*)d_offs.p + q * ncand, ncand,
                              (int*)d_tot.p + q, st));
        int tot[3];
        CK(cudaMemcpyAsync(tot, d_tot.p, sizeof(tot), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        CK(dalloc(d_next, sizeof(int) * 2 * std::max(1, tot[2])));
        CK(ensure(d_nearl, sizeof(int) * 4 * std::max(1, tot[1])));
        CK(ensure(d_farl, sizeof(int) * 4 * std::max(1, tot[0])));
        CK(tree_block_emit((const int*)d_cand.p, ncand, (const int*)d_kind.p, (const int*)d_child0.p,
                           (const int*)d_offs.p, (int*)d_next.p, (int*)d_nearl.p, (int*)d_farl.p, (const int*)d_lo.p,
                           (const int*)d_hi.p, st));
        size_t n0 = nearv.size(), f0 = farv.size();
        nearv.resize(n0 + tot[1]);
        farv.resize(f0 + tot[0]);
        if (tot[1]) CK(cudaMemcpyAsync(nearv.data() + n0, d_nearl.p, sizeof(BlockDesc) * tot[1], cudaMemcpyDeviceToHost, st));
        if (tot[0]) CK(cudaMemcpyAsync(farv.data() + f0, d_farl.p, sizeof(BlockDesc) * tot[0], cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        std::swap(d_cand, d_next);
        ncand = tot[2];
    }
    auto canon = [](std::vector<BlockDesc>& v) {
        std::sort(v.begin(), v.end(), [](const BlockDesc& a, const BlockDesc& b) {
            return a.r0 != b.r0 ? a.r0 < b.r0 : a.c0 < b.c0;
        });
    };
    canon(nearv);
    canon(farv);
    c->near_blocks.swap(nearv);
    c->far_blocks.swap(farv);
    return BEM_OK;
}

static bem_status build_singular(bem_ctx* c, cudaStream_t st) {
    const int nt = (int)c->nt;
    DevBuf d_counts, d_pair_a, d_cell_start, d_cell_tri, d_tri_cell;
    struct Guard {
        DevBuf* b[5];
        ~Guard() {
            for (DevBuf* x : b) dfree(*x);
        }
    } guard{{&d_counts, &d_pair_a, &d_cell_start, &d_cell_tri, &d_tri_cell}};
    // centroid grid: cell edge h > 2 x (longest edge), so a pair closer than twice
    // the larger of its longest edges, or sharing a vertex, sits in adjacent cells
    SingGrid G;
    {
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300}, dmax = 0.0;
        for (int a = 0; a < nt; ++a) {
            for (int d = 0; d < 3; ++d) {
                lo[d] = std::min(lo[d], c->cen[3 * a + d]);
                hi[d] = std::max(hi[d], c->cen[3 * a + d]);
            }
            dmax = std::max(dmax, c->diam[a]);
        }
        double h = 2.0 * dmax * (1.0 + 1e-6) + 1e-300;
        int dims[3];
        for (;;) {
            int64_t cells = 1;
            for (int d = 0; d < 3; ++d) {
                dims[d] = (int)std::floor((hi[d] - lo[d]) / h) + 1;
                cells *= dims[d];
            }
            if (cells <= 4 * (int64_t)nt + 64) break;
            h *= 1.5;
        }
        const int ncell = dims[0] * dims[1] * dims[2];
        std::vector<int> tri_cell(nt), start(ncell + 1, 0), order(nt);
        for (int a = 0; a < nt; ++a) {
            int ci[3];
            for (int d = 0; d < 3; ++d)
                ci[d] = std::min(dims[d] - 1, std::max(0, (int)std::floor((c->cen[3 * a + d] - lo[d]) / h)));
            tri_cell[a] = (ci[2] * dims[1] + ci[1]) * dims[0] + ci[0];
            ++start[tri_cell[a] + 1];
        }
        for (int k = 0; k < ncell; ++k) start[k + 1] += start[k];
        std::vector<int> fillp(start.begin(), start.end() - 1);
        for (int a = 0; a < nt; ++a) order[fillp[tri_cell[a]]++] = a;
        CK(upload(d_cell_start, start, st));
        CK(upload(d_cell_tri, order, st));
        CK(upload(d_tri_cell, tri_cell, st));
        G.nx = dims[0];
        G.ny = dims[1];
        G.nz = dims[2];
        G.cell_start = (const int*)d_cell_start.p;
        G.cell_tri = (const int*)d_cell_tri.p;
        G.tri_cell = (const int*)d_tri_cell.p;
    }
    CK(dalloc(d_counts, sizeof(int) * nt));
    CK(dalloc(c->d_sing_ptr, sizeof(int) * (nt + 1)));
    GeomDev g = geom_view(c);
    CK(singular_count(g, G, (int*)d_counts.p, st));
    CK(scan_exclusive((const int*)d_counts.p, (int*)c->d_sing_ptr.p, nt, (int*)c->d_sing_ptr.p + nt, st));
    std::vector<int> ptr(nt + 1);
    CK(cudaMemcpyAsync(ptr.data(), c->d_sing_ptr.p, sizeof(int) * (nt + 1), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int64_t total = ptr[nt];
    c->n_sing = total;
    CK(dalloc(c->d_sing_b, sizeof(int) * std::max<int64_t>(1, total)));
    g = geom_view(c);
    CK(singular_fill(g, G, (const int*)c->d_sing_ptr.p, (int*)c->d_sing_b.p, st));
    std::vector<int> pa(total);
    for (int a = 0; a < nt; ++a)
        for (int k = ptr[a]; k < ptr[a + 1]; ++k) pa[k] = a;
    CK(upload(d_pair_a, pa, st));
    CK(dalloc(c->d_sing_val, sizeof(c128) * 36 * std::max<int64_t>(1, total)));
    g = geom_view(c);
    CK(singular_values(g, (int)total, (const int*)d_pair_a.p, (c128*)c->d_sing_val.p, st));
    CK(cudaStreamSynchronize(st));
    return BEM_OK;
}

static bem_status build_leaves(bem_ctx* c, cudaStream_t st) {
    CK(upload(c->d_leaf_r0, c->leaf_lo, st));
    CK(upload(c->d_leaf_m, c->leaf_m, st));
    std::vector<int> plo(c->ne), pm(c->ne);
    for (size_t l = 0; l < c->leaf_lo.size(); ++l)
        for (int k = c->leaf_lo[l]; k < c->leaf_lo[l] + c->leaf_m[l]; ++k) {
            plo[k] = c->leaf_lo[l];
            pm[k] = c->leaf_m[l];
        }
    CK(upload(c->d_pos_leaf_lo, plo, st));
    CK(upload(c->d_pos_leaf_m, pm, st));
    return BEM_OK;
}

// Work schedule of the rows kernel.  Every row leaf's dense items and far pieces
// are split over work slots (one 64-thread CTA each), largest item first to the
// least loaded slot (ties: lowest slot), so that the CTAs of a leaf stream about
// the same number of bytes.  Forward: items are (row leaf x column range) and a
// far block gives a piece to every leaf of its rows; adjoint: items are the
// transposed items and a far block gives a piece to every leaf of its columns.
static bem_status build_rows_plan(bem_ctx* c, const Operator& o, const std::vector<BlockDesc>& dense, bool adjoint,
                                  RowsPlan& rp, size_t es, cudaStream_t st, int target_slots = 0,
                                  int ypart_nr = BEM_MAX_NR) {
    const int target = target_slots > 0 ? target_slots : o.row_target;
    const int nleaf = (int)c->leaf_lo.size();
    std::vector<int> leaf_of(c->ne + 1, -1);
    for (int l = 0; l < nleaf; ++l) leaf_of[c->leaf_lo[l]] = l;
    // dense items
    std::vector<int> nc0, nn;
    std::vector<int64_t> noff;
    std::vector<std::vector<std::pair<int64_t, int>>> items(nleaf);  // (cost, encoded item)
    int64_t off = 0;
    for (size_t k = 0; k < dense.size(); ++k) {
        const BlockDesc& b = dense[k];
        int l = leaf_of[b.r0];
        if (l < 0 || c->leaf_m[l] != b.m) return fail(c, BEM_ECUDA, "dense item rows are not a leaf");
        nc0.push_back(b.c0);
        nn.push_back(b.n);
        noff.push_back(off);
        int64_t cost = (int64_t)b.m * 2 * ((b.n + 1) / 2);
        off += cost;
        items[l].push_back({3 * cost, (int)k});
    }
    rp.near_stride = off;
    // far pieces: every leaf inside a far block's row range (adjoint: column range)
    std::vector<int> fblk, frow;
    for (size_t k = 0; k < o.far_desc.size(); ++k) {
        const BlockDesc& F = o.far_desc[k];
        const FarRec& R = o.recs[k];
        int64_t kp2 = 2 * (int64_t)((R.rk[0] + 1) / 2 + (R.rk[1] + 1) / 2 + (R.rk[2] + 1) / 2);
        const int lo = adjoint ? F.c0 : F.r0, sz = adjoint ? F.n : F.m;
        int l = leaf_of[lo];
        if (l < 0) return fail(c, BEM_ECUDA, "far block does not start at a leaf");
        for (; l < nleaf && c->leaf_lo[l] < lo + sz; ++l) {
            int id = (int)fblk.size();
            fblk.push_back((int)k);
            frow.push_back(c->leaf_lo[l] - lo);
            items[l].push_back({(int64_t)c->leaf_m[l] * kp2, -1 - id});
        }
    }
    // Slots: a leaf's items are split into parts proportional to its share of the
    // work (about o.row_target slots in total, at most 32 per leaf), by
    // longest-processing-time assignment; CTAs take the slots heaviest first.
    int64_t total = 0;
    std::vector<int64_t> lw(nleaf, 0);
    for (int l = 0; l < nleaf; ++l)
        for (auto& it : items[l]) lw[l] += it.first;
    for (int l = 0; l < nleaf; ++l) total += lw[l];
    const double per_slot = std::max(1.0, (double)total / target);
    std::vector<int> wptr(1, 0), witem, lparts(nleaf), sleaf, spart;
    std::vector<int64_t> scost;
    rp.pmax = 1;
    for (int l = 0; l < nleaf; ++l) {
        auto& v = items[l];
        std::stable_sort(v.begin(), v.end(), [](const std::pair<int64_t, int>& x, const std::pair<int64_t, int>& y) {
            return x.first > y.first;
        });
        const int S = (int)std::max<int64_t>(
            1, std::min<int64_t>({32, (int64_t)v.size(), (int64_t)std::ceil((double)lw[l] / per_slot)}));
        lparts[l] = S;
        rp.pmax = std::max(rp.pmax, S);
        std::vector<int64_t> load(S, 0);
        std::vector<std::vector<int>> slot(S);
        for (auto& it : v) {
            int best = 0;
            for (int q = 1; q < S; ++q)
                if (load[q] < load[best]) best = q;
            load[best] += it.first;
            slot[best].push_back(it.second);
        }
        for (int q = 0; q < S; ++q) {
            for (int e : slot[q]) witem.push_back(e);
            wptr.push_back((int)witem.size());
            sleaf.push_back(l);
            spart.push_back(q);
            scost.push_back(load[q]);
        }
    }
    rp.nslot = (int)sleaf.size();
    std::vector<int> sorder(rp.nslot);
    std::iota(sorder.begin(), sorder.end(), 0);
    std::stable_sort(sorder.begin(), sorder.end(), [&](int x, int y) { return scost[x] > scost[y]; });
    CK(upload(rp.d_leaf_parts, lparts, st));
    CK(upload(rp.d_slot_order, sorder, st));
    CK(upload(rp.d_slot_leaf, sleaf, st));
    CK(upload(rp.d_slot_part, spart, st));
    CK(upload(rp.d_work_ptr, wptr, st));
    CK(upload(rp.d_work_item, witem, st));
    CK(upload(rp.d_near_c0, nc0, st));
    CK(upload(rp.d_near_n, nn, st));
    CK(upload(rp.d_near_off, noff, st));
    // flat piece descriptors
    std::vector<PieceDesc> pieces(fblk.size());
    for (size_t q = 0; q < fblk.size(); ++q) {
        const FarRec& R = o.recs[fblk[q]];
        const int ro = frow[q];
        PieceDesc& d = pieces[q];
        for (int k = 0; k < 3; ++k) {
            d.kp[k] = (R.rk[k] + 1) / 2;
            // forward: U slice of the leaf (pair (kp, i) at ro kpc + kp ms + i, stride ms);
            // adjoint: W rows so + i (pair (kp, j) at kp n + j, stride n)
            d.base[k] = adjoint ? R.off_v[k] + 2 * (int64_t)ro : R.off_u[k] + 2 * (int64_t)ro * d.kp[k];
        }
        const int l = leaf_of[(adjoint ? R.c0 : R.r0) + ro];
        d.ld = adjoint ? R.n : c->leaf_m[l];
        d.t_off = R.off_t;
    }
    CK(upload(rp.d_pieces, pieces, st));
    rp.h_wptr = wptr;
    rp.h_witem = witem;
    rp.h_nc0 = nc0;
    rp.h_nn = nn;
    rp.h_noff = noff;
    rp.h_scost = scost;
    rp.h_pieces = pieces;
    CK(dalloc(rp.d_ypart, es * 2 * c->ne * (rp.pmax > 1 ? rp.pmax : 1) * ypart_nr));
    CK(dalloc(rp.d_arrive, sizeof(unsigned int) * std::max(1, nleaf)));
    CK(cudaMemsetAsync(rp.d_arrive.p, 0, sizeof(unsigned int) * std::max(1, nleaf), st));
    CK(cudaStreamSynchronize(st));
    return BEM_OK;
}

template <typename R>
static bem_status build_operator(bem_ctx* c, Operator& o, cudaStream_t st) {
    const size_t es = sizeof(cx<R>);
    GeomDev g = geom_view(c);
    const int64_t* perm = (const int64_t*)c->d_perm.p;
    auto tp = std::chrono::steady_clock::now();
    auto lap = [&](int phase) {
        auto now = std::chrono::steady_clock::now();
        c->phase_ms[phase] += std::chrono::duration<double, std::milli>(now - tp).count();
        tp = now;
    };
    // 1. ACA of the far blocks, in rounds; each round in batches bounded by a scratch
    //    budget.  A block's rank is capped at the break-even m n / (m + n) and at the
    //    user cap.  A block that does not reach the tolerance within the cap is split
    //    into the pairs of its clusters' children (still admissible: they are no
    //    larger and no closer) for the next round; a leaf x leaf block that fails is
    //    stored densely.
    struct Batch {
        DevBuf arena;
        int64_t len;
    };
    std::vector<Batch> batches;
    struct BatchGuard {
        std::vector<Batch>* v;
        ~BatchGuard() {
            for (auto& b : *v) dfree(b.arena);
        }
    } bguard{&batches};
    struct Kept {
        BlockDesc F;
        int rk[3], batch[3];
        int64_t ou[3], ov[3];
    };
    std::vector<Kept> kept;
    std::vector<BlockDesc> dense_far;
    std::map<std::pair<int, int>, int> node_of;
    for (size_t i = 0; i < c->node_lo.size(); ++i) node_of[{c->node_lo[i], c->node_hi[i]}] = (int)i;
    auto children = [&](int lo, int sz, std::vector<std::pair<int, int>>& out) {
        out.clear();
        auto it = node_of.find({lo, lo + sz});
        int ch = (it == node_of.end()) ? -1 : c->node_child0[it->second];
        if (ch < 0) {
            out.push_back({lo, sz});
            return false;
        }
        for (int k = 0; k < 2; ++k) out.push_back({c->node_lo[ch + k], c->node_hi[ch + k] - c->node_lo[ch + k]});
        return true;
    };
    // scratch budget per batch: 4 GiB (complex64) or 8 GiB (complex128), at most a
    // quarter of the free device memory
    int64_t budget_bytes = (int64_t)(sizeof(R) == 4 ? 4 : 8) << 30;
    {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) budget_bytes = std::min<int64_t>(budget_bytes, (int64_t)fr / 4);
    }
    const int64_t budget = std::max<int64_t>(1, budget_bytes / (int64_t)es);  // complex elements
    const int rcap = c->opt.aca_max_rank;
    // the refined operator of a near-field Calderon preconditioner keeps no far blocks
    std::vector<BlockDesc> work = c->near_only ? std::vector<BlockDesc>() : c->far_blocks;
    o.n_far_split = 0;
    while (!work.empty()) {
        const int nw = (int)work.size();
        const int ntask = 3 * nw;  // task t: block t / 3, operator t % 3
        std::vector<int> ranks(ntask, 0), flags(ntask, 0), task_batch(ntask, 0), rmax_of(ntask);
        std::vector<int64_t> task_off_u(ntask), task_off_v(ntask), cost(ntask);
        for (int t = 0; t < ntask; ++t) {
            const BlockDesc& F = work[t / 3];
            int even = (int)std::max<int64_t>(1, (int64_t)F.m * F.n / (F.m + F.n));
            rmax_of[t] = std::min(rcap, std::min(even, std::min(F.m, F.n)));
            cost[t] = (int64_t)(F.m + F.n) * rmax_of[t];
        }
        // largest tasks first: each batch is a run of this order, so its CTAs are
        // scheduled longest-first and the batches holding the largest blocks come first
        std::vector<int> order(ntask);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
        size_t ob = 0;
        while (ob < order.size()) {
            std::vector<int> ids;
            int64_t scr = 0;
            size_t oe = ob;
            while (oe < order.size()) {
                const int t = order[oe];
                int64_t need = cost[t] + work[t / 3].n;
                if (!ids.empty() && scr + need > budget) break;
                ids.push_back(t);
                scr += need;
                ++oe;
            }
            // one kernel per (CTA width, operator): group the batch so, order kept
            auto group = [&](int t) { return (sizeof(R) == 4 && cost[t] >= BEM_ACA_WIDE_COST ? 0 : 3) + t % 3; };
            std::stable_sort(ids.begin(), ids.end(), [&](int x, int y) { return group(x) < group(y); });
            std::vector<AcaTask> tasks;
            int counts[6] = {0, 0, 0, 0, 0, 0};
            int max_m = 1;
            scr = 0;
            for (int t : ids) {
                const BlockDesc& F = work[t / 3];
                tasks.push_back({F.r0, F.m, F.c0, F.n, t % 3, rmax_of[t], scr});
                scr += cost[t] + F.n;
                ++counts[group(t)];
                max_m = std::max(max_m, F.m);
            }
            DevBuf d_tasks, d_scr, d_ranks, d_flags, d_ou, d_ov;
            struct G3 {
                DevBuf* b[6];
                ~G3() {
                    for (DevBuf* x : b) dfree(*x);
                }
            } g3{{&d_tasks, &d_scr, &d_ranks, &d_flags, &d_ou, &d_ov}};
            const int nt = (int)tasks.size();
            CK(upload(d_tasks, tasks, st));
            CK(dalloc(d_scr, es * scr));
            CK(dalloc(d_ranks, sizeof(int) * nt));
            CK(dalloc(d_flags, sizeof(int) * nt));
            {
                cudaError_t e = aca_run<R>(g, perm, (const AcaTask*)d_tasks.p, counts, (cx<R>*)d_scr.p,
                                           c->opt.aca_tol, (int*)d_ranks.p, (int*)d_flags.p, st, max_m);
                if (e != cudaSuccess) {
                    char buf[256];
                    snprintf(buf, sizeof buf, "ACA batch (%d tasks, largest block %d rows, %lld scratch elements): %s",
                             nt, max_m, (long long)scr, cudaGetErrorString(e));
                    return fail(c, e == cudaErrorMemoryAllocation ? BEM_ENOMEM : BEM_ECUDA, buf);
                }
            }
            std::vector<int> rk(nt), fl(nt);
            CK(cudaMemcpyAsync(rk.data(), d_ranks.p, sizeof(int) * nt, cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(fl.data(), d_flags.p, sizeof(int) * nt, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            if (c->opt.aca_recompress) {
                // truncate each converged task to the rank its singular values need;
                // workspace: the two k x k transforms of each task
                const int km = recompress_kmax<R>();
                std::vector<int64_t> woff(nt, 0);
                int64_t wl = 0;
                for (int i = 0; i < nt; ++i)
                    if (!fl[i] && rk[i] >= 2 && rk[i] <= km) {
                        woff[i] = wl;
                        wl += 2 * (int64_t)rk[i] * rk[i];
                    }
                if (wl > 0) {
                    DevBuf d_ws, d_woff;
                    struct G2 {
                        DevBuf* b[2];
                        ~G2() {
                            for (DevBuf* x : b) dfree(*x);
                        }
                    } g2{{&d_ws, &d_woff}};
                    CK(dalloc(d_ws, es * wl));
                    CK(upload(d_woff, woff, st));
                    CK(aca_recompress<R>((const AcaTask*)d_tasks.p, nt, (cx<R>*)d_scr.p, (int*)d_ranks.p,
                                         (const int*)d_flags.p, c->opt.aca_tol, (cx<R>*)d_ws.p,
                                         (const int64_t*)d_woff.p, st));
                    CK(cudaMemcpyAsync(rk.data(), d_ranks.p, sizeof(int) * nt, cudaMemcpyDeviceToHost, st));
                    CK(cudaStreamSynchronize(st));
                }
            }
            // factors of a converged task are kept (a failed task stores nothing)
            std::vector<int64_t> ou(nt), ov(nt);
            int64_t len = 0;
            for (int i = 0; i < nt; ++i) {
                const int t = ids[i];
                flags[t] = fl[i];
                int r = fl[i] ? 0 : rk[i];
                int rp = r + (r & 1);
                ou[i] = len;
                len += (int64_t)tasks[i].m * rp;
                ov[i] = len;
                len += (int64_t)tasks[i].n * rp;
                ranks[t] = r;
                task_off_u[t] = ou[i];
                task_off_v[t] = ov[i];
                task_batch[t] = (int)batches.size();
                rk[i] = r;
            }
            CK(cudaMemcpyAsync(d_ranks.p, rk.data(), sizeof(int) * nt, cudaMemcpyHostToDevice, st));
            Batch Bt;
            Bt.len = len;
            Bt.arena = DevBuf();
            CK(dalloc(Bt.arena, es * std::max<int64_t>(1, len)));
            batches.push_back(Bt);
            CK(upload(d_ou, ou, st));
            CK(upload(d_ov, ov, st));
            CK(aca_compact<R>((const AcaTask*)d_tasks.p, nt, (const cx<R>*)d_scr.p, (const int*)d_ranks.p,
                              (const int64_t*)d_ou.p, (const int64_t*)d_ov.p, (cx<R>*)batches.back().arena.p,
                              (const int*)c->d_pos_leaf_lo.p, (const int*)c->d_pos_leaf_m.p, st));
            CK(cudaStreamSynchronize(st));
            ob = oe;
        }
        std::vector<BlockDesc> next;
        std::vector<std::pair<int, int>> ct, cs;
        for (int b = 0; b < nw; ++b) {
            const BlockDesc& F = work[b];
            if (!(flags[3 * b] || flags[3 * b + 1] || flags[3 * b + 2])) {
                Kept k;
                k.F = F;
                for (int q = 0; q < 3; ++q) {
                    k.rk[q] = ranks[3 * b + q];
                    k.batch[q] = task_batch[3 * b + q];
                    k.ou[q] = task_off_u[3 * b + q];
                    k.ov[q] = task_off_v[3 * b + q];
                }
                kept.push_back(k);
                continue;
            }
            // a failed block keeps nothing (its factors occupy no arena space)
            bool st_ = children(F.r0, F.m, ct);
            bool ss_ = children(F.c0, F.n, cs);
            if (!st_ && !ss_) {
                dense_far.push_back(F);
                continue;
            }
            ++o.n_far_split;
            for (auto& a2 : ct)
                for (auto& b2 : cs) next.push_back({a2.first, a2.second, b2.first, b2.second});
        }
        work.swap(next);
    }
    lap(BEM_PHASE_ACA);
    // 2. dense items: leaf x leaf near blocks plus leaf x leaf far blocks above the rank cap
    o.items = c->near_blocks;
    o.far_desc.clear();
    o.n_far_dense = (int64_t)dense_far.size();
    for (const BlockDesc& F : dense_far) o.items.push_back(F);
    std::sort(o.items.begin(), o.items.end(), [](const BlockDesc& a, const BlockDesc& b) {
        return a.r0 != b.r0 ? a.r0 < b.r0 : a.c0 < b.c0;
    });
    // 3. dense entries
    {
        std::vector<int64_t> offs;
        int64_t off = 0;
        for (const BlockDesc& b : o.items) {
            offs.push_back(off);
            off += (int64_t)b.m * 2 * ((b.n + 1) / 2);
        }
        DevBuf d_blocks, d_offs;
        struct G4 {
            DevBuf* b[2];
            ~G4() {
                for (DevBuf* x : b) dfree(*x);
            }
        } g4{{&d_blocks, &d_offs}};
        CK(upload(d_blocks, o.items, st));
        CK(upload(d_offs, offs, st));
        CK(dalloc(o.near, es * 3 * std::max<int64_t>(1, off)));
        CK(near_assemble<R>(g, perm, (const BlockDesc*)d_blocks.p, (const int64_t*)d_offs.p, (int)o.items.size(),
                            (cx<R>*)o.near.p, off, st));
        CK(cudaStreamSynchronize(st));
    }
    lap(BEM_PHASE_NEAR);
    // 4. one factor arena
    std::vector<int64_t> base(batches.size() + 1, 0);
    for (size_t i = 0; i < batches.size(); ++i) base[i + 1] = base[i] + batches[i].len;
    CK(dalloc(o.arena, es * std::max<int64_t>(1, base.back())));
    for (size_t i = 0; i < batches.size(); ++i)
        if (batches[i].len)
            CK(cudaMemcpyAsync((char*)o.arena.p + es * base[i], batches[i].arena.p, es * batches[i].len,
                               cudaMemcpyDeviceToDevice, st));
    CK(cudaStreamSynchronize(st));
    o.arena_len = base.back();
    if constexpr (sizeof(R) == 4) {
        if (c->opt.precision & BEM_PREC_BF16F) {
            CK(dalloc(o.arena_bf16, sizeof(bf16c) * std::max<int64_t>(1, o.arena_len)));
            CK(factors_to_bf16((const c64*)o.arena.p, (bf16c*)o.arena_bf16.p, o.arena_len, st));
            CK(cudaStreamSynchronize(st));
        }
    }
    // 5. records of the blocks kept as factors
    const int nkeep = (int)kept.size();
    o.recs.resize(nkeep);
    o.far_desc.resize(nkeep);
    int64_t toff = 0;
    o.max_rank = 0;
    for (int i = 0; i < 3; ++i) o.factor_entries[i] = 0;
    for (int k = 0; k < nkeep; ++k) {
        const Kept& K = kept[k];
        const BlockDesc& F = K.F;
        o.far_desc[k] = F;
        FarRec& r = o.recs[k];
        r.r0 = F.r0;
        r.m = F.m;
        r.c0 = F.c0;
        r.n = F.n;
        int kp[3];
        for (int q = 0; q < 3; ++q) {
            r.rk[q] = K.rk[q];
            kp[q] = (K.rk[q] + 1) / 2;
            r.off_u[q] = base[K.batch[q]] + K.ou[q];
            r.off_v[q] = base[K.batch[q]] + K.ov[q];
            o.factor_entries[q] += (int64_t)K.rk[q] * (F.m + F.n);
            o.max_rank = std::max(o.max_rank, K.rk[q]);
        }
        r.off_t = toff;
        toff += 2 * (kp[0] + 2 * kp[1] + kp[2]);
    }
    o.t_len = toff;
    // V^H x units: (block, 8 items) for every kept block, largest blocks first
    std::vector<int> order(nkeep);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const FarRec &A = o.recs[a], &B = o.recs[b];
        int64_t wa = (int64_t)A.n * (A.rk[0] + A.rk[1] + A.rk[2]), wb = (int64_t)B.n * (B.rk[0] + B.rk[1] + B.rk[2]);
        return wa > wb;
    });
    std::vector<int2> units;
    for (int k : order) {
        const FarRec& r = o.recs[k];
        int items = (r.rk[0] + 1) / 2 + (r.rk[1] + 1) / 2 + (r.rk[2] + 1) / 2;
        for (int u = 0; u < (items + 7) / 8; ++u) units.push_back(make_int2(k, u));
    }
    o.nvhx = (int)units.size();
    CK(upload(o.far_rec, o.recs, st));
    CK(upload(o.far_order, units, st));
    bem_status s;
    if ((s = build_rows_plan(c, o, o.items, false, o.fwd, es, st)) != BEM_OK) return s;
    CK(dalloc(o.xp, es * 2 * c->ne * BEM_MAX_NR));
    CK(dalloc(o.t, es * std::max<int64_t>(1, o.t_len) * BEM_MAX_NR));
    lap(BEM_PHASE_PLAN);
    o.built = true;
    return BEM_OK;
}

// Layered body: the body's geometry (right-hand sides and powers) and one operator
// per region, each assembled by its own context on the region's boundary.
static bem_status assemble_layered(bem_ctx* c, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    invalidate(c);
    for (double& p : c->phase_ms) p = 0.0;
    bem_status s;
    if ((s = upload_geometry(c, st)) != BEM_OK) return s;
    for (size_t r = 0; r < c->regions.size(); ++r) {
        bem_ctx::Region& R = c->regions[r];
        if ((s = bem_assemble(R.sub, stream)) != BEM_OK)
            return fail(c, s, "region " + std::to_string(r) + ": " + R.sub->err);
        CK(upload(R.d_edges, R.edges, st));
        CK(upload(R.d_sign, R.sign, st));
        for (int i = 0; i < BEM_PHASES; ++i) c->phase_ms[i] += R.sub->phase_ms[i];
    }
    CK(cudaStreamSynchronize(st));
    c->assemble_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    c->assembled = true;
    c->err.clear();
    return BEM_OK;
}

// ---------------------------------------------------------------------------
// Calderon preconditioner: the refined-mesh context and the sparse matrices
// (calderon.cu holds the constructions and the kernels)
// ---------------------------------------------------------------------------
static MeshTables mesh_tables(const bem_ctx* c) {
    MeshTables m;
    m.nv = c->nv;
    m.nt = c->nt;
    m.ne = c->ne;
    m.verts = c->verts.data();
    m.tris = c->tris.data();
    m.edge_v = c->edge_v.data();
    m.edge_tri = c->edge_tri.data();
    m.edge_loc = c->edge_loc.data();
    m.tri_edge = c->tri_edge.data();
    m.tri_coef = c->tri_coef.data();
    m.area = c->area.data();
    m.nrm = c->nrm.data();
    return m;
}

// refinement, refined-mesh context with its mesh, BC and Gram matrices, Chebyshev plan
static bem_status calderon_host(bem_ctx* c) {
    auto& K = c->cal;
    if (K.host) return BEM_OK;
    const MeshTables mc = mesh_tables(c);
    std::vector<double> fv;
    std::vector<int> ft;
    cald::refine(mc, fv, ft);
    bem_options fo = c->opt;
    fo.preconditioner = BEM_PRECOND_NONE;
    fo.aca_tol = c->opt.precond_aca_tol;
    bem_status s = bem_create(&fo, &K.fine);
    if (s != BEM_OK) return fail(c, s, "Calderon preconditioner: cannot create the refined-mesh context");
    auto sub_fail = [&](bem_status s2, const char* what) {
        return fail(c, s2, std::string("Calderon preconditioner, ") + what + ": " + K.fine->err);
    };
    if ((s = bem_set_mesh(K.fine, fv.data(), (int64_t)fv.size() / 3, ft.data(), (int64_t)ft.size() / 3)) != BEM_OK)
        return sub_fail(s, "refined mesh");
    const MeshTables mf = mesh_tables(K.fine);
    std::string err;
    if (!cald::bc_matrix(mc, mf, K.C, err)) return fail(c, BEM_EINVAL, "Calderon preconditioner: " + err);
    K.Ct = cald::transpose(K.C);
    cald::mixed_gram(mc, mf, K.C, K.G);
    K.Gt = cald::transpose(K.G);
    // G^-1 as accurate as the refined operator needs: a hundredth of its ACA tolerance,
    // between 1e-10 and 1e-4
    const double gram_target = std::min(1e-4, std::max(1e-10, 0.01 * c->opt.precond_aca_tol));
    if (!cald::chebyshev_plan(K.G, gram_target, 60, K.plan, err))
        return fail(c, BEM_EINVAL, "Calderon preconditioner: " + err);
    K.host = true;
    return BEM_OK;
}

static bem_status build_calderon(bem_ctx* c, cudaStream_t st) {
    auto t0 = std::chrono::steady_clock::now();
    auto& K = c->cal;
    bem_status s;
    if ((s = calderon_host(c)) != BEM_OK) return s;
    const bem_c128 e{c->eps.re, c->eps.im}, m{c->mu.re, c->mu.im};
    if ((s = bem_set_media(K.fine, c->k0, e, m)) != BEM_OK)
        return fail(c, s, std::string("Calderon preconditioner, media: ") + K.fine->err);
    K.fine->near_only = c->opt.precond_near_only != 0;
    if ((s = bem_assemble(K.fine, st)) != BEM_OK)
        return fail(c, s, std::string("Calderon preconditioner, refined operator: ") + K.fine->err);
    const cald::Csr* mats[4] = {&K.C, &K.Ct, &K.G, &K.Gt};
    for (int i = 0; i < 4; ++i) {
        CK(upload(K.ptr[i], mats[i]->ptr, st));
        CK(upload(K.col[i], mats[i]->col, st));
        CK(upload(K.val64[i], mats[i]->val, st));
        const std::vector<float> v32(mats[i]->val.begin(), mats[i]->val.end());
        CK(upload(K.val32[i], v32, st));
    }
    std::vector<double> dinv(c->ne, 0.0);
    for (int64_t r = 0; r < c->ne; ++r)
        for (int p = K.G.ptr[r]; p < K.G.ptr[r + 1]; ++p)
            if (K.G.col[p] == r) dinv[r] = 1.0 / K.G.val[p];
    CK(upload(K.dinv64, dinv, st));
    const std::vector<float> d32(dinv.begin(), dinv.end());
    CK(upload(K.dinv32, d32, st));
    CK(cudaStreamSynchronize(st));
    K.built = true;
    K.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return BEM_OK;
}

extern "C" bem_status bem_assemble(bem_ctx* c, void* stream) {
    if (!c) return BEM_EINVAL;
    if (!c->has_mesh || !c->has_media) return fail(c, BEM_ESTATE, "bem_assemble needs bem_set_mesh and bem_set_media");
    if (layered(c) && c->opt.preconditioner != BEM_PRECOND_NONE)
        return fail(c, BEM_EINVAL, "the Calderon preconditioner is available for single-body contexts only");
    if (layered(c)) return assemble_layered(c, stream);
    cudaStream_t st = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    invalidate(c);
    for (double& p : c->phase_ms) p = 0.0;
    bem_status s;
    if ((s = upload_geometry(c, st)) != BEM_OK) return s;
    if ((s = build_tree(c, st)) != BEM_OK) return s;
    if ((s = build_leaves(c, st)) != BEM_OK) return s;
    CK(cudaStreamSynchronize(st));
    auto t1 = std::chrono::steady_clock::now();
    c->phase_ms[BEM_PHASE_TREE] = std::chrono::duration<double, std::milli>(t1 - t0).count();
    if ((s = build_singular(c, st)) != BEM_OK) return s;
    CK(cudaStreamSynchronize(st));
    c->phase_ms[BEM_PHASE_SINGULAR] =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t1).count();
    if (c->opt.precision & (BEM_PREC_C64 | BEM_PREC_BF16F))
        if ((s = build_operator<float>(c, c->op[0], st)) != BEM_OK) return s;
    if (c->opt.precision & BEM_PREC_C128)
        if ((s = build_operator<double>(c, c->op[1], st)) != BEM_OK) return s;
    CK(cudaStreamSynchronize(st));
    if (c->opt.preconditioner == BEM_PRECOND_CALDERON)
        if ((s = build_calderon(c, st)) != BEM_OK) return s;
    c->assemble_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    c->assembled = true;
    c->err.clear();
    return BEM_OK;
}

extern "C" bem_status bem_stats_get(const bem_ctx* cc, bem_stats* out) {
    bem_ctx* c = const_cast<bem_ctx*>(cc);
    if (!c || !out) return BEM_EINVAL;
    if (!c->assembled) return fail(c, BEM_ESTATE, "not assembled");
    memset(out, 0, sizeof(*out));
    if (layered(c)) {
        // sums over the regions' operators (max_rank: their maximum)
        for (auto& R : c->regions) {
            bem_stats q;
            bem_status s = bem_stats_get(R.sub, &q);
            if (s != BEM_OK) return fail(c, s, R.sub->err);
            out->n_clusters += q.n_clusters;
            out->n_leaves += q.n_leaves;
            out->n_near += q.n_near;
            out->n_far += q.n_far;
            out->n_far_dense += q.n_far_dense;
            out->n_far_split += q.n_far_split;
            out->n_far_factored += q.n_far_factored;
            out->near_entries += q.near_entries;
            for (int k = 0; k < 3; ++k) {
                out->factor_entries[k] += q.factor_entries[k];
                out->kernel_bytes_c64[k] += q.kernel_bytes_c64[k];
                out->kernel_bytes_c128[k] += q.kernel_bytes_c128[k];
                out->kernel_bytes_bf16f[k] += q.kernel_bytes_bf16f[k];
            }
            out->max_rank = std::max(out->max_rank, q.max_rank);
            out->singular_pairs += q.singular_pairs;
            out->matvec_bytes_c64 += q.matvec_bytes_c64;
            out->matvec_bytes_c128 += q.matvec_bytes_c128;
            out->matvec_bytes_bf16f += q.matvec_bytes_bf16f;
            out->matvec_bytes_tc += q.matvec_bytes_tc;
            out->t_rows += q.t_rows;
            out->tc_passes += q.tc_passes;
            for (int k = 0; k < 3; ++k) out->kernel_bytes_tc[k] += q.kernel_bytes_tc[k];
        }
        out->ne = c->ne;
        out->nt = c->nt;
        out->assemble_ms = c->assemble_ms;
        for (int i = 0; i < BEM_PHASES; ++i) out->assemble_phase_ms[i] = c->phase_ms[i];
        return BEM_OK;
    }
    out->ne = c->ne;
    out->nt = c->nt;
    out->n_clusters = (int64_t)c->node_lo.size();
    out->n_leaves = (int64_t)c->leaf_lo.size();
    out->n_near = (int64_t)c->near_blocks.size();
    out->n_far = (int64_t)c->far_blocks.size();
    const Operator& o = c->op[0].built ? c->op[0] : c->op[1];
    for (const BlockDesc& b : o.items) out->near_entries += (int64_t)b.m * b.n;
    out->n_far_dense = o.n_far_dense;
    out->n_far_split = o.n_far_split;
    out->n_far_factored = (int64_t)o.far_desc.size();
    for (int q = 0; q < 3; ++q) out->factor_entries[q] = o.factor_entries[q];
    out->max_rank = o.max_rank;
    out->singular_pairs = c->n_sing;
    // algorithmic bytes: every stored entry once, x read once, y written once
    const int64_t nv = 2 * c->ne;
    for (int p = 0; p < 2; ++p) {
        const Operator& q = c->op[p];
        if (!q.built) continue;
        int64_t es = p == 0 ? 8 : 16;
        int64_t dense = 0, fu = 0, fv = 0;
        for (const BlockDesc& b : q.items) dense += (int64_t)b.m * b.n;
        for (const FarRec& r : q.recs)
            for (int k = 0; k < 3; ++k) {
                fu += (int64_t)r.rk[k] * r.m;
                fv += (int64_t)r.rk[k] * r.n;
            }
        int64_t* kb = p == 0 ? out->kernel_bytes_c64 : out->kernel_bytes_c128;
        kb[BEM_KERNEL_GATHER] = es * 2 * nv;
        kb[BEM_KERNEL_VHX] = es * (fv + nv);
        kb[BEM_KERNEL_ROWS] = es * (3 * dense + fu + 2 * nv);
        int64_t bytes = es * (3 * dense + fu + fv + 2 * nv);
        if (p == 0 && q.arena_bf16.p) {
            // factors as BF16 (4 bytes per complex value), everything else complex64
            out->kernel_bytes_bf16f[BEM_KERNEL_GATHER] = es * 2 * nv;
            out->kernel_bytes_bf16f[BEM_KERNEL_VHX] = 4 * fv + es * nv;
            out->kernel_bytes_bf16f[BEM_KERNEL_ROWS] = es * (3 * dense + 2 * nv) + 4 * fu;
            out->matvec_bytes_bf16f = es * (3 * dense + 2 * nv) + 4 * (fu + fv);
        }
        if (p == 0) {
            out->matvec_bytes_c64 = bytes;
            // tensor-core pass of BEM_TC_NR vectors
            const int64_t V = es * nv * BEM_TC_NR, T = es * q.t_len * BEM_TC_NR;
            out->matvec_bytes_tc = es * (3 * dense + fu + fv) + 2 * V;
            out->kernel_bytes_tc[BEM_KERNEL_GATHER] = 2 * V;
            out->kernel_bytes_tc[BEM_KERNEL_VHX] = es * fv + V + T;
            out->kernel_bytes_tc[BEM_KERNEL_ROWS] = es * (3 * dense + fu) + T + 2 * V;
            out->t_rows = q.t_len;
        } else {
            out->matvec_bytes_c128 = bytes;
        }
    }
    out->assemble_ms = c->assemble_ms;
    out->tc_passes = c->tc_passes;
    for (int i = 0; i < BEM_PHASES; ++i) out->assemble_phase_ms[i] = c->phase_ms[i];
    if (c->cal.built) {
        const auto& K = c->cal;
        bem_stats fs;
        bem_status s = bem_stats_get(K.fine, &fs);
        if (s != BEM_OK) return fail(c, s, K.fine->err);
        const int64_t ne = c->ne, nf = K.fine->ne, es = 8;
        const int64_t nnzC = (int64_t)K.C.val.size(), nnzG = (int64_t)K.G.val.size();
        // per vector (two blocks of ne): Chebyshev init reads b and writes r, d, x; every
        // further step reads G and d, reads and writes r and x, writes d'
        const int64_t gram = es * 2 * ne * 4 + (K.plan.steps - 1) * (8 * nnzG + es * 2 * ne * 6);
        const int64_t csr = 8 * nnzC + es * 2 * (ne + nf);
        out->precond_fine_ne = nf;
        out->precond_gram_nnz = nnzG;
        out->precond_gram_steps = K.plan.steps;
        out->precond_bytes_c64 = fs.matvec_bytes_c64 + 2 * gram + 2 * csr;
        out->precond_gram_interval[0] = K.plan.lmin;
        out->precond_gram_interval[1] = K.plan.lmax;
        out->precond_assemble_ms = K.ms;
    }
    return BEM_OK;
}

extern "C" bem_status bem_partition(const bem_ctx* cc, int64_t* perm, int32_t* nearo, int32_t* faro) {
    bem_ctx* c = const_cast<bem_ctx*>(cc);
    if (!c) return BEM_EINVAL;
    if (!c->assembled) return fail(c, BEM_ESTATE, "not assembled");
    if (layered(c)) return fail(c, BEM_ESTATE, "bem_partition is not available on a layered context");
    if (perm) memcpy(perm, c->perm.data(), sizeof(int64_t) * c->ne);
    if (nearo) memcpy(nearo, c->near_blocks.data(), sizeof(BlockDesc) * c->near_blocks.size());
    if (faro) memcpy(faro, c->far_blocks.data(), sizeof(BlockDesc) * c->far_blocks.size());
    return BEM_OK;
}

// operator p (0: complex64, 1: complex128) built (for a layered body: in every region)
static bool op_built(const bem_ctx* c, int p) {
    if (layered(c)) {
        for (const auto& R : c->regions)
            if (!R.sub->op[p].built) return false;
        return c->assembled;
    }
    return c->op[p].built;
}

static bool bf16_built(const bem_ctx* c) {
    if (layered(c)) {
        for (const auto& R : c->regions)
            if (!R.sub->op[0].built || !R.sub->op[0].arena_bf16.p) return false;
        return c->assembled;
    }
    return c->op[0].built && c->op[0].arena_bf16.p != nullptr;
}

static bool dtype_ok(const bem_ctx* c, int dtype) {
    if (dtype == BEM_C64 || dtype == BEM_C64_TC) return op_built(c, 0);
    if (dtype == BEM_C128) return op_built(c, 1);
    if (dtype == BEM_C64_BF16F) return bf16_built(c);
    return false;
}

extern "C" bem_status bem_eval_entries(bem_ctx* c, const int32_t* rows, const int32_t* cols, int64_t count, void* out,
                                       int dtype, void* stream) {
    if (!c) return BEM_EINVAL;
    if (!c->assembled) return fail(c, BEM_ESTATE, "bem_eval_entries needs bem_assemble");
    if (layered(c)) return fail(c, BEM_ESTATE, "bem_eval_entries is not available on a layered context");
    if (count < 0 || (count > 0 && (!rows || !cols || !out))) return fail(c, BEM_EINVAL, "bad arguments");
    if (dtype != BEM_C64 && dtype != BEM_C128) return fail(c, BEM_EINVAL, "dtype");
    GeomDev g = geom_view(c);
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == BEM_C64)
        CK(eval_entries<float>(g, rows, cols, count, (c64*)out, st));
    else
        CK(eval_entries<double>(g, rows, cols, count, (c128*)out, st));
    return BEM_OK;
}

static MatvecPlan make_plan(const bem_ctx* c, const Operator& o, bool adjoint = false, bool tc = false) {
    const RowsPlan& rp = tc ? o.tcp : (adjoint ? o.adj : o.fwd);
    MatvecPlan p;
    p.ne = (int)c->ne;
    p.nleaf = (int)c->leaf_lo.size();
    p.nfar = (int)o.far_desc.size();
    p.perm = (const int64_t*)c->d_perm.p;
    p.leaf_r0 = (const int*)c->d_leaf_r0.p;
    p.leaf_m = (const int*)c->d_leaf_m.p;
    p.nslot = rp.nslot;
    p.pmax = rp.pmax;
    p.leaf_parts = (const int*)rp.d_leaf_parts.p;
    p.slot_order = (const int*)rp.d_slot_order.p;
    p.slot_leaf = (const int*)rp.d_slot_leaf.p;
    p.slot_part = (const int*)rp.d_slot_part.p;
    p.work_ptr = (const int*)rp.d_work_ptr.p;
    p.work_item = (const int*)rp.d_work_item.p;
    p.ypart = rp.d_ypart.p;
    p.arrive = (unsigned int*)rp.d_arrive.p;
    p.near_c0 = (const int*)rp.d_near_c0.p;
    p.near_n = (const int*)rp.d_near_n.p;
    p.near_off = (const int64_t*)rp.d_near_off.p;
    p.near_op_stride = rp.near_stride;
    p.pieces = (const PieceDesc*)rp.d_pieces.p;
    p.far = (const FarRec*)o.far_rec.p;
    p.vhx_units = (const int2*)o.far_order.p;
    p.nvhx = o.nvhx;
    p.pos_leaf_lo = (const int*)c->d_pos_leaf_lo.p;
    p.pos_leaf_m = (const int*)c->d_pos_leaf_m.p;
    return p;
}

// Transposed dense items and the adjoint rows plan of operator o (first adjoint use)
template <typename R>
static bem_status ensure_adjoint(bem_ctx* c, Operator& o, cudaStream_t st) {
    if (o.adj_built) return BEM_OK;
    const size_t es = sizeof(cx<R>);
    const size_t ni = o.items.size();
    std::vector<BlockDesc> itemsT(ni);
    std::vector<int64_t> offF(ni), offT(ni);
    int64_t oF = 0, oT = 0;
    for (size_t k = 0; k < ni; ++k) {
        const BlockDesc& b = o.items[k];
        offF[k] = oF;
        oF += (int64_t)b.m * 2 * ((b.n + 1) / 2);
        itemsT[k] = {b.c0, b.n, b.r0, b.m};
        offT[k] = oT;
        oT += (int64_t)b.n * 2 * ((b.m + 1) / 2);
    }
    bem_status s;
    if ((s = build_rows_plan(c, o, itemsT, true, o.adj, es, st)) != BEM_OK) return s;
    if (o.adj.near_stride != oT || o.fwd.near_stride != oF) return fail(c, BEM_ECUDA, "adjoint item layout");
    DevBuf d_items, d_offF, d_offT;
    struct G {
        DevBuf* b[3];
        ~G() {
            for (DevBuf* x : b) dfree(*x);
        }
    } guard{{&d_items, &d_offF, &d_offT}};
    CK(upload(d_items, o.items, st));
    CK(upload(d_offF, offF, st));
    CK(upload(d_offT, offT, st));
    CK(dalloc(o.nearT, es * 3 * std::max<int64_t>(1, oT)));
    CK(transpose_items<R>((const BlockDesc*)d_items.p, (const int64_t*)d_offF.p, (const int64_t*)d_offT.p, (int)ni,
                          (const cx<R>*)o.near.p, oF, (cx<R>*)o.nearT.p, oT, st));
    CK(cudaStreamSynchronize(st));
    o.adj_built = true;
    return BEM_OK;
}

static bem_status ensure_adjoint_for(bem_ctx* c, int dtype, cudaStream_t st) {
    if (layered(c)) {
        for (auto& R : c->regions) {
            bem_status s = ensure_adjoint_for(R.sub, dtype, st);
            if (s != BEM_OK) return fail(c, s, R.sub->err);
        }
        return BEM_OK;
    }
    if (dtype == BEM_C64 || dtype == DT_C64_IN_FP64) return ensure_adjoint<float>(c, c->op[0], st);
    if (dtype == BEM_C128) return ensure_adjoint<double>(c, c->op[1], st);
    return fail(c, BEM_EINVAL, "the adjoint product exists for BEM_C64 and BEM_C128");
}

// Schedule and workspaces of the tensor-core product of the complex64 operator
// (first use): V^H x tasks (the far blocks' W column pairs grouped by column
// cluster and vector half, at most 32 pairs per task, largest first), a rows
// schedule with BEM_TC_ROW_TARGET slots, and the 64-vector workspaces.
static bem_status ensure_tc(bem_ctx* c, Operator& o, cudaStream_t st) {
    if (o.tc_built) return BEM_OK;
    {
        int dev = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev));
        int cc_major = 0, cc_minor = 0;
        CK(cudaDeviceGetAttribute(&cc_major, cudaDevAttrComputeCapabilityMajor, dev));
        CK(cudaDeviceGetAttribute(&cc_minor, cudaDevAttrComputeCapabilityMinor, dev));
        if (cc_major != 10 || cc_minor != 3)
            return fail(c, BEM_EINVAL, "the tensor-core product is built for sm_103 (GB300) only");
    }
    if (!c->tc_err_host) {
        CK(cudaHostAlloc((void**)&c->tc_err_host, sizeof(int), cudaHostAllocMapped));
        *c->tc_err_host = 0;
        CK(cudaHostGetDevicePointer((void**)&c->tc_err_dev, c->tc_err_host, 0));
    }
    // group (column cluster, half) -> list of pairs
    std::map<std::tuple<int, int, int>, std::vector<TcPair>> groups;
    for (const FarRec& r : o.recs) {
        const int kp[3] = {(r.rk[0] + 1) / 2, (r.rk[1] + 1) / 2, (r.rk[2] + 1) / 2};
        // t segments [tA | tB(J) | tB(M) | tC]
        const int64_t seg[4] = {0, 2 * (int64_t)kp[0], 2 * (int64_t)(kp[0] + kp[1]),
                                2 * (int64_t)(kp[0] + 2 * kp[1])};
        // half J: A -> tA, B -> tB(J); half M: B -> tB(M), C -> tC
        const int part_of[2][2] = {{0, 1}, {1, 2}};
        const int seg_of[2][2] = {{0, 1}, {2, 3}};
        for (int g = 0; g < 2; ++g) {
            auto& v = groups[std::make_tuple(r.c0, r.n, g)];
            for (int u = 0; u < 2; ++u) {
                const int q = part_of[g][u];
                for (int k = 0; k < kp[q]; ++k)
                    v.push_back({r.off_v[q] + 2 * (int64_t)k * r.n, r.off_t + seg[seg_of[g][u]] + 2 * (int64_t)k});
            }
        }
    }
    std::vector<TcVhxTask> all;
    std::vector<TcPair> pairs;
    for (auto& kv : groups) {
        const auto& v = kv.second;
        for (size_t p0 = 0; p0 < v.size(); p0 += 32) {
            TcVhxTask T{};
            T.c0 = std::get<0>(kv.first);
            T.n = std::get<1>(kv.first);
            T.g = std::get<2>(kv.first);
            T.npairs = (int)std::min<size_t>(32, v.size() - p0);
            T.pair0 = (int)pairs.size();
            for (int k = 0; k < T.npairs; ++k) pairs.push_back(v[p0 + k]);
            all.push_back(T);
        }
    }
    // Longest-processing-time assignment of work to the persistent CTAs: heaviest
    // first, each to the least loaded CTA (ties: lowest index); each CTA's share is
    // contiguous, in the order assigned.
    const int nsm = c->num_sms;
    auto lpt = [nsm](const std::vector<int64_t>& cost, std::vector<std::vector<int>>& per) {
        std::vector<int> order(cost.size());
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
        per.assign(nsm, {});
        std::vector<int64_t> load(nsm, 0);
        for (int i : order) {
            int best = 0;
            for (int q = 1; q < nsm; ++q)
                if (load[q] < load[best]) best = q;
            load[best] += cost[i];
            per[best].push_back(i);
        }
    };
    {
        std::vector<int64_t> cost(all.size());
        for (size_t i = 0; i < all.size(); ++i)  // K steps (one per 4 columns) plus a per-task epilogue
            cost[i] = (int64_t)((all[i].n + 3) / 4) + 16;
        std::vector<std::vector<int>> per;
        lpt(cost, per);
        std::vector<TcVhxTask> tasks;
        std::vector<int> vptr(1, 0);
        int64_t woff = 0;
        for (int b = 0; b < nsm; ++b) {
            for (int i : per[b]) {
                TcVhxTask T = all[i];
                T.wcopy = woff;
                woff += (int64_t)((T.n + 31) / 32) * 32 * 32;
                tasks.push_back(T);
            }
            vptr.push_back((int)tasks.size());
        }
        o.tc_ntask = (int)tasks.size();
        CK(upload(o.tc_tasks, tasks, st));
        CK(upload(o.tc_pairs, pairs, st));
        CK(upload(o.tc_vcta, vptr, st));
        CK(dalloc(o.tc_wcopy, sizeof(float4) * std::max<int64_t>(1, woff)));
        CK(tc_build_wcopy((const TcVhxTask*)o.tc_tasks.p, o.tc_ntask, (const TcPair*)o.tc_pairs.p, (const c64*)o.arena.p,
                          (float4*)o.tc_wcopy.p, st));
    }
    bem_status s;
    if ((s = build_rows_plan(c, o, o.items, false, o.tcp, sizeof(c64), st, BEM_TC_ROW_TARGET, 1)) != BEM_OK)
        return s;
    {
        // rows: slots by LPT; per CTA its slots' item records, an end record after each slot
        const RowsPlan& rp = o.tcp;
        std::vector<std::vector<int>> per;
        std::vector<int64_t> cost(rp.nslot);
        for (int k = 0; k < rp.nslot; ++k)
            cost[k] = rp.h_scost[k] + 2048 * (int64_t)(rp.h_wptr[k + 1] - rp.h_wptr[k]);  // + per-item overhead
        lpt(cost, per);
        std::vector<int> sptr(1, 0), slots, rptr(1, 0);
        std::vector<TcRec> recs;
        for (int b = 0; b < nsm; ++b) {
            for (int k : per[b]) {
                slots.push_back(k);
                for (int w = rp.h_wptr[k]; w < rp.h_wptr[k + 1]; ++w) {
                    const int item = rp.h_witem[w];
                    TcRec r{};
                    if (item >= 0) {
                        const int n = rp.h_nn[item];
                        for (int q = 0; q < 3; ++q) {
                            r.base[q] = rp.h_noff[item] + q * rp.near_stride;
                            r.npair[q] = (n + 1) / 2;
                        }
                        r.vec = rp.h_nc0[item];
                        r.n = n;
                        r.kind = 0;
                        r.ld = -1;  // the leaf's rows (set by the kernel from the slot)
                    } else {
                        const PieceDesc& d = rp.h_pieces[-1 - item];
                        for (int q = 0; q < 3; ++q) {
                            r.base[q] = d.base[q];
                            r.npair[q] = d.kp[q];
                        }
                        r.vec = d.t_off;
                        r.ld = d.ld;
                        r.kind = 1;
                    }
                    recs.push_back(r);
                }
                TcRec e{};
                e.kind = 2;
                recs.push_back(e);
            }
            sptr.push_back((int)slots.size());
            rptr.push_back((int)recs.size());
        }
        CK(upload(o.tc_cta_slot_ptr, sptr, st));
        CK(upload(o.tc_cta_slots, slots, st));
        CK(upload(o.tc_rec_ptr, rptr, st));
        CK(upload(o.tc_recs, recs, st));
    }
    const size_t nn = 2 * (size_t)c->ne;
    CK(dalloc(o.tc_xp, sizeof(c64) * nn * BEM_TC_NR));
    CK(dalloc(o.tc_t, sizeof(c64) * std::max<int64_t>(1, o.t_len) * BEM_TC_NR));
    CK(dalloc(o.tc_ypart, sizeof(c64) * nn * BEM_TC_NR * (o.tcp.pmax > 1 ? o.tcp.pmax : 1)));
    CK(cudaStreamSynchronize(st));
    o.tc_built = true;
    return BEM_OK;
}

static cudaError_t matvec_any(bem_ctx* c, int dtype, const void* x, void* y, int nrhs, cudaStream_t st,
                              bool record = false, bool adjoint = false);

// Layered body: y = sum_r Q_r^T Z_r Q_r x (adjoint: Z_r^H), Q_r taking region r's
// boundary unknowns with their signs (the continuity conditions of Eq. 7 written
// for every surface, each region's field radiated by its own boundary's currents)
static cudaError_t matvec_layered(bem_ctx* c, int dtype, const void* x, void* y, int nrhs, cudaStream_t st,
                                  bool record, bool adjoint) {
    const int es = esize_of(dtype);
    int64_t nmax = 0;
    for (const auto& R : c->regions) nmax = std::max<int64_t>(nmax, (int64_t)R.edges.size());
    const size_t need = (size_t)es * 2 * nmax * nrhs;
    BEM_CUDA_TRY(ensure(c->d_rx, need));
    BEM_CUDA_TRY(ensure(c->d_ry, need));
    BEM_CUDA_TRY(cudaMemsetAsync(y, 0, (size_t)es * 2 * c->ne * nrhs, st));
    for (auto& R : c->regions) {
        const int64_t ns = (int64_t)R.edges.size();
        const int* ed = (const int*)R.d_edges.p;
        const signed char* sg = (const signed char*)R.d_sign.p;
        BEM_CUDA_TRY(region_gather(x, es, c->ne, ed, sg, ns, nrhs, c->d_rx.p, st));
        BEM_CUDA_TRY(matvec_any(R.sub, dtype, c->d_rx.p, c->d_ry.p, nrhs, st, record, adjoint));
        BEM_CUDA_TRY(region_scatter_add(c->d_ry.p, es, c->ne, ed, sg, ns, nrhs, y, st));
    }
    return cudaSuccess;
}

// y = Z x (adjoint: y = Z^H x, after ensure_adjoint_for)
static cudaError_t matvec_any(bem_ctx* c, int dtype, const void* x, void* y, int nrhs, cudaStream_t st,
                              bool record, bool adjoint) {
    if (layered(c)) return matvec_layered(c, dtype, x, y, nrhs, st, record, adjoint);
    const cudaEvent_t* ev = nullptr;
    if (record && c->prof) {
        // 6 events per operator pass: chunks of 8, 4, 2, 1 right-hand sides (at most 4
        // for the FP64-sum form)
        size_t passes = 0;
        if (dtype == BEM_C64_TC) {
            passes = (size_t)((nrhs + BEM_TC_NR - 1) / BEM_TC_NR);
        } else {
            const int maxc = dtype == DT_C64_IN_FP64 ? 4 : 8;
            for (int left = nrhs; left > 0;) {
                left -= (left >= 8 && maxc >= 8) ? 8 : (left >= 4 ? 4 : (left >= 2 ? 2 : 1));
                ++passes;
            }
        }
        size_t need = c->ev_used + 6 * passes;
        while (c->ev_pool.size() < need) {
            cudaEvent_t e;
            cudaError_t err = cudaEventCreate(&e);
            if (err != cudaSuccess) return err;
            c->ev_pool.push_back(e);
        }
        ev = c->ev_pool.data() + c->ev_used;
        c->ev_used = need;
    }
    if (dtype == BEM_C64_TC) {
        if (adjoint) return cudaErrorInvalidValue;
        Operator& o = c->op[0];
        if (!o.tc_built) return cudaErrorNotReady;  // ensure_tc first
        c->tc_passes += (nrhs + BEM_TC_NR - 1) / BEM_TC_NR;
        const MatvecPlan p = make_plan(c, o, false, true);
        TcPlan tp;
        tp.tasks = (const TcVhxTask*)o.tc_tasks.p;
        tp.pairs = (const TcPair*)o.tc_pairs.p;
        tp.ntask = o.tc_ntask;
        tp.nsm = c->num_sms;
        tp.vcta_ptr = (const int*)o.tc_vcta.p;
        tp.wcopy = (const float4*)o.tc_wcopy.p;
        tp.cta_slot_ptr = (const int*)o.tc_cta_slot_ptr.p;
        tp.cta_slots = (const int*)o.tc_cta_slots.p;
        tp.cta_rec_ptr = (const int*)o.tc_rec_ptr.p;
        tp.recs = (const TcRec*)o.tc_recs.p;
        tp.xp = (c64*)o.tc_xp.p;
        tp.t = (c64*)o.tc_t.p;
        tp.ypart = (c64*)o.tc_ypart.p;
        tp.err = c->tc_err_dev;
        return matvec_tc_run(p, tp, o.near.p, o.arena.p, (const c64*)x, (c64*)y, nrhs, st, ev);
    }
    if (dtype == BEM_C64 || dtype == BEM_C64_BF16F) {
        Operator& o = c->op[0];
        const bool bf = dtype == BEM_C64_BF16F;
        if (bf && adjoint) return cudaErrorInvalidValue;
        return matvec_run<float>(make_plan(c, o, adjoint), adjoint ? o.nearT.p : o.near.p,
                                 bf ? o.arena_bf16.p : o.arena.p, (const c64*)x, (c64*)y, (c64*)o.xp.p, (c64*)o.t.p,
                                 nrhs, o.t_len, st, ev, bf ? BEM_FORM_BF16F : BEM_FORM_NATIVE, adjoint);
    }
    if (dtype == DT_C64_IN_FP64) {
        // complex128 vectors through the complex64 operator (double-float arithmetic,
        // chunks of up to 4 right-hand sides)
        Operator& o = c->op[0];
        return matvec_run<double>(make_plan(c, o, adjoint), adjoint ? o.nearT.p : o.near.p, o.arena.p,
                                  (const c128*)x, (c128*)y, (c128*)o.xp.p, (c128*)o.t.p, nrhs, o.t_len, st, ev,
                                  BEM_FORM_C64_IN_FP64, adjoint);
    }
    Operator& o = c->op[1];
    return matvec_run<double>(make_plan(c, o, adjoint), adjoint ? o.nearT.p : o.near.p, o.arena.p, (const c128*)x,
                              (c128*)y, (c128*)o.xp.p, (c128*)o.t.p, nrhs, o.t_len, st, ev, BEM_FORM_NATIVE, adjoint);
}

// y = P x with the Calderon preconditioner for k vectors (2 k blocks of ne):
// u = G^-1 x, v = C u, w = Z_fine v, u = -C^T w, y = G^-T u
template <typename R>
static cudaError_t calderon_steps(bem_ctx* c, int dtype, const void* x, void* y, int k, cudaStream_t st) {
    auto& K = c->cal;
    typedef cx<R> V;
    const bool dp = sizeof(R) == 8;
    const int64_t ne = c->ne, nf = K.fine->ne;
    const int nb = 2 * k;
    auto ptr = [&](int i) { return (const int*)K.ptr[i].p; };
    auto col = [&](int i) { return (const int*)K.col[i].p; };
    auto val = [&](int i) { return (const R*)(dp ? K.val64[i].p : K.val32[i].p); };
    const R* dinv = (const R*)(dp ? K.dinv64.p : K.dinv32.p);
    V *u = (V*)K.u.p, *r = (V*)K.r.p, *d0 = (V*)K.d0.p, *d1 = (V*)K.d1.p, *vf = (V*)K.vf.p, *wf = (V*)K.wf.p;
    BEM_CUDA_TRY(cald::chebyshev_solve<R>(ptr(2), col(2), val(2), dinv, ne, K.plan, (const V*)x, u, r, d0, d1, nb, st));
    BEM_CUDA_TRY(cald::csr_apply<R>(ptr(0), col(0), val(0), nf, u, ne, vf, nf, nb, (R)1, st));
    BEM_CUDA_TRY(matvec_any(K.fine, dtype, vf, wf, k, st));
    BEM_CUDA_TRY(cald::csr_apply<R>(ptr(1), col(1), val(1), ne, wf, nf, u, ne, nb, (R)-1, st));
    return cald::chebyshev_solve<R>(ptr(3), col(3), val(3), dinv, ne, K.plan, u, (V*)y, r, d0, d1, nb, st);
}

static cudaError_t calderon_apply(bem_ctx* c, int dtype, const void* x, void* y, int nrhs, cudaStream_t st) {
    auto& K = c->cal;
    const bool dp = vec_dtype(dtype) == BEM_C128;
    const size_t es = dp ? sizeof(c128) : sizeof(c64);
    const int64_t ne = c->ne, nf = K.fine->ne;
    const int chunk = 32767;  // two blocks per vector on grid.y
    const int kmax = std::min(nrhs, chunk);
    BEM_CUDA_TRY(ensure(K.u, es * ne * 2 * kmax));
    BEM_CUDA_TRY(ensure(K.r, es * ne * 2 * kmax));
    BEM_CUDA_TRY(ensure(K.d0, es * ne * 2 * kmax));
    BEM_CUDA_TRY(ensure(K.d1, es * ne * 2 * kmax));
    BEM_CUDA_TRY(ensure(K.vf, es * nf * 2 * kmax));
    BEM_CUDA_TRY(ensure(K.wf, es * nf * 2 * kmax));
    for (int r0 = 0; r0 < nrhs; r0 += chunk) {
        const int k = std::min(chunk, nrhs - r0);
        const char* xk = (const char*)x + es * 2 * ne * r0;
        char* yk = (char*)y + es * 2 * ne * r0;
        BEM_CUDA_TRY(dp ? calderon_steps<double>(c, dtype, xk, yk, k, st)
                        : calderon_steps<float>(c, dtype, xk, yk, k, st));
    }
    return cudaSuccess;
}

// the operator the inner solver iterates on: Z, or Z P with the Calderon preconditioner
static cudaError_t apply_op(bem_ctx* c, int dtype, const void* x, void* y, int nrhs, cudaStream_t st, bool adjoint) {
    if (adjoint || !c->cal.built) return matvec_any(c, dtype, x, y, nrhs, st, false, adjoint);
    const size_t es = vec_dtype(dtype) == BEM_C128 ? sizeof(c128) : sizeof(c64);
    BEM_CUDA_TRY(ensure(c->cal.py, es * 2 * c->ne * nrhs));
    BEM_CUDA_TRY(calderon_apply(c, dtype, x, c->cal.py.p, nrhs, st));
    return matvec_any(c, dtype, c->cal.py.p, y, nrhs, st, false, false);
}

// ---------------------------------------------------------------------------
// autotuner of the rows-kernel schedule
// ---------------------------------------------------------------------------
extern "C" bem_status bem_autotune(bem_ctx* c, int dtype, void* stream, int* chosen, double* ms_best) {
    if (!c) return BEM_EINVAL;
    if (!c->assembled) return fail(c, BEM_ESTATE, "bem_autotune needs bem_assemble");
    if (layered(c)) return fail(c, BEM_ESTATE, "bem_autotune is not available on a layered context");
    if (dtype != BEM_C64 && dtype != BEM_C128 && dtype != BEM_C64_BF16F) return fail(c, BEM_EINVAL, "dtype");
    if (!dtype_ok(c, dtype)) return fail(c, BEM_EINVAL, "no operator of that precision was assembled");
    cudaStream_t st = (cudaStream_t)stream;
    Operator& o = c->op[dtype == BEM_C128 ? 1 : 0];
    const size_t es = esize_of(dtype);
    const int64_t n = 2 * c->ne;
    DevBuf x, y;
    struct G {
        DevBuf* b[2];
        ~G() {
            for (DevBuf* z : b) dfree(*z);
        }
    } guard{{&x, &y}};
    CK(dalloc(x, es * n));
    CK(dalloc(y, es * n));
    CK(cudaMemsetAsync(x.p, 0, es * n, st));  // the schedule's time does not depend on the values
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    struct GE {
        cudaEvent_t a, b;
        ~GE() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } gev{e0, e1};
    // candidate slot counts: multiples of the SM count (4 .. 96 CTAs per SM over the product)
    const int cand[] = {4 * 152, 8 * 152, 16 * 152, 32 * 152, 48 * 152, 64 * 152, 96 * 152};
    int best = o.row_target;
    double best_ms = 1e300;
    bem_status s;
    for (int target : cand) {
        release_rows_plan(o.fwd);
        o.row_target = target;
        if ((s = build_rows_plan(c, o, o.items, false, o.fwd, es, st)) != BEM_OK) return s;
        for (int w = 0; w < 3; ++w) CK(matvec_any(c, dtype, x.p, y.p, 1, st));
        CK(cudaEventRecord(e0, st));
        const int reps = 10;
        for (int r = 0; r < reps; ++r) CK(matvec_any(c, dtype, x.p, y.p, 1, st));
        CK(cudaEventRecord(e1, st));
        CK(cudaEventSynchronize(e1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms / reps < best_ms) {
            best_ms = ms / reps;
            best = target;
        }
    }
    release_rows_plan(o.fwd);
    o.row_target = best;
    if ((s = build_rows_plan(c, o, o.items, false, o.fwd, es, st)) != BEM_OK) return s;
    if (o.adj_built) {  // the adjoint plan follows the same target
        release_rows_plan(o.adj);
        o.adj_built = false;
        dfree(o.nearT);
    }
    CK(cudaStreamSynchronize(st));
    if (chosen) *chosen = best;
    if (ms_best) *ms_best = best_ms;
    return BEM_OK;
}

// ---------------------------------------------------------------------------
// several operators' products in one CUDA graph
// ---------------------------------------------------------------------------
struct bem_batch {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int n = 0;
};

extern "C" bem_status bem_batch_create(bem_ctx* const* ctxs, int n, const void* const* x, void* const* y,
                                       const int* nrhs, int dtype, void* stream, bem_batch** out) {
    if (!out || n < 1 || !ctxs || !x || !y || !nrhs) return BEM_EINVAL;
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        bem_ctx* c = ctxs[i];
        if (!c || !c->assembled || layered(c) || !dtype_ok(c, dtype) || nrhs[i] < 1 || !x[i] || !y[i])
            return BEM_EINVAL;
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == c) return fail(c, BEM_EINVAL, "a context appears twice in a batch (shared workspaces)");
        if (c->prof) return fail(c, BEM_ESTATE, "bem_batch_create during bem_profile_begin");
    }
    cudaStream_t st = (cudaStream_t)stream;
    // capture on a private stream: one forked branch per operator, joined at the end
    cudaStream_t cap;
    bem_ctx* c = ctxs[0];  // errors are reported on the first context
    CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    std::vector<cudaStream_t> br(n, nullptr);
    std::vector<cudaEvent_t> ev(n + 1, nullptr);
    bem_batch* b = new (std::nothrow) bem_batch();
    cudaError_t e = b ? cudaSuccess : cudaErrorMemoryAllocation;
    for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&br[i], cudaStreamNonBlocking);
    for (int i = 0; i <= n && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    bool capturing = false;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        capturing = true;
        e = cudaEventRecord(ev[n], cap);
    }
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        e = cudaStreamWaitEvent(br[i], ev[n], 0);
        if (e == cudaSuccess) e = matvec_any(ctxs[i], dtype, x[i], y[i], nrhs[i], br[i]);
        if (e == cudaSuccess) e = cudaEventRecord(ev[i], br[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, ev[i], 0);
    }
    if (capturing) {
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (e == cudaSuccess) e = e2;
        if (b) b->graph = g;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e == cudaSuccess) e = cudaGraphUpload(b->exec, st);
    for (int i = 0; i < n; ++i)
        if (br[i]) cudaStreamDestroy(br[i]);
    for (cudaEvent_t v : ev)
        if (v) cudaEventDestroy(v);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
        if (b) {
            if (b->exec) cudaGraphExecDestroy(b->exec);
            if (b->graph) cudaGraphDestroy(b->graph);
            delete b;
        }
        return fail(ctxs[0], e == cudaErrorMemoryAllocation ? BEM_ENOMEM : BEM_ECUDA, cudaGetErrorString(e));
    }
    b->n = n;
    *out = b;
    return BEM_OK;
}

extern "C" bem_status bem_batch_launch(bem_batch* b, void* stream) {
    if (!b || !b->exec) return BEM_EINVAL;
    return cudaGraphLaunch(b->exec, (cudaStream_t)stream) == cudaSuccess ? BEM_OK : BEM_ECUDA;
}

extern "C" void bem_batch_destroy(bem_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    delete b;
}

extern "C" bem_status bem_profile_begin(bem_ctx* c) {
    if (!c) return BEM_EINVAL;
    c->prof = true;
    c->ev_used = 0;
    for (auto& R : c->regions) bem_profile_begin(R.sub);  // a layered body times its regions' products
    return BEM_OK;
}

extern "C" bem_status bem_profile_end(bem_ctx* c, double* ms_sum, int64_t* launches) {
    if (!c) return BEM_EINVAL;
    if (!c->prof) return fail(c, BEM_ESTATE, "bem_profile_end without bem_profile_begin");
    double ms[3] = {0, 0, 0};
    int64_t cnt[3] = {0, 0, 0};
    for (auto& R : c->regions) {
        if (!R.sub->prof) continue;
        double m2[3];
        int64_t n2[3];
        bem_status s = bem_profile_end(R.sub, m2, n2);
        if (s != BEM_OK) return fail(c, s, R.sub->err);
        for (int k = 0; k < 3; ++k) {
            ms[k] += m2[k];
            cnt[k] += n2[k];
        }
    }
    for (size_t i = 0; i + 6 <= c->ev_used; i += 6)
        for (int k = 0; k < 3; ++k) {
            CK(cudaEventSynchronize(c->ev_pool[i + 2 * k + 1]));
            float t = 0;
            CK(cudaEventElapsedTime(&t, c->ev_pool[i + 2 * k], c->ev_pool[i + 2 * k + 1]));
            ms[k] += t;
            cnt[k] += 1;
        }
    c->prof = false;
    c->ev_used = 0;
    if (ms_sum) memcpy(ms_sum, ms, sizeof(ms));
    if (launches) memcpy(launches, cnt, sizeof(cnt));
    return BEM_OK;
}

// The tensor-core product's schedule on this context (every region of a layered
// body), and the report of a tensor-core kernel whose bounded wait ran out
static bem_status prepare_tc(bem_ctx* c, cudaStream_t st) {
    if (layered(c)) {
        for (auto& R : c->regions) {
            bem_status s = prepare_tc(R.sub, st);
            if (s != BEM_OK) return fail(c, s, R.sub->err);
        }
        return BEM_OK;
    }
    bem_status s = ensure_tc(c, c->op[0], st);
    if (s != BEM_OK) return s;
    if (c->tc_err_host && *(volatile int*)c->tc_err_host)
        return fail(c, BEM_ETIMEOUT, "a tensor-core kernel gave up waiting for the tensor core (earlier call)");
    return BEM_OK;
}

extern "C" bem_status bem_matvec(bem_ctx* c, const void* x, void* y, int nrhs, int dtype, void* stream) {
    if (!c) return BEM_EINVAL;
    if (!c->assembled) return fail(c, BEM_ESTATE, "bem_matvec needs bem_assemble");
    if (!dtype_ok(c, dtype)) return fail(c, BEM_EINVAL, "no operator of that precision was assembled");
    if (nrhs < 1 || !x || !y) return fail(c, BEM_EINVAL, "bad arguments");
    int64_t bytes = (int64_t)esize_of(dtype) * 2 * c->ne * nrhs;
    const char* xa = (const char*)x;
    const char* ya = (const char*)y;
    if (xa < ya + bytes && ya < xa + bytes) return fail(c, BEM_EINVAL, "x and y overlap");
    if (dtype == BEM_C64_TC) {
        bem_status s = prepare_tc(c, (cudaStream_t)stream);
        if (s != BEM_OK) return s;
    }
    CK(matvec_any(c, dtype, x, y, nrhs, (cudaStream_t)stream, true));
    return BEM_OK;
}

extern "C" bem_status bem_matvec_adjoint(bem_ctx* c, const void* x, void* y, int nrhs, int dtype, void* stream) {
    if (!c) return BEM_EINVAL;
    if (!c->assembled) return fail(c, BEM_ESTATE, "bem_matvec_adjoint needs bem_assemble");
    if (dtype != BEM_C64 && dtype != BEM_C128) return fail(c, BEM_EINVAL, "dtype: BEM_C64 or BEM_C128");
    if (!dtype_ok(c, dtype)) return fail(c, BEM_EINVAL, "no operator of that precision was assembled");
    if (nrhs < 1 || !x || !y) return fail(c, BEM_EINVAL, "bad arguments");
    int64_t bytes = (int64_t)esize_of(dtype) * 2 * c->ne * nrhs;
    const char* xa = (const char*)x;
    const char* ya = (const char*)y;
    if (xa < ya + bytes && ya < xa + bytes) return fail(c, BEM_EINVAL, "x and y overlap");
    cudaStream_t st = (cudaStream_t)stream;
    bem_status s;
    if ((s = ensure_adjoint_for(c, dtype, st)) != BEM_OK) return s;
    CK(matvec_any(c, dtype, x, y, nrhs, st, true, true));
    return BEM_OK;
}

extern "C" bem_status bem_precond_apply(bem_ctx* c, const void* x, void* y, int nrhs, int dtype, void* stream) {
    if (!c) return BEM_EINVAL;
    if (!c->assembled || !c->cal.built)
        return fail(c, BEM_ESTATE, "bem_precond_apply needs bem_assemble with BEM_PRECOND_CALDERON");
    if (!dtype_ok(c, dtype)) return fail(c, BEM_EINVAL, "no operator of that precision was assembled");
    if (nrhs < 1 || !x || !y) return fail(c, BEM_EINVAL, "bad arguments");
    const int64_t bytes = (int64_t)esize_of(dtype) * 2 * c->ne * nrhs;
    const char* xa = (const char*)x;
    const char* ya = (const char*)y;
    if (xa < ya + bytes && ya < xa + bytes) return fail(c, BEM_EINVAL, "x and y overlap");
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == BEM_C64_TC) {
        bem_status s = prepare_tc(c->cal.fine, st);
        if (s != BEM_OK) return fail(c, s, c->cal.fine->err);
    }
    CK(calderon_apply(c, dtype, x, y, nrhs, st));
    return BEM_OK;
}

extern "C" bem_status bem_precond_matrix(const bem_ctx* cc, int which, int64_t* rows, int64_t* cols, int64_t* nnz,
                                         int32_t* ptr, int32_t* col, double* val) {
    bem_ctx* c = const_cast<bem_ctx*>(cc);
    if (!c) return BEM_EINVAL;
    if (c->opt.preconditioner != BEM_PRECOND_CALDERON)
        return fail(c, BEM_EINVAL, "bem_precond_matrix needs a context created with BEM_PRECOND_CALDERON");
    if (!c->has_mesh || layered(c)) return fail(c, BEM_ESTATE, "bem_precond_matrix needs a single-body mesh");
    if (which != 0 && which != 1) return fail(c, BEM_EINVAL, "which: 0 (BC functions) or 1 (mixed Gram matrix)");
    bem_status s = calderon_host(c);
    if (s != BEM_OK) return s;
    const cald::Csr& a = which == 0 ? c->cal.C : c->cal.G;
    if (rows) *rows = a.rows;
    if (cols) *cols = a.cols;
    if (nnz) *nnz = (int64_t)a.val.size();
    if (ptr) std::copy(a.ptr.begin(), a.ptr.end(), ptr);
    if (col) std::copy(a.col.begin(), a.col.end(), col);
    if (val) std::copy(a.val.begin(), a.val.end(), val);
    return BEM_OK;
}

extern "C" bem_status bem_rhs_planewave(bem_ctx* c, const double* khat, const bem_c128* e0, int nrhs, void* b,
                                        int dtype, void* stream) {
    if (!c) return BEM_EINVAL;
    if (!c->assembled) return fail(c, BEM_ESTATE, "bem_rhs_planewave needs bem_assemble");
    if (nrhs > BEM_MAX_NRHS) return fail(c, BEM_EINVAL, nrhs_msg("bem_rhs_planewave", nrhs));
    if (nrhs < 1 || !khat || !e0 || !b || (dtype != BEM_C64 && dtype != BEM_C128))
        return fail(c, BEM_EINVAL, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<double> buf(3 * nrhs + 6 * nrhs);
    memcpy(buf.data(), khat, sizeof(double) * 3 * nrhs);
    memcpy(buf.data() + 3 * nrhs, e0, sizeof(double) * 6 * nrhs);
    CK(ensure(c->d_tmp_in, sizeof(double) * buf.size()));
    CK(cudaMemcpyAsync(c->d_tmp_in.p, buf.data(), sizeof(double) * buf.size(), cudaMemcpyHostToDevice, st));
    GeomDev g = geom_view(c);
    const double* kd = (const double*)c->d_tmp_in.p;
    const c128* ed = (const c128*)(kd + 3 * nrhs);
    if (dtype == BEM_C64)
        CK(rhs_planewave<float>(g, kd, ed, nrhs, (c64*)b, st));
    else
        CK(rhs_planewave<double>(g, kd, ed, nrhs, (c128*)b, st));
    if (layered(c)) {
        // the incident field lives in region 0: zero on the surfaces that do not bound it
        const bem_ctx::Region& R = c->regions[0];
        const int es = dtype == BEM_C64 ? 8 : 16;
        const int64_t ns = (int64_t)R.edges.size();
        CK(ensure(c->d_rx, (size_t)es * 2 * ns * nrhs));
        CK(region_gather(b, es, c->ne, (const int*)R.d_edges.p, (const signed char*)R.d_sign.p, ns, nrhs, c->d_rx.p,
                         st));
        CK(cudaMemsetAsync(b, 0, (size_t)es * 2 * c->ne * nrhs, st));
        CK(region_scatter_add(c->d_rx.p, es, c->ne, (const int*)R.d_edges.p, (const signed char*)R.d_sign.p, ns,
                              nrhs, b, st));
    }
    CK(cudaStreamSynchronize(st));
    return BEM_OK;
}

// ---------------------------------------------------------------------------
// solve: restarted GMRES (FP64 inner products) + optional FP64 refinement
// ---------------------------------------------------------------------------
static const int NPART = 304;  // 2 x 152 SMs of reduction partials

static bem_status norm_dev(bem_ctx* c, int dtype, const void* v, int64_t n, double* out, cudaStream_t st) {
    CK(ensure(c->d_part, sizeof(double) * NPART * 2));
    CK(kv_norm2(v, dtype, n, (double*)c->d_part.p, NPART, st));
    double h[NPART];
    CK(cudaMemcpyAsync(h, c->d_part.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    double s = 0;
    for (int i = 0; i < NPART; ++i) s += h[i];
    *out = std::sqrt(s);
    return BEM_OK;
}

// inner right-hand side and iterate of the CG-type solvers
static bem_status krylov_work(bem_ctx* c, int dtype) {
    GmresWork& w = c->gw;
    int64_t n = 2 * c->ne;
    if (w.dtype == dtype && w.n == n && w.xin.p) return BEM_OK;
    size_t es = esize_of(dtype);
    CK(dalloc(w.xin, es * n));
    CK(dalloc(w.rin, es * n));
    w.dtype = dtype;
    w.n = n;
    return BEM_OK;
}
// ---------------------------------------------------------------------------
// batched GMRES: all right-hand sides of a solve advance together, one product
// call per iteration over every basis vector; Gram-Schmidt, rotations, residual
// estimates and the restart's triangular solve run on the device (gmres.cu), and
// the host reads one mapped counter per iteration, one iteration behind.
// ---------------------------------------------------------------------------
static bem_status bgs_ensure(bem_ctx* c, int dtype, int nrhs, int m, cudaStream_t st) {
    BgsWork& w = c->bw;
    const int64_t n = 2 * c->ne;
    if (!w.host_active) {
        CK(cudaHostAlloc((void**)&w.host_active, sizeof(int), cudaHostAllocMapped));
        *w.host_active = 0;
        CK(cudaHostGetDevicePointer((void**)&w.dev_active, w.host_active, 0));
    }
    if (w.dtype == dtype && w.n == n && w.nrhs == nrhs && w.m == m && w.V.p) return BEM_OK;
    const size_t es = esize_of(dtype);
    int chunk, nblk, chunk16, nblk16;
    bgs_layout(n, nrhs, (int)es, &chunk, &nblk);
    bgs_layout(n, nrhs, 16, &chunk16, &nblk16);  // complex128 column norms (col_norms2)
    const int nblk_cap = std::max(nblk, nblk16);
    const size_t nc = (size_t)nrhs * ((size_t)(m + 1) * m + 3 * (size_t)(m + 1) + 3 * (size_t)m);
    CK(dalloc(w.V, es * n * nrhs * (m + 1)));
    CK(dalloc(w.x, es * n * nrhs));
    CK(dalloc(w.b, es * n * nrhs));
    CK(dalloc(w.cplx, sizeof(c128) * nc));
    CK(dalloc(w.dbl, sizeof(double) * 8 * nrhs));
    CK(dalloc(w.ints, sizeof(int) * 4 * nrhs));
    CK(dalloc(w.part, sizeof(c128) * nrhs * (m + 2) * (size_t)nblk));
    CK(dalloc(w.npart, sizeof(double) * nrhs * (size_t)nblk_cap));
    CK(dalloc(w.zr, sizeof(c128) * n * nrhs));
    CK(dalloc(w.rr, sizeof(c128) * n * nrhs));
    CK(dalloc(w.cn, sizeof(double) * nrhs));
    CK(cudaMemsetAsync(w.ints.p, 0, sizeof(int) * 4 * nrhs, st));  // arrival counters start at zero
    w.dtype = dtype;
    w.n = n;
    w.nrhs = nrhs;
    w.m = m;
    w.chunk = chunk;
    w.nblk = nblk;
    w.npart_cap = nblk_cap;
    return BEM_OK;
}

static BgsArgs bgs_args(bem_ctx* c, int maxit) {
    BgsWork& w = c->bw;
    BgsArgs a{};
    const int nr = w.nrhs, m = w.m;
    a.V = w.V.p;
    a.x = w.x.p;
    a.b = w.b.p;
    a.n = w.n;
    a.nrhs = nr;
    a.m = m;
    a.chunk = w.chunk;
    a.nblk = w.nblk;
    a.maxit = maxit;
    // Hessenberg state in the vectors' precision: complex values of es bytes
    const size_t es = esize_of(w.dtype);
    char* cp = (char*)w.cplx.p;
    a.H = cp;
    cp += es * nr * (m + 1) * m;
    a.g = cp;
    cp += es * nr * (m + 1);
    a.h1 = cp;
    cp += es * nr * (m + 1);
    a.h2 = cp;
    cp += es * nr * (m + 1);
    a.cs = cp;
    cp += es * nr * m;
    a.sn = cp;
    cp += es * nr * m;
    a.y = cp;
    double* dp = (double*)w.dbl.p;
    a.wn0 = dp;
    a.wn1 = dp + nr;
    a.wn2 = dp + 2 * nr;
    a.beta = dp + 3 * nr;
    a.tol = dp + 4 * nr;
    a.scale = dp + 5 * nr;
    a.res = dp + 6 * nr;
    int* ip = (int*)w.ints.p;
    a.cnt = (unsigned*)ip;
    a.state = ip + nr;
    a.kk = ip + 2 * nr;
    a.it = ip + 3 * nr;
    a.part = (c128*)w.part.p;
    a.npart = (double*)w.npart.p;
    a.host_active = w.dev_active;
    return a;
}

// Z x = b for the nrhs columns of bw.b (dtype vectors), x (bw.x) from zero.
// tol_abs: host, per right-hand side (infinity: leave it at zero); it_io: host,
// iterations so far per right-hand side (updated; each stops at maxit);
// beta_out: host, the true residual norm of the last restart per right-hand side.
static bem_status gmres_batched(bem_ctx* c, int pdt, const double* tol_abs, int maxit, int* it_io, double* beta_out,
                                cudaStream_t st, bool adjoint) {
    BgsWork& w = c->bw;
    const int nr = w.nrhs, m = w.m;
    const int64_t n = w.n;
    const size_t es = esize_of(w.dtype);
    const bool fp64 = w.dtype != BEM_C64;
    BgsArgs a = bgs_args(c, maxit);
    CK(cudaMemcpyAsync(a.tol, tol_abs, sizeof(double) * nr, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(a.it, it_io, sizeof(int) * nr, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(w.x.p, 0, es * n * nr, st));
    char* V = (char*)w.V.p;
    const size_t slot = es * n * nr;
    cudaEvent_t ev[2];
    CK(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
    struct GE {
        cudaEvent_t* e;
        ~GE() {
            cudaEventDestroy(e[0]);
            cudaEventDestroy(e[1]);
        }
    } gev{ev};
    bool x_zero = true;
    for (;;) {
        // restart: slot 0 = b - Z x, normalised; which right-hand sides go on
        if (!x_zero) CK(apply_op(c, pdt, w.x.p, V, nr, st, adjoint));
        CK(fp64 ? bgs_cycle_start<double>(a, x_zero, st) : bgs_cycle_start<float>(a, x_zero, st));
        x_zero = false;
        CK(cudaStreamSynchronize(st));
        if (*(volatile int*)w.host_active == 0) break;
        for (int j = 0; j < m; ++j) {
            CK(apply_op(c, pdt, V + slot * j, V + slot * (j + 1), nr, st, adjoint));
            CK(fp64 ? bgs_iteration<double>(a, j, st) : bgs_iteration<float>(a, j, st));
            CK(cudaEventRecord(ev[j & 1], st));
            if (j >= 1) {
                // iteration j is queued: wait for j - 1 and stop once nothing is active
                CK(cudaEventSynchronize(ev[(j - 1) & 1]));
                if (*(volatile int*)w.host_active == 0) break;
            }
        }
        CK(fp64 ? bgs_cycle_end<double>(a, st) : bgs_cycle_end<float>(a, st));
    }
    CK(cudaMemcpyAsync(it_io, a.it, sizeof(int) * nr, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(beta_out, a.beta, sizeof(double) * nr, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int r = 0; r < nr; ++r)
        if (!std::isfinite(beta_out[r]))
            return fail(c, BEM_ENOCONV,
                        "non-finite GMRES residual (NaN or Inf in the operator or the right-hand side)");
    return BEM_OK;
}

// Batched GMRES with optional FP64 refinement for nrhs right-hand sides (b, x device
// complex128, column-major), in groups whose basis fits the workspace budget.
static bem_status solve_gmres_batched(bem_ctx* c, const void* b, void* x, int nrhs, cudaStream_t st, int* iters,
                                      double* relres, bool adjoint, int din, int dres) {
    const int64_t n = 2 * c->ne;
    const int vin = vec_dtype(din);
    const int m = c->opt.gmres_restart;
    const size_t per_rhs = (size_t)esize_of(vin) * n * (m + 1);
    const size_t budget = (size_t)8 << 30;  // bytes of Krylov basis per group
    int nb = (int)std::max<size_t>(1, std::min<size_t>((size_t)nrhs, budget / per_rhs));
    if (nb >= BEM_TC_NR) nb -= nb % BEM_TC_NR;
    // many right-hand sides of a complex64 solve: the tensor-core product
    int pin = din;
    if (!adjoint && vin == BEM_C64 && nb >= BEM_TC_MIN_RHS && op_built(c, 0)) {
        int dev = 0, mj = 0, mn = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&mj, cudaDevAttrComputeCapabilityMajor, dev));
        CK(cudaDeviceGetAttribute(&mn, cudaDevAttrComputeCapabilityMinor, dev));
        if (mj == 10 && mn == 3) {
            bem_status s0 = prepare_tc(c, st);
            if (s0 != BEM_OK) return s0;
            if (c->cal.built && (s0 = prepare_tc(c->cal.fine, st)) != BEM_OK) return fail(c, s0, c->cal.fine->err);
            pin = BEM_C64_TC;
        }
    }
    int total_it = 0;
    bool all_ok = true;
    for (int r0 = 0; r0 < nrhs; r0 += nb) {
        const int k = std::min(nb, nrhs - r0);
        bem_status s;
        if ((s = bgs_ensure(c, vin, k, m, st)) != BEM_OK) return s;
        BgsWork& w = c->bw;
        const c128* br = (const c128*)b + (size_t)r0 * n;
        c128* xr = (c128*)x + (size_t)r0 * n;
        unsigned* cnt = (unsigned*)w.ints.p;
        double* cn = (double*)w.cn.p;
        std::vector<double> bn(k), rn(k), rel(k, 0.0), tol_abs(k), fres(k);
        std::vector<int> used(k, 0), before(k);
        std::vector<char> stopped(k, 0), fin(k, 0), inner_ok(k, 1);
        std::vector<double> xn(k);
        CK(col_norms2(br, true, n, k, (double*)w.npart.p, w.npart_cap, cnt, cn, st));
        CK(cudaMemcpyAsync(bn.data(), cn, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        CK(col_norms2(xr, true, n, k, (double*)w.npart.p, w.npart_cap, cnt, cn, st));
        CK(cudaMemcpyAsync(xn.data(), cn, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        bool x_zero = true;  // the usual start: the first residual is b itself
        for (int r = 0; r < k; ++r) x_zero = x_zero && xn[r] == 0.0;
        for (int r = 0; r < k; ++r) {
            if (!std::isfinite(bn[r])) return fail(c, BEM_EINVAL, "the right-hand side has non-finite entries");
            bn[r] = std::sqrt(bn[r]);
            if (bn[r] == 0) CK(cudaMemsetAsync(xr + (size_t)r * n, 0, sizeof(c128) * n, st));
        }
        const bool refine = c->opt.refine_tol > 0;
        const int steps = refine ? c->opt.refine_maxit : 1;
        for (int step = 0;; ++step) {
            // r = b - Z x with the most accurate operator, for every column of the group
            if (step == 0 && x_zero) {
                CK(cudaMemcpyAsync(w.rr.p, br, sizeof(c128) * n * k, cudaMemcpyDeviceToDevice, st));
            } else {
                CK(matvec_any(c, dres, xr, w.zr.p, k, st, false, adjoint));
                CK(kv_sub(br, w.zr.p, w.rr.p, BEM_C128, n * k, st));
            }
            CK(col_norms2(w.rr.p, true, n, k, (double*)w.npart.p, w.npart_cap, cnt, cn, st));
            CK(cudaMemcpyAsync(rn.data(), cn, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            bool more = false;
            for (int r = 0; r < k; ++r) {
                rn[r] = std::sqrt(rn[r]);
                if (bn[r] == 0) {
                    rel[r] = 0;
                    fin[r] = 1;
                    continue;
                }
                rel[r] = rn[r] / bn[r];
                fin[r] = refine ? rel[r] <= c->opt.refine_tol : step >= 1;
                if (!fin[r] && !stopped[r] && step < steps) more = true;
            }
            if (!more) break;
            for (int r = 0; r < k; ++r) {
                const bool go = !fin[r] && !stopped[r] && bn[r] != 0;
                // refinement steps after the first need only reach the outer target
                tol_abs[r] = go ? (refine ? std::max(c->opt.tol * rn[r], 0.5 * c->opt.refine_tol * bn[r])
                                          : c->opt.tol * rn[r])
                                : HUGE_VAL;
                before[r] = used[r];
            }
            // inner system Z d = r in the inner precision
            if (vin == BEM_C64)
                CK(kv_cast<float>(w.rr.p, BEM_C128, (c64*)w.b.p, n * k, st));
            else
                CK(cudaMemcpyAsync(w.b.p, w.rr.p, sizeof(c128) * n * k, cudaMemcpyDeviceToDevice, st));
            if ((s = gmres_batched(c, pin, tol_abs.data(), c->opt.maxit, used.data(), fres.data(), st, adjoint)) !=
                BEM_OK)
                return s;
            for (int r = 0; r < k; ++r) {
                if (tol_abs[r] == HUGE_VAL) continue;
                inner_ok[r] = fres[r] <= tol_abs[r] * 1.0000001;
                if (used[r] >= c->opt.maxit || used[r] == before[r]) stopped[r] = 1;  // measured next, then left
            }
            const void* dx = w.x.p;
            if (c->cal.built && !adjoint) {  // right preconditioning: the correction is P y
                CK(ensure(c->cal.py, (size_t)esize_of(vin) * n * k));
                CK(calderon_apply(c, pin, w.x.p, c->cal.py.p, k, st));
                dx = c->cal.py.p;
            }
            CK(kv_axpy_c128(xr, dx, vin, (const c128*)c->d_one.p, 1.0, n * k, 1, n * k, st));
        }
        for (int r = 0; r < k; ++r) {
            total_it += used[r];
            if (relres) relres[r0 + r] = rel[r];
            const bool ok = bn[r] == 0 || (refine ? rel[r] <= c->opt.refine_tol : (bool)inner_ok[r]);
            all_ok = all_ok && ok;
        }
    }
    CK(cudaStreamSynchronize(st));
    if (iters) *iters = total_it;
    if (!all_ok) return fail(c, BEM_ENOCONV, "solver did not reach its tolerance");
    return BEM_OK;
}

// a^H b with FP64 sums (host result; synchronises)
static bem_status dotc(bem_ctx* c, int dtype, const void* a, const void* b, int64_t n, c128* out, cudaStream_t st) {
    CK(ensure(c->d_part, sizeof(c128) * (NPART + 1)));
    c128* part = (c128*)c->d_part.p;
    CK(kv_multidot(a, dtype, n, 1, b, n, part, NPART, st));
    CK(kv_reduce_partials(part, NPART, 1, part + NPART, st));
    CK(cudaMemcpyAsync(out, part + NPART, sizeof(c128), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return BEM_OK;
}

static bem_status cg_work(bem_ctx* c, int dtype) {
    const int64_t n = 2 * c->ne;
    if (c->cgw.dtype == dtype && c->cgw.n == n && c->cgw.v[0].p) return BEM_OK;
    for (DevBuf& b : c->cgw.v) CK(dalloc(b, esize_of(dtype) * n));
    c->cgw.dtype = dtype;
    c->cgw.n = n;
    return BEM_OK;
}

// CGS, BiCGStab or CGNR on A x = rin (A = Z, or Z^H when adjoint), x = xin from zero;
// stops when the recurred residual norm reaches tol_abs.  Scalars on the host from
// FP64 inner products; vector updates fused in kv_lincomb.
static bem_status cg_family(bem_ctx* c, int pdt, int solver, double tol_abs, int maxit, int* iters,
                            double* final_res, cudaStream_t st, bool adjoint) {
    const int dtype = vec_dtype(pdt);
    const int64_t n = 2 * c->ne;
    bem_status s;
    if ((s = cg_work(c, dtype)) != BEM_OK) return s;
    GmresWork& gw = c->gw;
    void* x = gw.xin.p;
    void *r = c->cgw.v[0].p, *rt = c->cgw.v[1].p, *p = c->cgw.v[2].p, *q = c->cgw.v[3].p, *u = c->cgw.v[4].p,
         *v = c->cgw.v[5].p, *w = c->cgw.v[6].p, *t = c->cgw.v[7].p;
    const c128 one = mk<double>(1, 0), zero = mk<double>(0, 0);
    auto A = [&](const void* in, void* out, bool adj) { return matvec_any(c, pdt, in, out, 1, st, false, adj); };
    CK(cudaMemsetAsync(x, 0, esize_of(dtype) * n, st));
    CK(cudaMemcpyAsync(r, gw.rin.p, esize_of(dtype) * n, cudaMemcpyDeviceToDevice, st));
    double rn;
    if ((s = norm_dev(c, dtype, r, n, &rn, st)) != BEM_OK) return s;
    int it = 0;
    if (solver == BEM_SOLVER_CGS) {
        CK(cudaMemcpyAsync(rt, r, esize_of(dtype) * n, cudaMemcpyDeviceToDevice, st));
        c128 rho_prev = one;
        while (rn > tol_abs && it < maxit) {
            c128 rho;
            if ((s = dotc(c, dtype, rt, r, n, &rho, st)) != BEM_OK) return s;
            if (cabs2(rho) == 0.0) break;
            if (it == 0) {
                CK(kv_lincomb(u, dtype, one, r, zero, nullptr, zero, nullptr, n, st));
                CK(kv_lincomb(p, dtype, one, u, zero, nullptr, zero, nullptr, n, st));
            } else {
                const c128 beta = cdiv(rho, rho_prev);
                CK(kv_lincomb(u, dtype, one, r, beta, q, zero, nullptr, n, st));        // u = r + beta q
                CK(kv_lincomb(p, dtype, one, u, beta, q, beta * beta, p, n, st));      // p = u + beta q + beta^2 p
            }
            CK(A(p, v, adjoint));
            c128 sigma;
            if ((s = dotc(c, dtype, rt, v, n, &sigma, st)) != BEM_OK) return s;
            if (cabs2(sigma) == 0.0) break;
            const c128 alpha = cdiv(rho, sigma);
            const c128 malpha = mk<double>(-alpha.re, -alpha.im);
            CK(kv_lincomb(q, dtype, one, u, malpha, v, zero, nullptr, n, st));         // q = u - alpha v
            CK(kv_lincomb(w, dtype, one, u, one, q, zero, nullptr, n, st));            // w = u + q
            CK(kv_lincomb(x, dtype, one, x, alpha, w, zero, nullptr, n, st));          // x += alpha w
            CK(A(w, t, adjoint));
            CK(kv_lincomb(r, dtype, one, r, malpha, t, zero, nullptr, n, st));         // r -= alpha A w
            rho_prev = rho;
            ++it;
            if ((s = norm_dev(c, dtype, r, n, &rn, st)) != BEM_OK) return s;
        }
    } else if (solver == BEM_SOLVER_BICGSTAB) {
        CK(cudaMemcpyAsync(rt, r, esize_of(dtype) * n, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemsetAsync(p, 0, esize_of(dtype) * n, st));
        CK(cudaMemsetAsync(v, 0, esize_of(dtype) * n, st));
        c128 rho = one, alpha = one, omega = one;
        while (rn > tol_abs && it < maxit) {
            c128 rho_new;
            if ((s = dotc(c, dtype, rt, r, n, &rho_new, st)) != BEM_OK) return s;
            if (cabs2(rho_new) == 0.0 || cabs2(omega) == 0.0) break;
            const c128 beta = cdiv(rho_new, rho) * cdiv(alpha, omega);
            const c128 mbo = mk<double>(-(beta * omega).re, -(beta * omega).im);
            CK(kv_lincomb(p, dtype, one, r, beta, p, mbo, v, n, st));                 // p = r + beta (p - omega v)
            CK(A(p, v, adjoint));
            c128 rv;
            if ((s = dotc(c, dtype, rt, v, n, &rv, st)) != BEM_OK) return s;
            if (cabs2(rv) == 0.0) break;
            alpha = cdiv(rho_new, rv);
            const c128 malpha = mk<double>(-alpha.re, -alpha.im);
            CK(kv_lincomb(q, dtype, one, r, malpha, v, zero, nullptr, n, st));        // s = r - alpha v (in q)
            double sn;
            if ((s = norm_dev(c, dtype, q, n, &sn, st)) != BEM_OK) return s;
            ++it;
            if (sn <= tol_abs) {
                CK(kv_lincomb(x, dtype, one, x, alpha, p, zero, nullptr, n, st));
                CK(cudaMemcpyAsync(r, q, esize_of(dtype) * n, cudaMemcpyDeviceToDevice, st));
                rn = sn;
                break;
            }
            CK(A(q, t, adjoint));
            c128 ts, tt;
            if ((s = dotc(c, dtype, t, q, n, &ts, st)) != BEM_OK) return s;
            if ((s = dotc(c, dtype, t, t, n, &tt, st)) != BEM_OK) return s;
            if (tt.re == 0.0) break;
            omega = cdiv(ts, tt);
            CK(kv_lincomb(x, dtype, one, x, alpha, p, omega, q, n, st));              // x += alpha p + omega s
            const c128 momega = mk<double>(-omega.re, -omega.im);
            CK(kv_lincomb(r, dtype, one, q, momega, t, zero, nullptr, n, st));        // r = s - omega t
            rho = rho_new;
            if ((s = norm_dev(c, dtype, r, n, &rn, st)) != BEM_OK) return s;
        }
    } else {  // CGNR: CG on A^H A x = A^H b
        CK(A(r, u, !adjoint));  // z = A^H r (in u)
        CK(cudaMemcpyAsync(p, u, esize_of(dtype) * n, cudaMemcpyDeviceToDevice, st));
        double zn;
        if ((s = norm_dev(c, dtype, u, n, &zn, st)) != BEM_OK) return s;
        while (rn > tol_abs && it < maxit && zn > 0.0) {
            CK(A(p, w, adjoint));
            double wn;
            if ((s = norm_dev(c, dtype, w, n, &wn, st)) != BEM_OK) return s;
            if (wn == 0.0) break;
            const c128 alpha = mk<double>((zn * zn) / (wn * wn), 0.0);
            CK(kv_lincomb(x, dtype, one, x, alpha, p, zero, nullptr, n, st));
            CK(kv_lincomb(r, dtype, one, r, mk<double>(-alpha.re, 0.0), w, zero, nullptr, n, st));
            CK(A(r, u, !adjoint));
            double zn_new;
            if ((s = norm_dev(c, dtype, u, n, &zn_new, st)) != BEM_OK) return s;
            const c128 beta = mk<double>((zn_new * zn_new) / (zn * zn), 0.0);
            CK(kv_lincomb(p, dtype, one, u, beta, p, zero, nullptr, n, st));
            zn = zn_new;
            ++it;
            if ((s = norm_dev(c, dtype, r, n, &rn, st)) != BEM_OK) return s;
        }
    }
    *iters += it;
    *final_res = rn;
    return BEM_OK;
}

static bem_status solve_impl(bem_ctx* c, const void* b, void* x, int nrhs, void* stream, int* iters, double* relres,
                             bool adjoint) {
    if (!c) return BEM_EINVAL;
    if (!c->assembled) return fail(c, BEM_ESTATE, "bem_solve needs bem_assemble");
    if (nrhs < 1 || !b || !x) return fail(c, BEM_EINVAL, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    // the BF16-factor product has no adjoint form (nor does CGNR run on it)
    const bool bf_ok = !adjoint && c->opt.solver != BEM_SOLVER_CGNR && dtype_ok(c, BEM_C64_BF16F);
    const int din = bf_ok ? BEM_C64_BF16F : (op_built(c, 0) ? BEM_C64 : BEM_C128);
    const int vin = vec_dtype(din);
    const bool out128 = op_built(c, 1);
    const int dres = out128 ? BEM_C128 : DT_C64_IN_FP64;
    if (adjoint || c->opt.solver == BEM_SOLVER_CGNR) {
        bem_status s0;
        if ((s0 = ensure_adjoint_for(c, din, st)) != BEM_OK) return s0;
        if ((s0 = ensure_adjoint_for(c, dres, st)) != BEM_OK) return s0;
    }
    bem_status s;
    if (c->opt.solver == BEM_SOLVER_GMRES) {
        CK(ensure(c->d_one, sizeof(c128)));
        const c128 one1 = mk<double>(1, 0);
        CK(cudaMemcpyAsync(c->d_one.p, &one1, sizeof(c128), cudaMemcpyHostToDevice, st));
        return solve_gmres_batched(c, b, x, nrhs, st, iters, relres, adjoint, din, dres);
    }
    if (c->cal.built && !adjoint)
        return fail(c, BEM_EINVAL, "the Calderon preconditioner is applied by the GMRES solver only");
    if ((s = krylov_work(c, vin)) != BEM_OK) return s;
    const int64_t n = 2 * c->ne;
    DevBuf zr, rr;
    struct G {
        DevBuf* b[2];
        ~G() {
            for (DevBuf* x : b) dfree(*x);
        }
    } guard{{&zr, &rr}};
    CK(dalloc(zr, sizeof(c128) * n));
    CK(dalloc(rr, sizeof(c128) * n));
    CK(ensure(c->d_one, sizeof(c128)));
    c128 one = mk<double>(1, 0);
    CK(cudaMemcpyAsync(c->d_one.p, &one, sizeof(c128), cudaMemcpyHostToDevice, st));
    int total_it = 0;
    bool all_ok = true;
    for (int r = 0; r < nrhs; ++r) {
        const c128* br = (const c128*)b + r * n;
        c128* xr = (c128*)x + r * n;
        double bn;
        if ((s = norm_dev(c, BEM_C128, br, n, &bn, st)) != BEM_OK) return s;
        if (!std::isfinite(bn)) return fail(c, BEM_EINVAL, "the right-hand side has non-finite entries");
        if (bn == 0) {
            CK(cudaMemsetAsync(xr, 0, sizeof(c128) * n, st));
            if (relres) relres[r] = 0;
            continue;
        }
        const bool refine = c->opt.refine_tol > 0;
        const int steps = refine ? c->opt.refine_maxit : 1;
        double rel = 0;
        bool inner_ok = true;
        for (int step = 0;; ++step) {
            // r = b - Z x with the most accurate operator
            CK(matvec_any(c, dres, xr, zr.p, 1, st, false, adjoint));
            CK(kv_sub(br, zr.p, rr.p, BEM_C128, n, st));
            double rn;
            if ((s = norm_dev(c, BEM_C128, rr.p, n, &rn, st)) != BEM_OK) return s;
            rel = rn / bn;
            if (refine ? rel <= c->opt.refine_tol : step >= 1) break;
            if (step >= steps) break;
            // inner solve Z d = r
            if (vin == BEM_C64)
                CK(kv_cast<float>(rr.p, BEM_C128, (c64*)c->gw.rin.p, n, st));
            else
                CK(cudaMemcpyAsync(c->gw.rin.p, rr.p, sizeof(c128) * n, cudaMemcpyDeviceToDevice, st));
            double fres;
            int before = total_it;
            const double tin = refine ? std::max(c->opt.tol * rn, 0.5 * c->opt.refine_tol * bn) : c->opt.tol * rn;
            s = cg_family(c, din, c->opt.solver, tin, c->opt.maxit - total_it, &total_it, &fres, st,
                          adjoint);
            if (s != BEM_OK)
                return s;
            inner_ok = fres <= tin * 1.0000001;
            CK(kv_axpy_c128(xr, c->gw.xin.p, vin, (const c128*)c->d_one.p, 1.0, n, 1, n, st));
            if (total_it >= c->opt.maxit || total_it == before) {
                // out of iterations (or no progress possible): measure and stop
                CK(matvec_any(c, dres, xr, zr.p, 1, st, false, adjoint));
                CK(kv_sub(br, zr.p, rr.p, BEM_C128, n, st));
                if ((s = norm_dev(c, BEM_C128, rr.p, n, &rn, st)) != BEM_OK) return s;
                rel = rn / bn;
                break;
            }
        }
        if (relres) relres[r] = rel;
        bool ok = refine ? rel <= c->opt.refine_tol : inner_ok;
        all_ok = all_ok && ok;
    }
    CK(cudaStreamSynchronize(st));
    if (iters) *iters = total_it;
    if (!all_ok) return fail(c, BEM_ENOCONV, "solver did not reach its tolerance");
    return BEM_OK;
}

extern "C" bem_status bem_solve(bem_ctx* c, const void* b, void* x, int nrhs, void* stream, int* iters,
                                double* relres) {
    return solve_impl(c, b, x, nrhs, stream, iters, relres, false);
}

extern "C" bem_status bem_solve_adjoint(bem_ctx* c, const void* g, void* lambda, int nrhs, void* stream, int* iters,
                                        double* relres) {
    return solve_impl(c, g, lambda, nrhs, stream, iters, relres, true);
}

// ---------------------------------------------------------------------------
// powers
// ---------------------------------------------------------------------------
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(BEM_PI * (i + 0.75) / (n + 0.5));
        double dp = 1;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1, p1 = z;
            for (int j = 2; j <= n; ++j) {
                double p2 = ((2.0 * j - 1) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1 - z * z) * dp * dp);
    }
}

// The currents that radiate into region 0: x itself for one body; for a layered
// body a copy with every surface that does not bound region 0 zeroed (the power
// leaving region 0 -- absorbed, extinguished, scattered by the whole body --
// depends on those alone; region 0's boundary signs are all +1)
static bem_status exterior_view(bem_ctx* c, const void* x, int nrhs, const c128** out, cudaStream_t st) {
    if (!layered(c)) {
        *out = (const c128*)x;
        return BEM_OK;
    }
    const bem_ctx::Region& R = c->regions[0];
    const int64_t ns = (int64_t)R.edges.size();
    const size_t n = sizeof(c128) * 2 * c->ne * nrhs;
    CK(ensure(c->d_xext, n));
    CK(ensure(c->d_rx, sizeof(c128) * 2 * ns * nrhs));
    CK(cudaMemsetAsync(c->d_xext.p, 0, n, st));
    CK(region_gather(x, 16, c->ne, (const int*)R.d_edges.p, (const signed char*)R.d_sign.p, ns, nrhs, c->d_rx.p, st));
    CK(region_scatter_add(c->d_rx.p, 16, c->ne, (const int*)R.d_edges.p, (const signed char*)R.d_sign.p, ns, nrhs,
                          c->d_xext.p, st));
    *out = (const c128*)c->d_xext.p;
    return BEM_OK;
}

extern "C" bem_status bem_power(bem_ctx* c, const void* x, const void* b, int nrhs, double* p_abs, double* p_ext,
                                double* p_sca, void* stream) {
    if (!c) return BEM_EINVAL;
    if (!c->assembled) return fail(c, BEM_ESTATE, "bem_power needs bem_assemble");
    if (nrhs < 1 || !x || (p_ext && !b)) return fail(c, BEM_EINVAL, "bad arguments");
    if (nrhs > BEM_MAX_NRHS) return fail(c, BEM_EINVAL, nrhs_msg("bem_power", nrhs));
    cudaStream_t st = (cudaStream_t)stream;
    GeomDev g = geom_view(c);
    const c128* xe;
    bem_status s0;
    if ((s0 = exterior_view(c, x, nrhs, &xe, st)) != BEM_OK) return s0;
    const int nta = 64, nph = 128;
    int npa = (int)((c->nt + 255) / 256);
    size_t need = sizeof(double) * (size_t)nrhs * std::max(npa, std::max(NPART, nta * nph));
    CK(ensure(c->d_part, need));
    CK(ensure(c->d_red, sizeof(double) * nrhs));
    std::vector<double> host(nrhs);
    if (p_abs) {
        CK(power_abs(g, xe, nrhs, nullptr, (double*)c->d_part.p, npa, st));
        CK(kv_reduce_real((const double*)c->d_part.p, npa, nrhs, (double*)c->d_red.p, st));
        CK(cudaMemcpyAsync(p_abs, c->d_red.p, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
    }
    if (p_ext) {
        CK(dot_real_parts(xe, (const c128*)b, c->ne, nrhs, (double*)c->d_part.p, NPART, st));
        CK(kv_reduce_real((const double*)c->d_part.p, NPART, nrhs, (double*)c->d_red.p, st));
        CK(cudaMemcpyAsync(host.data(), c->d_red.p, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        memcpy(p_ext, host.data(), sizeof(double) * nrhs);
    }
    if (p_sca) {
        if (!c->d_gl.p) {
            std::vector<double> gx, gw;
            gauss_legendre(nta, gx, gw);
            gx.insert(gx.end(), gw.begin(), gw.end());
            CK(upload(c->d_gl, gx, st));
        }
        CK(ensure(c->d_far, power_sca_scratch(g, nrhs)));
        CK(power_sca(g, xe, nrhs, (double*)c->d_part.p, nta, nph, (const double*)c->d_gl.p,
                     (const double*)c->d_gl.p + nta, c->d_far.p, st));
        CK(kv_reduce_real((const double*)c->d_part.p, nta * nph, nrhs, (double*)c->d_red.p, st));
        CK(cudaMemcpyAsync(host.data(), c->d_red.p, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        memcpy(p_sca, host.data(), sizeof(double) * nrhs);
    }
    CK(cudaStreamSynchronize(st));
    return BEM_OK;
}

extern "C" bem_status bem_absorbed_power_gradient(bem_ctx* c, const void* x, void* g, int nrhs, void* stream) {
    if (!c) return BEM_EINVAL;
    if (!c->assembled) return fail(c, BEM_ESTATE, "bem_absorbed_power_gradient needs bem_assemble");
    if (nrhs < 1 || !x || !g || x == g) return fail(c, BEM_EINVAL, "bad arguments");
    if (nrhs > BEM_MAX_NRHS) return fail(c, BEM_EINVAL, nrhs_msg("bem_absorbed_power_gradient", nrhs));
    const c128* xe;
    bem_status s0;
    if ((s0 = exterior_view(c, x, nrhs, &xe, (cudaStream_t)stream)) != BEM_OK) return s0;
    CK(power_abs_grad(geom_view(c), xe, nrhs, (c128*)g, (cudaStream_t)stream));
    return BEM_OK;
}

extern "C" bem_status bem_grad_weights(bem_ctx* c, const void* bm, int nw, const bem_c128* w, double* p_abs,
                                       bem_c128* grad, void* x_out, void* lambda_out, void* stream, int* iters) {
    if (!c) return BEM_EINVAL;
    if (!c->assembled) return fail(c, BEM_ESTATE, "bem_grad_weights needs bem_assemble");
    if (nw < 1 || !bm || !w || !p_abs || !grad) return fail(c, BEM_EINVAL, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = 2 * c->ne;
    GeomDev gv = geom_view(c);
    DevBuf d_w, d_b, d_x, d_lam, d_g, d_part, d_red;
    struct G {
        DevBuf* b[7];
        ~G() {
            for (DevBuf* x : b) dfree(*x);
        }
    } guard{{&d_w, &d_b, &d_x, &d_lam, &d_g, &d_part, &d_red}};
    std::vector<c128> wh(nw);
    for (int i = 0; i < nw; ++i) wh[i] = mk<double>(w[i].re, w[i].im);
    CK(upload(d_w, wh, st));
    CK(dalloc(d_b, sizeof(c128) * n));
    CK(dalloc(d_g, sizeof(c128) * n));
    c128* x = (c128*)x_out;
    c128* lam = (c128*)lambda_out;
    if (!x) {
        CK(dalloc(d_x, sizeof(c128) * n));
        x = (c128*)d_x.p;
    }
    if (!lam) {
        CK(dalloc(d_lam, sizeof(c128) * n));
        lam = (c128*)d_lam.p;
    }
    // b = Bm w
    CK(cudaMemsetAsync(d_b.p, 0, sizeof(c128) * n, st));
    CK(kv_update(d_b.p, bm, BEM_C128, n, nw, (const c128*)d_w.p, 1.0, n, st));
    // x = Z^-1 b
    CK(cudaMemsetAsync(x, 0, sizeof(c128) * n, st));
    int it1 = 0, it2 = 0;
    double rr;
    bem_status s = solve_impl(c, d_b.p, x, 1, stream, &it1, &rr, false);
    if (s != BEM_OK) return s;
    // P = Re(xJ^H X xM)
    const int npa = (int)((c->nt + 255) / 256);
    CK(dalloc(d_part, sizeof(c128) * std::max<int64_t>(npa, (int64_t)NPART * nw)));
    CK(dalloc(d_red, sizeof(c128) * nw));
    const c128* xe;
    if ((s = exterior_view(c, x, 1, &xe, st)) != BEM_OK) return s;
    CK(power_abs(gv, xe, 1, nullptr, (double*)d_part.p, npa, st));
    CK(kv_reduce_real((const double*)d_part.p, npa, 1, (double*)d_red.p, st));
    CK(cudaMemcpyAsync(p_abs, d_red.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    // g = dP/dconj(x); Z^H lambda = g
    CK(power_abs_grad(gv, xe, 1, (c128*)d_g.p, st));
    CK(cudaMemsetAsync(lam, 0, sizeof(c128) * n, st));
    s = solve_impl(c, d_g.p, lam, 1, stream, &it2, &rr, true);
    if (s != BEM_OK) return s;
    // dP/dconj(w_i) = Bm_i^H lambda
    CK(kv_multidot(bm, BEM_C128, n, nw, lam, n, (c128*)d_part.p, NPART, st));
    CK(kv_reduce_partials((const c128*)d_part.p, NPART, nw, (c128*)d_red.p, st));
    std::vector<c128> gh(nw);
    CK(cudaMemcpyAsync(gh.data(), d_red.p, sizeof(c128) * nw, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int i = 0; i < nw; ++i) grad[i] = {gh[i].re, gh[i].im};
    if (iters) *iters = it1 + it2;
    return BEM_OK;
}

// dP/d eps_r of one body's interior medium (the k1 slot), from x and lambda
static bem_status grad_eps_one(bem_ctx* c, const void* x, const void* lambda, double* dp, cudaStream_t st) {
    const int64_t nsing = c->n_sing;
    DevBuf d_pair_a, d_dvals, d_part, d_out;
    struct G {
        DevBuf* b[4];
        ~G() {
            for (DevBuf* z : b) dfree(*z);
        }
    } guard{{&d_pair_a, &d_dvals, &d_part, &d_out}};
    // k-derivatives of the singular-pair tables at k1
    std::vector<int> ptr(c->nt + 1);
    CK(cudaMemcpyAsync(ptr.data(), c->d_sing_ptr.p, sizeof(int) * (c->nt + 1), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    std::vector<int> pa(std::max<int64_t>(1, nsing));
    for (int64_t t = 0; t < c->nt; ++t)
        for (int k = ptr[t]; k < ptr[t + 1]; ++k) pa[k] = (int)t;
    CK(upload(d_pair_a, pa, st));
    CK(dalloc(d_dvals, sizeof(c128) * 18 * std::max<int64_t>(1, nsing)));
    GeomDev g = geom_view(c);
    CK(singular_dvalues(g, (int)nsing, (const int*)d_pair_a.p, (c128*)d_dvals.p, st));
    CK(dalloc(d_part, sizeof(c128) * 6 * c->nt));
    CK(dalloc(d_out, sizeof(c128) * 6));
    CK(interior_forms(g, (const c128*)d_dvals.p, (const c128*)x, (const c128*)lambda, (c128*)d_part.p,
                      (c128*)d_out.p, st));
    c128 f[6];
    CK(cudaMemcpyAsync(f, d_out.p, sizeof(f), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    // dZ/d eps_r applied between lambda and x: k1' = k1 / (2 eps_r), eta_r' = -eta_r / (2 eps_r),
    // dA = eta_r' T1 + eta_r k1' T1', dB = k1' K1', dC = k1' T1' / eta_r - (eta_r' / eta_r^2) T1
    const c128 two_eps = 2.0 * c->eps;
    const c128 dk1 = cdiv(c->k1, two_eps);
    const c128 der = cdiv(mk<double>(-c->eta_r.re, -c->eta_r.im), two_eps);
    const c128 s = der * f[0] + (c->eta_r * dk1) * f[2] + dk1 * (f[4] - f[5]) + cdiv(dk1, c->eta_r) * f[3] -
                   cdiv(der, c->eta_r * c->eta_r) * f[1];
    // dP = -2 Re(lambda^H dZ x), dZ = (dZ/d eps_r) d eps_r, d eps_r = d eps' + j d eps''
    dp[0] = -2.0 * s.re;
    dp[1] = 2.0 * s.im;
    return BEM_OK;
}

extern "C" int bem_num_regions(const bem_ctx* c) {
    if (!c || !c->has_media) return -1;
    return layered(c) ? (int)c->regions.size() : 2;
}

extern "C" bem_status bem_grad_eps(bem_ctx* c, const void* x, const void* lambda, double* dp, void* stream) {
    if (!c) return BEM_EINVAL;
    if (!c->assembled) return fail(c, BEM_ESTATE, "bem_grad_eps needs bem_assemble");
    if (!x || !lambda || !dp) return fail(c, BEM_EINVAL, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    if (!layered(c)) return grad_eps_one(c, x, lambda, dp, st);
    // layered body: only Z_r depends on eps_r, so lambda^H Q_r^T (dZ_r/d eps_r) Q_r x is
    // region r's single-medium form between its signed boundary currents
    int64_t nmax = 0;
    for (const auto& R : c->regions) nmax = std::max<int64_t>(nmax, (int64_t)R.edges.size());
    DevBuf xr, lr;
    struct G {
        DevBuf* b[2];
        ~G() {
            for (DevBuf* z : b) dfree(*z);
        }
    } guard{{&xr, &lr}};
    CK(dalloc(xr, sizeof(c128) * 2 * nmax));
    CK(dalloc(lr, sizeof(c128) * 2 * nmax));
    for (size_t r = 1; r < c->regions.size(); ++r) {
        bem_ctx::Region& R = c->regions[r];
        const int64_t ns = (int64_t)R.edges.size();
        const int* ed = (const int*)R.d_edges.p;
        const signed char* sg = (const signed char*)R.d_sign.p;
        CK(region_gather(x, 16, c->ne, ed, sg, ns, 1, xr.p, st));
        CK(region_gather(lambda, 16, c->ne, ed, sg, ns, 1, lr.p, st));
        bem_status s = grad_eps_one(R.sub, xr.p, lr.p, dp + 2 * (r - 1), st);
        if (s != BEM_OK) return fail(c, s, "region " + std::to_string(r) + ": " + R.sub->err);
    }
    return BEM_OK;
}

extern "C" bem_status bem_power_density(bem_ctx* c, const void* x, double* per_tri, void* stream) {
    if (!c) return BEM_EINVAL;
    if (!c->assembled) return fail(c, BEM_ESTATE, "bem_power_density needs bem_assemble");
    if (!x || !per_tri) return fail(c, BEM_EINVAL, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    GeomDev g = geom_view(c);
    int npa = (int)((c->nt + 255) / 256);
    CK(ensure(c->d_part, sizeof(double) * std::max(npa, NPART)));
    const c128* xe;
    bem_status s0;
    if ((s0 = exterior_view(c, x, 1, &xe, st)) != BEM_OK) return s0;
    CK(power_abs(g, xe, 1, per_tri, (double*)c->d_part.p, npa, st));
    return BEM_OK;
}

// ---------------------------------------------------------------------------
// accessors for the fixed-scratch entry point (static_scratch.cu)
// ---------------------------------------------------------------------------
GeomDev bem_geom_view_for_static(const bem_ctx* c) { return geom_view(c); }
bool bem_ctx_has_geometry(const bem_ctx* c) { return c->assembled; }
bool bem_ctx_is_layered(const bem_ctx* c) { return layered(c); }
void bem_ctx_set_error(bem_ctx* c, const char* msg) { c->err = msg; }
