// Internal definitions shared by the libbem translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/bem.h"

#define BEM_PI 3.14159265358979323846
#define BEM_MAX_LEAF 64
// storage/arithmetic forms of a product (matvec_run)
#define BEM_FORM_NATIVE 0       // entries and factors stored in the product's arithmetic
#define BEM_FORM_BF16F 1        // complex64 product, far factors stored as BF16
#define BEM_FORM_C64_IN_FP64 2  // complex64 entries and factors, FP64 vectors and sums
// ACA tasks whose scratch (m + n) * rank cap reaches this many elements get a whole
// SM (1024 threads) in the FP32 build
#define BEM_ACA_WIDE_COST (1 << 19)
#define BEM_MAX_NR 8   // right-hand sides applied per pass over the operator
#define BEM_MAX_NRHS 65535  // right-hand sides per call of an entry point that launches one grid row per vector
#define BEM_ROW_GROUPS 1     // 64-thread groups per CTA of the rows kernel (one work slot each)
#define BEM_ROW_TARGET_CTAS (48 * 152)  // rows-kernel CTAs aimed at per product (about 3 waves)
#define BEM_TC_NR 64                   // right-hand sides per pass of the tensor-core product
#define BEM_TC_MIN_RHS 16              // batched solves of at least this many right-hand sides use it
#define BEM_TC_ROW_TARGET (4 * 152)     // work slots of the tensor-core rows kernel (persistent CTAs take them in turn)

// ---------------------------------------------------------------------------
// complex arithmetic on interleaved (re, im) pairs
// ---------------------------------------------------------------------------
template <typename R>
struct cx {
    R re, im;
};

template <typename R>
__host__ __device__ __forceinline__ cx<R> mk(R a, R b) {
    cx<R> z;
    z.re = a;
    z.im = b;
    return z;
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return mk<R>(a.re + b.re, a.im + b.im); }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return mk<R>(a.re - b.re, a.im - b.im); }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
    return mk<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return mk<R>(s * a.re, s * a.im); }
template <typename R>
__host__ __device__ __forceinline__ cx<R> cconj(cx<R> a) { return mk<R>(a.re, -a.im); }
template <typename R>
__host__ __device__ __forceinline__ R cabs2(cx<R> a) { return a.re * a.re + a.im * a.im; }
template <typename R>
__host__ __device__ __forceinline__ cx<R> cdiv(cx<R> a, cx<R> b) {
    R d = b.re * b.re + b.im * b.im;
    return mk<R>((a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d);
}
// a += b * c
template <typename R>
__host__ __device__ __forceinline__ void cfma(cx<R>& a, cx<R> b, cx<R> c) {
    a.re += b.re * c.re - b.im * c.im;
    a.im += b.re * c.im + b.im * c.re;
}
// a += conj(b) * c
template <typename R>
__host__ __device__ __forceinline__ void cfma_conj(cx<R>& a, cx<R> b, cx<R> c) {
    a.re += b.re * c.re + b.im * c.im;
    a.im += b.re * c.im - b.im * c.re;
}

typedef cx<float> c64;
typedef cx<double> c128;

// A complex value stored as two BF16 numbers (real part in the low 16 bits of the
// 32-bit word).  A BF16 number is the upper half of an IEEE binary32, so widening
// is a shift; narrowing rounds to nearest even.
struct __align__(4) bf16c {
    __nv_bfloat16 re, im;
};
__device__ __forceinline__ float2 bf16c_to_float2(unsigned int w) {
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
__device__ __forceinline__ bf16c float2_to_bf16c(float re, float im) {
    bf16c r;
    r.re = __float2bfloat16_rn(re);
    r.im = __float2bfloat16_rn(im);
    return r;
}

// ---------------------------------------------------------------------------
// device view of the mesh, media and singular-pair table
// ---------------------------------------------------------------------------
// Constants of the two media in the arithmetic of one precision (computed on the
// host in FP64, so the quadrature kernels do no FP64 work in their FP32 build).
template <typename R>
struct MediaConst {
    R k0, k1r, k1i;          // wavenumbers (k1 = k1r + j k1i, k1i <= 0)
    cx<R> jk0, jk1;          // j k0, j k1
    cx<R> jok0, jok1;        // j / k0, j / k1
    cx<R> er, ie;            // eta_r = eta1 / eta0 and 1 / eta_r
    R w0;                    // 1: both media (one body); 0: the k1 medium alone (a region of a layered body)
};

// One triangle for the FP32 quadrature: the centroid split into a high and a low
// float (centroid differences keep ~48 bits), the vertices relative to the
// centroid, the signed edge coefficients and 1 / area.
struct TriF {
    float4 c_hi;  // x, y, z high parts; w = area
    float4 c_lo;  // x, y, z low parts; w = longest edge
    float4 v[3];  // vertex - centroid; w = 0
    float4 coef;  // tri_coef[0..2]; w = 1 / area
};

struct GeomDev {
    int nt, ne;
    const TriF* trif;        // nt FP32 triangle records
    const double* tv;        // nt x 9: vertices v0, v1, v2 of each triangle
    const double* area;      // nt
    const double* nrm;       // nt x 3 unit outward normal
    const double* cen;       // nt x 3 centroid ((v0 + v1) + v2) / 3
    const double* diam;      // nt longest edge
    const int* tvid;         // nt x 3 vertex indices
    const int* tri_edge;     // nt x 3 edge opposite local vertex i
    const double* tri_coef;  // nt x 3 s_i * l_i (sign +1 on T+, -1 on T-, times edge length)
    const int* edge_tri;     // ne x 2 (T+, T-)
    const int* edge_loc;     // ne x 2 local index of the free vertex in T+, T-
    // singular pairs: CSR by test triangle, partners sorted ascending
    const int* sing_ptr;     // nt + 1
    const int* sing_b;       // partner triangle
    const c128* sing_val;    // per pair 36 complex: T^0[3][3], K0[3][3], T^1[3][3], K1[3][3]
    // media
    double k0;
    c128 k1;
    c128 eta_r;
    MediaConst<float> mf;
    MediaConst<double> md;
};

template <typename R>
__device__ __forceinline__ const MediaConst<R>& media(const GeomDev& g);
template <>
__device__ __forceinline__ const MediaConst<float>& media<float>(const GeomDev& g) {
    return g.mf;
}
template <>
__device__ __forceinline__ const MediaConst<double>& media<double>(const GeomDev& g) {
    return g.md;
}

// Block descriptors (tree positions)
struct BlockDesc {
    int r0, m, c0, n;
};

// Far block record used by the product kernels
struct FarRec {
    int r0, m, c0, n;
    int rk[3];          // ranks of A, B, C (padded to even in storage)
    int64_t off_u[3];   // offset (in complex elements) of U of A, B, C
    int64_t off_v[3];   // offset of V-bar (the conjugate of V) of A, B, C
    int64_t off_t;      // offset of this block's t values: [tA | tB(J) | tB(M) | tC], each padded rank
};

// Kernel-side launch helpers implemented in the .cu files
namespace bem {

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

cudaError_t dalloc(DevBuf& b, size_t bytes);
void dfree(DevBuf& b);

// tree.cu
cudaError_t tree_bbox_level(const double* pts, const int64_t* perm, const int* lo, const int* hi, int ncl,
                            double* bbmin, double* bbmax, cudaStream_t st);
cudaError_t tree_split_level(const double* pts, const int64_t* perm_in, int64_t* perm_out, const int* lo,
                             const int* hi, const double* bbmin, const double* bbmax, const int* split_cl,
                             int nsplit, const int* pos_cl, int npos_total, cudaStream_t st);
cudaError_t tree_block_level(const int* cand, int ncand, const int* nlo, const int* nhi, const int* child0,
                             const double* bbmin, const double* bbmax, double eta, int* kind, int* counts,
                             cudaStream_t st);
cudaError_t tree_block_emit(const int* cand, int ncand, const int* kind, const int* child0, const int* offs,
                            int* next_cand, int* near_out, int* far_out, const int* nlo, const int* nhi,
                            cudaStream_t st);
cudaError_t scan_exclusive(const int* in, int* out, int n, int* total_dev, cudaStream_t st);

// singular.cu
// Uniform grid of triangle centroids with cells no smaller than twice the longest
// edge of the mesh: every singular partner of a triangle lies in its own or an
// adjacent cell.
struct SingGrid {
    int nx, ny, nz;
    const int* cell_start;  // nx ny nz + 1
    const int* cell_tri;    // triangles sorted by cell
    const int* tri_cell;    // nt: cell of each triangle
};
cudaError_t singular_count(GeomDev g, SingGrid G, int* counts, cudaStream_t st);
cudaError_t singular_fill(GeomDev g, SingGrid G, const int* ptr, int* partners, cudaStream_t st);
cudaError_t singular_values(GeomDev g, int npairs, const int* pair_a, c128* vals, cudaStream_t st);
// k-derivatives (k = k1) of the singular-pair tables: 18 complex per pair, dT^_1 then dK_1
cudaError_t singular_dvalues(GeomDev g, int npairs, const int* pair_a, c128* dvals, cudaStream_t st);
// Bilinear forms of the interior operators for the permittivity gradient, summed
// over all triangle pairs (FP64, O(nt^2)): out[6] = {lJ^H T1 xJ, lM^H T1 xM,
// lJ^H T1' xJ, lM^H T1' xM, lJ^H K1' xM, lM^H K1' xJ} (' = d/dk at k1)
cudaError_t interior_forms(GeomDev g, const c128* dvals, const c128* x, const c128* lam, c128* partial, c128* out,
                           cudaStream_t st);

// assemble.cu
template <typename R>
cudaError_t near_assemble(GeomDev g, const int64_t* perm, const BlockDesc* blocks, const int64_t* entry_off,
                          int nblocks, cx<R>* entries, int64_t op_stride, cudaStream_t st);
template <typename R>
cudaError_t eval_entries(GeomDev g, const int* rows, const int* cols, int64_t count, cx<R>* out,
                         cudaStream_t st);
struct AcaTask {
    int r0, m, c0, n;
    int op;             // 0 = A, 1 = B, 2 = C
    int rmax;
    int64_t scratch;    // offset of this task's scratch (complex elements)
};
template <typename R>
cudaError_t aca_run(GeomDev g, const int64_t* perm, const AcaTask* tasks, const int counts[6], cx<R>* scratch,
                    double tol, int* ranks, int* flags, cudaStream_t st, int max_m);
// SVD recompression of converged ACA tasks in their scratch (recompress.cu): ranks
// updated in place; ws holds 2 k^2 values per task at ws_off (k its ACA rank);
// tasks with k above recompress_kmax<R>() keep their factors
template <typename R>
int recompress_kmax();
template <typename R>
cudaError_t aca_recompress(const AcaTask* tasks, int ntasks, cx<R>* scratch, int* ranks, const int* flags,
                           double tol, cx<R>* ws, const int64_t* ws_off, cudaStream_t st);
// U is written slice-major (leaf slices of the block rows), W column-pair-major
template <typename R>
cudaError_t aca_compact(const AcaTask* tasks, int ntasks, const cx<R>* scratch, const int* ranks,
                        const int64_t* off_u, const int64_t* off_v, cx<R>* arena, const int* pos_leaf_lo,
                        const int* pos_leaf_m, cudaStream_t st);

// matvec.cu
// One far piece of the rows kernel (a leaf's rows of one factored block): the
// complex offsets in the arena of the three factor slices it streams (U slices in
// the forward product, W rows in the adjoint), their pair stride, the column-pair
// counts of A, B, C and the offset of the block's t values, so that a piece costs
// one 48-byte descriptor load instead of a chain of lookups.
struct __align__(16) PieceDesc {
    int64_t base[3];
    int64_t t_off;
    int kp[3];
    int ld;
};

struct MatvecPlan {
    int ne, nleaf, nfar;
    int nslot;                   // CTAs of the rows kernel (work slots)
    int pmax;                    // largest number of slots of one leaf
    const int64_t* perm;         // tree position -> edge
    const int* leaf_r0;          // nleaf
    const int* leaf_m;           // nleaf
    const int* leaf_parts;       // nleaf: slots of each leaf
    const int* slot_order;       // nslot: slot handled by CTA b, heaviest slot first
    const int* slot_leaf;        // nslot
    const int* slot_part;        // nslot: index of the slot within its leaf
    const int* work_ptr;         // nslot + 1: work slot -> range of work_item
    const int* work_item;        // >= 0: dense item; < 0: far piece -1 - item
    const int* near_c0;          // per dense item: column start
    const int* near_n;           // per dense item: columns
    const int64_t* near_off;     // per dense item: offset (complex elements) of its A entries
    int64_t near_op_stride;      // distance between the A, B, C arrays
    const PieceDesc* pieces;     // per far piece: factor bases, strides, ranks and t offset
    const FarRec* far;           // nfar
    const int2* vhx_units;       // nvhx units of the V^H x kernel: (far block, group of 8 items), largest first
    int nvhx;
    const int* pos_leaf_lo;      // ne: first tree position of each position's leaf (adjoint U^T x pass)
    const int* pos_leaf_m;       // ne: size of each position's leaf
    void* ypart;                 // pmax x 2ne partial rows (pmax > 1)
    unsigned int* arrive;        // nleaf arrival counters, zero between products
};
// Tensor-core product (matvec_tc.cu).  V^H x work: a task is up to 32 column pairs
// of W (two ranks each) of the far blocks sharing one column cluster, all applied
// to the same half (J or M) of the vectors.
struct TcPair {
    int64_t w;     // complex offset in the arena of the pair's W column pair (pair (kp, j) at w + 2 j)
    int64_t trow;  // t row of the pair's first rank (the second follows)
};
struct TcVhxTask {
    int c0, n;       // column cluster (tree positions)
    int g;           // 0: x_J, 1: x_M
    int npairs;      // 1..32
    int pair0;       // first entry in the pair list
    int pad;
    int64_t wcopy;   // float4 offset of the task's W copy: chunk c, column j, pair p at wcopy + (32 c + j) 32 + p
};
// One work item of the tensor-core rows kernel, in the order a CTA processes them
// (the items of each of its slots, then an end record)
struct __align__(16) TcRec {
    int64_t base[3];   // complex offsets of the operator parts A, B, C (dense entries, or the arena for far pieces)
    int64_t vec;       // dense item: first column (tree position); far piece: t row of its t_A
    int npair[3];      // column (rank) pairs per part
    int ld;            // pair stride (rows of the leaf)
    int n;             // dense item: columns
    int kind;          // 0 dense item, 1 far piece, 2 end of slot
    int pad[2];
};
struct TcPlan {
    const TcVhxTask* tasks;   // grouped by CTA: CTA b takes [vcta_ptr[b], vcta_ptr[b + 1])
    const TcPair* pairs;
    int ntask;
    int nsm;                  // persistent CTAs (one per SM)
    const int* vcta_ptr;      // nsm + 1
    const float4* wcopy;      // task-major copy of the W factors (see TcVhxTask::wcopy)
    const int* cta_slot_ptr;  // nsm + 1: rows slots of CTA b at cta_slots[cta_slot_ptr[b] ..]
    const int* cta_slots;
    const int* cta_rec_ptr;   // nsm + 1: item records of CTA b
    const TcRec* recs;
    c64* xp;                  // 2ne x 64 vectors, tree order
    c64* t;                   // t_len x 64
    c64* ypart;               // pmax x 64 x 2ne partial rows (tree order)
    int* err;                 // device-visible flag, 1 after a bounded wait ran out
};
// task-major copy of the W factors of the V^H x tasks
cudaError_t tc_build_wcopy(const TcVhxTask* tasks, int ntask, const TcPair* pairs, const c64* arena, float4* wcopy,
                           cudaStream_t st);
// y = Z x for nrhs complex64 vectors in passes of 64 (rows schedule p, complex64
// entries and factors); ev: NULL, or 6 events per pass as for matvec_run
cudaError_t matvec_tc_run(const MatvecPlan& p, const TcPlan& tp, const void* near, const void* arena, const c64* x,
                          c64* y, int nrhs, cudaStream_t st, const cudaEvent_t* ev);

// ev: NULL, or 6 events per right-hand side recorded around the three kernels
template <typename R>
cudaError_t matvec_run(const MatvecPlan& p, const void* near_entries, const void* arena, const cx<R>* x,
                       cx<R>* y, cx<R>* xp, cx<R>* t, int nrhs, int64_t t_len, cudaStream_t st,
                       const cudaEvent_t* ev, int form = BEM_FORM_NATIVE, bool adjoint = false);
// Transposed copy of the dense items (adjoint product); layouts as k_transpose_items
template <typename R>
cudaError_t transpose_items(const BlockDesc* items, const int64_t* offF, const int64_t* offT, int nitems,
                            const cx<R>* near, int64_t strideF, cx<R>* nearT, int64_t strideT, cudaStream_t st);
// BF16 copy of n complex64 factor values
cudaError_t factors_to_bf16(const c64* in, bf16c* out, int64_t n, cudaStream_t st);

// rhs_power.cu
template <typename R>
cudaError_t rhs_planewave(GeomDev g, const double* khat, const c128* e0, int nrhs, cx<R>* b, cudaStream_t st);
cudaError_t power_abs(GeomDev g, const c128* x, int nrhs, double* per_tri, double* partial, int npart,
                      cudaStream_t st);
// out = d P_abs / d conj(x) = (1/2) [X xM ; X^T xJ] (device complex128, 2ne x nrhs)
cudaError_t power_abs_grad(GeomDev g, const c128* x, int nrhs, c128* out, cudaStream_t st);
#define PSCA_CHUNK 16  // right-hand sides per pass of the scattered-power kernels (bounds their scratch)
size_t power_sca_scratch(GeomDev g, int nrhs);
cudaError_t power_sca(GeomDev g, const c128* x, int nrhs, double* partial, int ntheta, int nphi,
                      const double* ct, const double* wt, void* scratch, cudaStream_t st);
cudaError_t dot_real_parts(const c128* a, const c128* b, int64_t n, int nrhs, double* partial, int npart,
                           cudaStream_t st);

// krylov.cu
template <typename R>
cudaError_t kv_cast(const void* src, int src_dtype, cx<R>* dst, int64_t n, cudaStream_t st);
cudaError_t kv_multidot(const void* V, int dtype, int64_t ld, int k, const void* w, int64_t n, c128* out_partial,
                        int npart, cudaStream_t st);
cudaError_t kv_reduce_partials(const c128* partial, int npart, int count, c128* out, cudaStream_t st);
cudaError_t kv_reduce_real(const double* partial, int npart, int count, double* out, cudaStream_t st);
cudaError_t kv_update(void* w, const void* V, int dtype, int64_t ld, int k, const c128* h, double sign, int64_t n,
                      cudaStream_t st);
cudaError_t kv_norm2(const void* w, int dtype, int64_t n, double* out_partial, int npart, cudaStream_t st);
cudaError_t kv_axpy_c128(c128* y, const void* x, int dtype, const c128* coef, double sign, int64_t n, int k,
                         int64_t ld, cudaStream_t st);
cudaError_t kv_sub(const void* b, const void* zx, void* r, int dtype, int64_t n, cudaStream_t st);
// z = a x + b y + c w (null operands skipped; z may alias them)
cudaError_t kv_lincomb(void* z, int dtype, c128 a, const void* x, c128 b, const void* y, c128 c, const void* w,
                       int64_t n, cudaStream_t st);

// Batched GMRES on the device (gmres.cu).  Per right-hand side r (nrhs of them,
// vectors n long, column r at offset r n of each block): basis V = (m + 1) blocks of
// nrhs vectors, slot j + 1 receiving Z v_j.  The Hessenberg state is in the
// vectors' precision R (cx<R> unless noted): H (m + 1) x m row-major, g (m + 1),
// rotation cosines cs (m, real R) and sines sn (m), pass results h1, h2 (m + 1),
// y (m); state bits below.
#define BGS_ACTIVE 1
#define BGS_REORTH 2
#define BGS_MISS_SHIFT 8  // bits 8..15 of the state: cycles in a row whose residual did not follow its estimate
struct BgsArgs {
    void* V;            // (m + 1) x nrhs x n vectors (complex64 or complex128)
    void* x;            // nrhs x n: the cycle corrections accumulate here
    const void* b;      // nrhs x n: right-hand sides of the inner system
    int64_t n;
    int nrhs, m, chunk, nblk, maxit;
    void *H, *g, *cs, *sn, *h1, *h2, *y;
    c128* part;         // nrhs x (m + 2) x nblk partial inner products (FP64)
    double *wn0, *wn1, *wn2, *beta, *tol, *scale, *res, *npart;  // npart: nrhs x nblk partial norms
    int *state, *kk, *it;
    unsigned* cnt;      // nrhs arrival counters (zero between launches)
    int* host_active;   // host-mapped: right-hand sides still iterating
};
// CTA rows and CTAs per right-hand side for vectors of n complex values of esize bytes
void bgs_layout(int64_t n, int nrhs, int esize, int* chunk, int* nblk);
template <typename R>
cudaError_t bgs_iteration(const BgsArgs& a, int j, cudaStream_t st);
template <typename R>
cudaError_t bgs_cycle_start(const BgsArgs& a, bool x_zero, cudaStream_t st);
template <typename R>
cudaError_t bgs_cycle_end(const BgsArgs& a, cudaStream_t st);
// out[r] = |v_r|^2 (FP64 sums) for k columns of n complex64 (fp64: complex128)
// values; npart holds k x npart_cap partials (at least the nblk of bgs_layout for
// this element size, else cudaErrorInvalidValue), cnt k zeroed counters
cudaError_t col_norms2(const void* v, bool fp64, int64_t n, int k, double* npart, int npart_cap, unsigned* cnt,
                       double* out, cudaStream_t st);
// layered bodies: xs = sign * x[edges] (both halves [J ; M] of every column) and
// y[edges] += sign * ys; esize 8 (complex64) or 16 (complex128); edges distinct
cudaError_t region_gather(const void* x, int esize, int64_t ne, const int* edges, const signed char* sign,
                          int64_t ns, int nrhs, void* xs, cudaStream_t st);
cudaError_t region_scatter_add(const void* ys, int esize, int64_t ne, const int* edges, const signed char* sign,
                               int64_t ns, int nrhs, void* y, cudaStream_t st);


// ---------------------------------------------------------------------------
// Calderon preconditioner (calderon.cu): Buffa-Christiansen functions on the
// barycentric refinement, their mixed Gram matrix and its Chebyshev inverse
// ---------------------------------------------------------------------------
struct MeshTables {  // host views of a mesh and its RWG table (bem_set_mesh conventions)
    int64_t nv = 0, nt = 0, ne = 0;
    const double* verts = nullptr;    // nv x 3
    const int* tris = nullptr;        // nt x 3, outward (counter-clockwise) order
    const int* edge_v = nullptr;      // ne x 2, lexicographic (lo, hi)
    const int* edge_tri = nullptr;    // ne x 2: T+, T-
    const int* edge_loc = nullptr;    // ne x 2: corner of the free vertex in T+, T-
    const int* tri_edge = nullptr;    // nt x 3: edge opposite corner i
    const double* tri_coef = nullptr; // nt x 3: +l on T+, -l on T-
    const double* area = nullptr;     // nt
    const double* nrm = nullptr;      // nt x 3 unit outward normals
};
namespace cald {
struct Csr {  // compressed sparse rows, FP64 values
    int64_t rows = 0, cols = 0;
    std::vector<int> ptr, col;
    std::vector<double> val;
};
struct ChebPlan {  // fixed Chebyshev iteration for D^-1 A x = D^-1 b, eigenvalues in [lmin, lmax]
    double lmin = 0, lmax = 0, theta = 0;
    int steps = 0;                 // updates of x
    std::vector<double> c1, c2;    // d_{k+1} = c1[k] d_k + c2[k] r_{k+1}
    double reduction = 0;          // residual reduction measured on the host at plan time
};
void refine(const MeshTables& c, std::vector<double>& fverts, std::vector<int>& ftris);
bool bc_matrix(const MeshTables& c, const MeshTables& f, Csr& C, std::string& err);
Csr transpose(const Csr& a);
void mixed_gram(const MeshTables& c, const MeshTables& f, const Csr& C, Csr& G);
bool chebyshev_plan(const Csr& G, double target, int max_steps, ChebPlan& plan, std::string& err);
// y_b = scale * A x_b for nblk blocks (x_b = x + b * xs, y_b = y + b * ys, complex R)
template <typename R>
cudaError_t csr_apply(const int* ptr, const int* col, const R* val, int64_t rows, const cx<R>* x, int64_t xs,
                      cx<R>* y, int64_t ys, int nblk, R scale, cudaStream_t st);
// x_b ~ A^-1 b_b for nblk blocks of n (stride n) by the plan's fixed Chebyshev steps;
// dinv = 1 / diag(A); r, d0, d1: work of nblk * n values each
template <typename R>
cudaError_t chebyshev_solve(const int* ptr, const int* col, const R* val, const R* dinv, int64_t n,
                            const ChebPlan& p, const cx<R>* b, cx<R>* x, cx<R>* r, cx<R>* d0, cx<R>* d1, int nblk,
                            cudaStream_t st);
}  // namespace cald
}  // namespace bem

#define BEM_CUDA_TRY(expr)                      \
    do {                                        \
        cudaError_t _e = (expr);                \
        if (_e != cudaSuccess) return _e;       \
    } while (0)
