/*
 * bem.h -- C interface of libbem, a GB300 (sm_103a) boundary-element library for
 * the compressed matrix-vector product of the PMCHWT surface-integral operator of
 * a penetrable (lossy dielectric) body, and the solve and dosimetry built on it.
 *
 * Problem statement (arXiv:2310.15644).  A body with boundary Gamma in free space
 * (Sec. II) is illuminated by an incident field; its equivalent surface currents
 * j (electric) and m (magnetic) satisfy the PMCHWT system of Eq. 7 (rows 2-3),
 * discretised by Galerkin testing with piecewise-linear bases (Sec. III, Eq. 8 and
 * the matrices P11..P22 after it).  The library works in three dimensions with
 * RWG bases on a closed triangle mesh and the kernel e^{-jkR}/(4 pi R) under the
 * e^{+j w t} convention (the paper's H0^(2) kernel and 1 + j w tau Debye terms of
 * Eq. 6 fix that convention).  The interior medium has a complex relative
 * permittivity (Eq. 6 gives the skin model) and the outputs are the currents and
 * the absorbed power, the dosimetric quantity the paper is after (Sec. I).
 *
 * Unknowns and scaling.  For a mesh with ne interior edges the unknown vector has
 * 2*ne complex entries x = [eta0*J ; M] (J, M the RWG coefficients of j and m, in
 * the edge order returned by bem_edges), and the operator is
 *
 *     Z = [[ T0 + eta_r T1 ,  K0 + K1       ],
 *          [ -(K0 + K1)    ,  T0 + T1/eta_r ]],      eta_r = eta1/eta0,
 *
 *     Tk[m,n] = jk <f_m, G_k f_n> - (j/k) <div f_m, G_k div f_n>,
 *     Kk[m,n] = p.v. <f_m, grad G_k x f_n>,
 *
 * i.e. the paper's P11 = sum of single layers at k0 and k1, P12 = sum of double
 * layers, P21 = minus that sum, P22 = sum of the dual single layers, with the
 * impedances scaled out.  The right-hand side is b = [e ; eta0*h] with
 * e_m = <f_m, E_inc>, h_m = <f_m, H_inc> (the tested fields after Eq. 8).
 *
 * Compression.  Edges are ordered by a cluster tree over their midpoints; blocks of
 * the operator whose clusters are well separated are stored as low-rank factors
 * U V^H computed by adaptive cross approximation (the skeleton U V^T of Eq. 17),
 * the other blocks densely.
 *
 * Conventions for every entry point:
 *   - Returns a bem_status and never aborts, throws or exits.  On failure the
 *     message is available from bem_last_error(ctx).
 *   - "host" pointers are read (or written) before the call returns; the library
 *     keeps its own copies.  "device" pointers are caller-owned CUDA device memory,
 *     accessed asynchronously on the caller's stream (a cudaStream_t passed as
 *     void*; NULL means the legacy default stream).
 *   - Complex data are interleaved (re, im) pairs: complex64 = 2 x float,
 *     complex128 = 2 x double.  Several right-hand sides are stored column-major:
 *     element (i, r) of a 2*ne x nrhs array is at index i + r * 2*ne.
 *   - Calls out of order (e.g. bem_matvec before bem_assemble) return BEM_ESTATE.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef BEM_H
#define BEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bem_ctx bem_ctx;

typedef struct {
    double re, im;
} bem_c128;

typedef enum {
    BEM_OK = 0,
    BEM_EINVAL = 1,    /* invalid argument or mesh */
    BEM_ENOMEM = 2,    /* device or host allocation failed */
    BEM_ECUDA = 3,     /* a CUDA call failed (message holds cudaGetErrorString) */
    BEM_ENOCONV = 4,   /* iterative solver did not reach its tolerance; x holds the last iterate */
    BEM_ETIMEOUT = 5,  /* a bounded device wait gave up */
    BEM_ESTATE = 6     /* call made in the wrong order */
} bem_status;

/* Precision of the stored operator (bit mask for bem_options.precision). */
#define BEM_PREC_C64 1   /* near entries and factors in complex64, FP32 arithmetic */
#define BEM_PREC_C128 2  /* near entries and factors in complex128, FP64 arithmetic */
#define BEM_PREC_BF16F 4 /* the complex64 operator also keeps a BF16 copy of its far factors (4 bytes per
                            complex value; products in FP32); implies BEM_PREC_C64 */

/* Element type of a vector argument. */
#define BEM_C64 0
#define BEM_C128 1
#define BEM_C64_BF16F 2  /* complex64 vectors; bem_matvec uses the complex64 near entries and the BF16 factors */
#define BEM_C64_TC 3     /* complex64 vectors; bem_matvec applies the complex64 operator on the tensor cores in
                            passes of 64 vectors (three-term TF32 split, FP32-level accuracy) */

typedef struct {
    int precision;       /* bit mask of BEM_PREC_*: which operators bem_assemble builds (default C64) */
    int leaf_size;       /* maximum edges per leaf cluster, 2..64 (default 64) */
    double eta;          /* admissibility: min(diam) <= eta * dist; eta <= 0 stores every block densely (default 2) */
    double aca_tol;      /* relative Frobenius tolerance of each compressed block (default 1e-4) */
    int aca_max_rank;    /* rank cap per compressed block, 1..128 (default 96); a block that needs more, or more
                            than the break-even m n / (m + n), is split into its children's block pairs
                            (stored densely once both clusters are leaves) */
    int gmres_restart;   /* GMRES restart length (default 50) */
    int maxit;           /* maximum inner iterations: per right-hand side for GMRES, in total for the
                            CG-type solvers (default 1000) */
    double tol;          /* inner GMRES relative residual tolerance (default 1e-6) */
    double refine_tol;   /* outer FP64 iterative-refinement target; 0 disables refinement (default 0) */
    int refine_maxit;    /* maximum outer refinement steps (default 10) */
    int solver;          /* inner Krylov solver, BEM_SOLVER_* (default GMRES) */
    int aca_recompress;  /* 1 (default): after ACA, truncate each block's factors to the rank its singular
                            values need at aca_tol (Gram/Cholesky factors of U and V, SVD of the small core);
                            0: keep the ACA ranks */
    int preconditioner;  /* BEM_PRECOND_*: preconditioner of the GMRES solves (default BEM_PRECOND_NONE) */
    double precond_aca_tol; /* ACA tolerance of the refined-mesh operator inside the Calderon preconditioner
                               (default 3e-2): the preconditioner only has to be spectrally close (on the
                               61k-unknown sphere 1e-3, 1e-2, 3e-2 and 1e-1 give 32, 32, 32 and 34 GMRES
                               iterations for 12.9, 8.7, 6.9 and 5.2 GB per application) */
    int precond_near_only;  /* 1: the refined-mesh operator keeps only its densely stored (near-field) blocks,
                               which carry the singular part that the Calderon identity needs; 0 (default):
                               near and compressed far field */
} bem_options;

/* Preconditioners (bem_options.preconditioner).  Only the GMRES solver applies one;
 * the CG-type solvers return BEM_EINVAL when it is set, and adjoint solves run
 * without it. */
#define BEM_PRECOND_NONE 0
#define BEM_PRECOND_CALDERON 1  /* Calderon multiplicative preconditioner of PMCHWT, the 3-D counterpart of the
                                   Calderon-preconditioned CFIE of Sec. III: P = -Gb^-T Cb^T Z_fine Cb Gb^-1,
                                   applied on the right (Z P y = b, x = P y).  Z_fine is the PMCHWT operator of
                                   the barycentric refinement (six triangles per triangle, assembled and
                                   compressed at precond_aca_tol), C holds the Buffa-Christiansen
                                   functions of the edges in its RWG basis, G[m, e] = int (n x f_m) . g_e dS
                                   is the mixed Gram matrix (Gb = diag(G, G), Cb = diag(C, C)) and G^-1 is a
                                   fixed Chebyshev polynomial in D^-1 G (D = diag G) reaching a hundredth of
                                   precond_aca_tol (between 1e-10 and 1e-4) on a pseudo-random vector.
                                   bem_assemble builds it (about 6x the unknowns of Z); single-body contexts
                                   only.  GMRES iteration counts then stay bounded under mesh refinement. */

/* Inner Krylov solvers (bem_options.solver).  maxit counts iterations: one product
 * per GMRES iteration, two per CGS, BiCGStab and CGNR iteration. */
#define BEM_SOLVER_GMRES 0     /* restarted GMRES on all right-hand sides at once: one batched product per
                                  iteration, classical Gram-Schmidt (second pass where the first cancels),
                                  rotations and restarts on the device */
#define BEM_SOLVER_CGS 1       /* conjugate gradient squared */
#define BEM_SOLVER_BICGSTAB 2  /* stabilised bi-conjugate gradient */
#define BEM_SOLVER_CGNR 3      /* conjugate gradient on Z^H Z x = Z^H b (uses the adjoint product; not with
                                  BF16 factors, whose solves then use the complex64 operator) */

/* Parts of bem_assemble timed in bem_stats.assemble_phase_ms (host wall time, milliseconds). */
#define BEM_PHASE_TREE 0     /* geometry upload, cluster tree, block partition, leaf tables */
#define BEM_PHASE_SINGULAR 1 /* list and analytic integrals of the singular triangle pairs */
#define BEM_PHASE_ACA 2      /* adaptive cross approximation of the far blocks (all splitting rounds) */
#define BEM_PHASE_NEAR 3     /* quadrature of the densely stored blocks */
#define BEM_PHASE_PLAN 4     /* factor arena, product plan and work slots */
#define BEM_PHASES 5

/* Summary of an assembled operator (bem_stats). */
typedef struct {
    int64_t ne;                 /* RWG edges (unknowns = 2 ne) */
    int64_t nt;                 /* triangles */
    int64_t n_clusters;         /* nodes of the cluster tree */
    int64_t n_leaves;           /* leaf clusters */
    int64_t n_near;             /* dense (near) blocks */
    int64_t n_far;              /* admissible (far) blocks of the partition */
    int64_t n_far_dense;        /* leaf x leaf far blocks stored densely (ACA rank above the cap) */
    int64_t n_far_split;        /* far blocks split into their children's pairs (ACA rank above the cap) */
    int64_t n_far_factored;     /* blocks stored as low-rank factors after splitting */
    int64_t near_entries;       /* sum of m*n over densely stored blocks (per operator A, B or C) */
    int64_t factor_entries[3];  /* sum of r*(m+n) over far blocks, for A, B, C */
    int64_t max_rank;           /* largest ACA rank */
    int64_t singular_pairs;     /* triangle pairs integrated with singularity extraction */
    int64_t matvec_bytes_c64;   /* algorithmic HBM bytes of one complex64 product: every stored entry once,
                                   x read once, y written once */
    int64_t matvec_bytes_c128;  /* same for complex128 */
    int64_t kernel_bytes_c64[3];  /* algorithmic bytes of the product's kernels (gather, vhx, rows), complex64:
                                     gather: x read + permuted copy written; vhx: V factors + x;
                                     rows: dense entries + U factors + x + y */
    int64_t kernel_bytes_c128[3]; /* same for complex128 */
    int64_t matvec_bytes_bf16f;   /* same as matvec_bytes_c64 with the factors read as BF16 (BEM_C64_BF16F) */
    int64_t kernel_bytes_bf16f[3]; /* same as kernel_bytes_c64 for BEM_C64_BF16F */
    int64_t matvec_bytes_tc;      /* one BEM_C64_TC pass of 64 vectors: every stored entry once, 64 vectors read
                                     and 64 written (complex64) */
    int64_t kernel_bytes_tc[3];   /* its kernels: gather (x read, tree-order copy written), V^H x (V factors,
                                     the tree-order vectors once, t written: 64 values per t row), rows (dense
                                     entries, U factors, t read, the tree-order vectors once, y written) */
    int64_t t_rows;             /* t values per vector: sum over factored blocks of 2 (kA + 2 kB + kC) pairs */
    double assemble_ms;         /* wall time of the last bem_assemble */
    double assemble_phase_ms[BEM_PHASES]; /* its parts: see BEM_PHASE_* (ACA, near and plan summed over precisions) */
    int64_t tc_passes;          /* tensor-core operator passes (64 vectors each) run since bem_assemble, by
                                   bem_matvec with BEM_C64_TC and by batched solves */
    int64_t precond_fine_ne;    /* Calderon preconditioner (else 0): RWG edges of the barycentric refinement */
    int64_t precond_gram_nnz;   /* nonzeros of the mixed Gram matrix G */
    int64_t precond_gram_steps; /* Chebyshev steps per solve with G or G^T */
    int64_t precond_bytes_c64;  /* algorithmic bytes of one complex64 application of P to one vector: the
                                   refined operator's product bytes, C and C^T once, G and G^T once per
                                   Chebyshev step, and the vectors each step reads and writes */
    double precond_gram_interval[2]; /* eigenvalue interval of D^-1 G that the Chebyshev steps assume */
    double precond_assemble_ms; /* wall time of the preconditioner's share of bem_assemble (refinement, refined
                                   operator, BC and Gram matrices, Chebyshev plan) */
} bem_stats;

/* Kernels of one product, in launch order (index into the profiling arrays). */
#define BEM_KERNEL_GATHER 0  /* x -> tree order */
#define BEM_KERNEL_VHX 1     /* t = V^H x for every far block */
#define BEM_KERNEL_ROWS 2    /* per leaf: dense items + U t, writes y */

/* Fill *opt with the defaults listed above. */
void bem_default_options(bem_options* opt);

/* Create a context.  opt may be NULL (defaults).  *out receives the context. */
bem_status bem_create(const bem_options* opt, bem_ctx** out);

/* Release the context and every device buffer it owns.  NULL is accepted. */
void bem_destroy(bem_ctx* ctx);

/* Message of the last failed call on ctx ("" if none).  Valid until the next call. */
const char* bem_last_error(const bem_ctx* ctx);

/* Set the boundary mesh (Sec. III: the mesh of Gamma carrying the bases).
 * verts: host, nv x 3 double (row-major); tris: host, nt x 3 int32 vertex indices,
 * counter-clockwise seen from outside (outward normals).  The mesh must be
 * closed, two-manifold and consistently oriented with no degenerate triangle
 * (twice the area <= 1e-12 x longest edge squared); otherwise BEM_EINVAL.
 * RWG edges are numbered in lexicographic order of (min vertex, max vertex); T+ is
 * the adjacent triangle with the smaller index.  Invalidates any assembled operator. */
bem_status bem_set_mesh(bem_ctx* ctx, const double* verts, int64_t nv, const int32_t* tris, int64_t nt);

/* Set the media (Sec. III, after Eq. 7): exterior wavenumber k0 > 0 (rad per mesh
 * unit), interior relative permittivity and permeability for e^{+j w t}
 * (Im eps_r <= 0 and Im mu_r <= 0 for a lossy medium, else BEM_EINVAL).
 * k1 = k0 sqrt(eps_r mu_r) and eta_r = sqrt(mu_r/eps_r) use principal square roots.
 * Invalidates any assembled operator. */
bem_status bem_set_media(bem_ctx* ctx, double k0, bem_c128 eps_r, bem_c128 mu_r);

/* Layered bodies: several closed surfaces, each between two homogeneous regions
 * (a coated sphere, a body with inclusions).  The two rows of Eq. 7 hold on every
 * surface, with the field of each region radiated by the currents on that
 * region's own boundary; written region by region the operator is
 *
 *     Z = sum_r Q_r^T Z_r Q_r,   Z_r = [[ eta_r T_r , K_r ], [ -K_r , T_r / eta_r ]],
 *
 * Z_r the single-medium operator of region r (k_r = k0 sqrt(eps_r mu_r),
 * eta_r = sqrt(mu_r / eps_r); region 0: k0, 1) between the surfaces of its
 * boundary, Q_r selecting those surfaces' unknowns with the sign +1 where region
 * r lies on the normal side and -1 behind.  One surface between regions 0 and 1
 * gives the single-body operator above.  No paper counterpart (the paper treats
 * one homogeneous body).
 *
 * The mesh of bem_set_mesh holds every surface; the unknowns are as for one body
 * (x = [eta0 J ; M] over all edges, J and M taken on each surface's normal side).
 * tri_regions: host, nt x 2 int32, for each triangle the region its normal points
 * into and the region behind it: two different values in [0, n_regions); the two
 * triangles of every edge must carry the same pair; region 0 is the exterior
 * (free space, wavenumber k0 > 0) and must lie on the normal side of every
 * surface bounding it; every region needs a boundary.  eps_r, mu_r: host,
 * n_regions values for e^{+j w t} (Im <= 0, nonzero; entries 0 are ignored).
 * Else BEM_EINVAL (the context keeps its previous media).  Requires
 * bem_set_mesh; replaces bem_set_media (bem_set_media afterwards returns to one
 * body; bem_set_mesh afterwards drops the regions, and the media or regions must
 * be set again).  Invalidates any assembled operator.  Host only.
 *
 * On such a context bem_assemble builds one compressed single-medium operator per
 * region on the region's boundary (same options); bem_matvec, bem_matvec_adjoint,
 * bem_solve and bem_solve_adjoint apply Z or Z^H through them; bem_rhs_planewave
 * gives the incident field of region 0 (zero on the surfaces that do not bound
 * it); bem_power, bem_power_density, bem_absorbed_power_gradient and
 * bem_grad_weights use the currents of region 0's boundary alone, i.e. the power
 * absorbed, extinguished and scattered by the whole body; bem_stats_get and
 * bem_profile_end report sums over the regions' operators; bem_grad_eps gives
 * one pair of derivatives per region r >= 1.  bem_eval_entries,
 * bem_partition, bem_autotune and bem_absorbed_power_static return
 * BEM_ESTATE, bem_batch_create BEM_EINVAL. */
bem_status bem_set_regions(bem_ctx* ctx, double k0, int n_regions, const bem_c128* eps_r, const bem_c128* mu_r,
                           const int32_t* tri_regions);

/* Boundary of region r of a layered context (after bem_set_regions; host only).
 * *n_edges receives the number of RWG edges on it; edges and sign (host, room for
 * *n_edges values, or NULL) receive, in the order of the region's own operator,
 * the context's index of each of those edges and +1 / -1 (region r on the normal
 * side of the edge's surface / behind it).  BEM_ESTATE on a single body. */
bem_status bem_region_boundary(const bem_ctx* ctx, int r, int64_t* n_edges, int32_t* edges, int8_t* sign);

/* Double-Debye permittivity of Eq. 6 at freq_hz >= 0:
 * params = {eps_inf, eps_s, eps_2, tau1 [s], tau2 [s]}; NULL selects the skin
 * values given after Eq. 6 (3, 60, 3.6, 10 ps, 0.2 ps).  Host only, no context. */
bem_status bem_debye_eps(double freq_hz, const double* params, bem_c128* eps_out);

/* Build the operator on the GPU: cluster and block trees, singular-pair table,
 * dense near blocks, ACA factors of far blocks, for every precision requested in
 * the options.  Blocks until done (it reads block counts and ranks back to size
 * its buffers) and runs its kernels on `stream`.  Requires bem_set_mesh and
 * bem_set_media. */
bem_status bem_assemble(bem_ctx* ctx, void* stream);

/* Number of RWG edges ne and of unknowns 2*ne; -1 before bem_set_mesh. */
int64_t bem_num_edges(const bem_ctx* ctx);
int64_t bem_num_unknowns(const bem_ctx* ctx);

/* RWG table, host output ne x 4 int32: (v0, v1, T+, T-), v0 < v1. */
bem_status bem_edges(const bem_ctx* ctx, int32_t* out);

/* Operator summary (after bem_assemble). */
bem_status bem_stats_get(const bem_ctx* ctx, bem_stats* out);

/* Cluster order and block partition (after bem_assemble), host outputs:
 * perm: ne int64, perm[k] = edge at position k of the tree order;
 * near: n_near x 4 int32 and far: n_far x 4 int32 rows (row_lo, m, col_lo, n) in
 * tree positions, sorted by (row_lo, col_lo).  Any pointer may be NULL. */
bem_status bem_partition(const bem_ctx* ctx, int64_t* perm, int32_t* near, int32_t* far);

/* Evaluate operator entries directly by quadrature (no compression), device I/O:
 * rows, cols: device int32[count] edge indices (0..ne-1); out: device, count x 3
 * complex of type `dtype`: (A, B, C) = (T0 + eta_r T1, K0 + K1, T0 + T1/eta_r) at
 * (rows[i], cols[i]).  The same quadrature routine fills the dense blocks and
 * feeds the cross approximation.  Requires bem_assemble (for the singular-pair
 * table) with the matching precision. */
bem_status bem_eval_entries(bem_ctx* ctx, const int32_t* rows, const int32_t* cols, int64_t count,
                            void* out, int dtype, void* stream);

/* y = Z x for nrhs vectors.  x, y: device, 2ne x nrhs complex of type `dtype`
 * (BEM_C64, BEM_C128, BEM_C64_BF16F or BEM_C64_TC, needing the operator of that
 * precision: BEM_PREC_C64, BEM_PREC_C128, BEM_PREC_BF16F, BEM_PREC_C64;
 * BEM_C64_BF16F and BEM_C64_TC vectors are complex64); x and y must not
 * overlap.  Asynchronous on `stream`; no allocation after the first call with a
 * given nrhs.  The CUDA-core forms stream the operator once per chunk of up to 8
 * vectors; BEM_C64_TC streams it once per pass of up to 64 vectors, each stored
 * block entering a dense contraction on the tensor cores (Eq. 8's matrix times
 * many excitations at once; complex products embedded in real ones, each factor
 * split into TF32 high and low parts so that the result keeps FP32 accuracy).
 * The first BEM_C64_TC call builds that form's schedule and its workspaces
 * (64 vectors, 64 x the t values of the far blocks), synchronises `stream` and
 * needs a GB300 (sm_103); BEM_ETIMEOUT reports a tensor-core kernel of an earlier
 * call whose bounded wait ran out. */
bem_status bem_matvec(bem_ctx* ctx, const void* x, void* y, int nrhs, int dtype, void* stream);

/* y = Z^H x, the conjugate transpose of the assembled operator (adjoint solves
 * and gradients; the paper gives no adjoint).  Exact for the stored operator: the
 * transposed dense entries and, for every far block U V^H, the product V (U^H x)
 * through the same factors.  The matrix is complex symmetric only up to
 * quadrature and compression, so Z^T is not used in its place.
 * x, y: device 2ne x nrhs complex of type `dtype` (BEM_C64 or BEM_C128; the
 * BF16-factor form has no adjoint).  The first call for a precision builds the
 * transposed dense entries (as much memory as the dense entries) and their work
 * schedule, allocates and synchronises `stream`; later calls are asynchronous.
 * Errors as bem_matvec. */
bem_status bem_matvec_adjoint(bem_ctx* ctx, const void* x, void* y, int nrhs, int dtype, void* stream);

/* Autotuner of the product's block-to-CTA schedule: times the product of the
 * operator of `dtype` (10 products after 3 warm-ups, CUDA events on `stream`)
 * for rows-kernel schedules of 4 to 96 slots per SM in total, and keeps the
 * fastest (the sums of a leaf's slots are taken in a different grouping, so
 * results change at rounding level).  chosen (host, may be NULL): slots chosen;
 * ms_best (host, may be NULL): its time per product.  Allocates two vectors;
 * synchronises `stream`; drops the adjoint schedule, rebuilt on next use.
 * No paper counterpart. */
bem_status bem_autotune(bem_ctx* ctx, int dtype, void* stream, int* chosen, double* ms_best);

/* Several operators' products as one CUDA graph (many meshes of uneven size in
 * one launch).  bem_batch_create captures y[i] = Z_i x[i] (nrhs[i] vectors, type
 * `dtype`) of every context, each on its own branch of the graph so that small
 * meshes run side by side, and instantiates it; contexts must be distinct
 * (their workspaces are per context), assembled, not profiling, and they, x and
 * y must stay alive and unchanged (no re-assembly or autotuning) while the batch
 * exists.  bem_batch_launch runs the whole graph on `stream` (asynchronous);
 * bem_batch_destroy frees it.  No paper counterpart. */
typedef struct bem_batch bem_batch;
bem_status bem_batch_create(bem_ctx* const* ctxs, int n, const void* const* x, void* const* y, const int* nrhs,
                            int dtype, void* stream, bem_batch** out);
bem_status bem_batch_launch(bem_batch* batch, void* stream);
void bem_batch_destroy(bem_batch* batch);

/* Kernel timing of bem_matvec.  After bem_profile_begin, every bem_matvec on ctx
 * records a CUDA event pair around each of its kernels on the caller's stream
 * (a few microseconds of overhead per product); bem_profile_end synchronises those
 * events and returns, per kernel (BEM_KERNEL_*), the summed device time in
 * milliseconds (ms_sum, host, 3 doubles) and the number of launches (launches,
 * host, 3 int64), then stops recording.  Either output may be NULL. */
bem_status bem_profile_begin(bem_ctx* ctx);
bem_status bem_profile_end(bem_ctx* ctx, double* ms_sum, int64_t* launches);

/* Apply the Calderon preconditioner (BEM_PRECOND_CALDERON at bem_assemble): y = P x
 * for nrhs vectors; x, y device 2ne x nrhs (column-major) of type dtype (BEM_C64,
 * BEM_C64_BF16F, BEM_C64_TC or BEM_C128, as for bem_matvec; the refined operator
 * uses the same form).  x and y must not overlap.  Asynchronous on `stream`.
 * BEM_ESTATE without the preconditioner. */
bem_status bem_precond_apply(bem_ctx* ctx, const void* x, void* y, int nrhs, int dtype, void* stream);

/* A sparse matrix of the Calderon preconditioner, FP64 compressed rows (host):
 * which = 0: C, the Buffa-Christiansen function of every edge written in the RWG
 *            basis of the barycentric refinement (rows: refined edges, in the
 *            lexicographic order of the refined vertices, numbered vertices, then
 *            edge midpoints in edge order, then centroids in triangle order;
 *            columns: edges);
 * which = 1: the mixed Gram matrix G[m, e] = int (n x f_m) . g_e dS.
 * rows, cols, nnz (host, may be NULL) receive the sizes; ptr (rows + 1), col and
 * val (nnz each) receive the matrix when not NULL.  Host computation, available
 * once the mesh is set (no device work).  BEM_EINVAL if the context was not
 * created with BEM_PRECOND_CALDERON, BEM_ESTATE without a single-body mesh. */
bem_status bem_precond_matrix(const bem_ctx* ctx, int which, int64_t* rows, int64_t* cols, int64_t* nnz,
                              int32_t* ptr, int32_t* col, double* val);

/* Normalised plane-wave right-hand sides (tested fields after Eq. 8):
 * E_inc = e0 exp(-j k0 khat.r), H_inc = khat x E_inc / eta0, b = [e ; eta0 h].
 * khat: host nrhs x 3 double unit directions; e0: host nrhs x 3 complex
 * polarisations; b: device 2ne x nrhs complex of type `dtype`. */
bem_status bem_rhs_planewave(bem_ctx* ctx, const double* khat, const bem_c128* e0, int nrhs,
                             void* b, int dtype, void* stream);

/* Solve Z x = b for nrhs right-hand sides, b and x device complex128 2ne x nrhs.
 * Inner solver: restarted GMRES on the least precise operator assembled (BF16
 * factors, else complex64, else complex128), all right-hand sides together: each
 * iteration applies the operator once to every active basis vector (the
 * tensor-core product, BEM_C64_TC, for 16 or more right-hand sides of a complex64
 * solve on an sm_103 device), and each right-hand side keeps its own basis,
 * Hessenberg matrix and tolerance; inner products FP32 within a warp's rows and
 * FP64 beyond (complex64 inner solves) or FP64 throughout (complex128).  The
 * CG-type solvers (bem_options.solver) take the right-hand sides one at a time.
 * If refine_tol > 0 an outer loop recomputes r = b - Z x with complex128 vectors
 * through the most precise operator assembled (complex128 entries in FP64, else
 * the complex64 entries and FP32 factors with double-float products and sums,
 * about 2^-44 relative) and corrects x until |r|/|b| <= refine_tol.
 * x is used as the initial guess.
 * iters (host, may be NULL): total inner iterations over all right-hand sides;
 * relres (host, may be NULL): final relative residual per right-hand side (nrhs
 * doubles), measured with the most accurate operator available.  Synchronises
 * `stream`.  BEM_ENOCONV if any right-hand side misses its tolerance. */
bem_status bem_solve(bem_ctx* ctx, const void* b, void* x, int nrhs, void* stream, int* iters, double* relres);

/* Solve Z^H lambda = g (the adjoint system of gradient computations) for nrhs
 * right-hand sides, g and lambda device complex128 2ne x nrhs.  Same solver,
 * options and outputs as bem_solve with every product replaced by
 * bem_matvec_adjoint (inner GMRES on complex64 when assembled, else complex128;
 * BF16 factors are not used); lambda is used as the initial guess. */
bem_status bem_solve_adjoint(bem_ctx* ctx, const void* g, void* lambda, int nrhs, void* stream, int* iters,
                             double* relres);

/* Powers of a solution x (device complex128 2ne x nrhs) for its right-hand side b,
 * in units of 1/(2 eta0) (efficiency Q = value / (pi a^2 |E0|^2)):
 *   p_abs = Re(xJ^H X xM),  X[m,n] = int f_m . (n x f_n)   (absorbed, -Re oint E x H* . n)
 *   p_ext = Re(xJ^H bJ + bM^H xM)                           (extinguished)
 *   p_sca = oint |E_far|^2 dOmega on a 64 x 128 Gauss-Legendre x uniform grid,
 *           E_far = (j k0/4pi) (rhat x L - N_t) of the normalised currents.
 * Host outputs of nrhs doubles each (any may be NULL).  Synchronises `stream`. */
bem_status bem_power(bem_ctx* ctx, const void* x, const void* b, int nrhs, double* p_abs, double* p_ext,
                     double* p_sca, void* stream);

/* Gradient of the absorbed power with respect to the conjugate coefficients:
 * g = dP_abs/d conj(x) = (1/2) [X xM ; X^T xJ] (X as in bem_power; P_abs = x^H H x
 * with H Hermitian, so g = H x).  x, g: device complex128 2ne x nrhs, distinct.
 * Asynchronous on `stream`.  No paper counterpart (the source term of the
 * adjoint solve of a gradient). */
bem_status bem_absorbed_power_gradient(bem_ctx* ctx, const void* x, void* g, int nrhs, void* stream);

/* Absorbed power of a weighted sum of excitations and its gradient with respect to
 * the weights, by one forward and one adjoint solve.  bm: device complex128
 * 2ne x nw, column i the right-hand side of excitation i (e.g. from
 * bem_rhs_planewave); w: host nw complex weights; b = bm w, Z x = b,
 * P = Re(xJ^H X xM) (host *p_abs), Z^H lambda = dP/d conj(x), and
 * grad[i] = dP/d conj(w_i) = bm_i^H lambda (host nw complex; the real gradient is
 * (2 Re grad, 2 Im grad) with respect to (Re w, Im w)).  x_out, lambda_out: device
 * complex128 2ne, or NULL.  iters (host, may be NULL): inner iterations of both
 * solves.  Solver options as bem_solve.  Allocates scratch; synchronises `stream`.
 * No paper counterpart. */
bem_status bem_grad_weights(bem_ctx* ctx, const void* bm, int nw, const bem_c128* w, double* p_abs,
                            bem_c128* grad, void* x_out, void* lambda_out, void* stream, int* iters);

/* Gradient of the absorbed power with respect to the interior permittivity,
 * given the forward solution x (Z x = b) and the adjoint solution lambda
 * (Z^H lambda = dP/d conj(x), e.g. the x_out and lambda_out of bem_grad_weights):
 * dp[0] = dP/d Re(eps_r), dp[1] = dP/d Im(eps_r) (host), from
 * dP = -2 Re(lambda^H (dZ/d eps_r) x d eps_r).  The derivative of the interior
 * blocks is applied between lambda and x by an O(nt^2) pass over all triangle
 * pairs in FP64 (the k-derivative of the quadrature: dG/dk = -j e^{-jkR}/(4 pi),
 * and of the singular-pair extraction), so it is exact for the uncompressed
 * discretisation; meant for the moderate meshes of design problems.  x, lambda:
 * device complex128 2ne.  On a layered context (bem_set_regions) dp holds
 * 2 (bem_num_regions - 1) values, the pair for region 1, then region 2, ...: only
 * region r's operator depends on its permittivity, so its pair is the same form
 * of region r's operator between the signed currents of its boundary.
 * Allocates scratch; synchronises `stream`.  No paper counterpart. */
bem_status bem_grad_eps(bem_ctx* ctx, const void* x, const void* lambda, double* dp, void* stream);

/* Number of regions: 2 for one body (exterior and interior), n_regions after
 * bem_set_regions, -1 before the media are set.  Host only. */
int bem_num_regions(const bem_ctx* ctx);

/* Absorbed power density per triangle for the first right-hand side of x
 * (device complex128): per_tri (device, nt doubles) = Re(sum_ij conj(xJ_i) X_t[i,j] xM_j) / area_t,
 * same units as bem_power. */
bem_status bem_power_density(bem_ctx* ctx, const void* x, double* per_tri, void* stream);

/* Absorbed power written to device memory, with no device allocation.
 * No counterpart in the paper: this entry point exists for callers that cannot
 * let a library allocate device memory during the call -- a framework that owns
 * all device memory through its own pool allocator and budget, or a
 * latency-critical loop that must not take the implicit synchronisation of
 * cudaMalloc/cudaFree.  It computes the p_abs of bem_power (same units) for nrhs
 * right-hand sides: x device complex128 2ne x nrhs, p_abs device nrhs doubles,
 * asynchronously on `stream`; nothing is copied to the host.  Its partial sums
 * live in a fixed 512 KiB array inside the library on each device (65536 doubles,
 * held until the process exits): nrhs * ceil(nt / 256) must not exceed 65536,
 * else BEM_EINVAL with the sizes in bem_last_error.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress) once; make that
 * first call before any stream capture.  All calls share the array and every
 * call rewrites the partial sums it reads, so nothing carries over between
 * calls; calls whose work can overlap on the GPU (different streams without
 * ordering between them) race on the array, so order them.  Requires
 * bem_assemble. */
bem_status bem_absorbed_power_static(bem_ctx* ctx, const void* x, int nrhs, double* p_abs, void* stream);

/* The paper's own two-dimensional setting (Sec. II: fields invariant along z):
 * dense Galerkin matrices of the single-layer S, double-layer D and hypersingular
 * N operators of Eqs. 1-4 with the kernel -(j/4) H0^(2)(k R) (Eq. 5), tested and
 * expanded with hat functions on the closed polygon verts (host, n x 2 doubles,
 * counter-clockwise, n >= 3): (O)_ij = (lambda_i, O lambda_j) with lambda_i the
 * hat function of vertex i.  The adjoint double layer of Eq. 3 is D^T.  N uses
 * the identity (lambda_i, N lambda_j) = int int G (lambda_i' lambda_j' -
 * k^2 n.n' lambda_i lambda_j) (N = -d_n D).  Quadrature: segment pairs whose
 * midpoints lie at least 6 segment lengths apart take the 5 x 5 Gauss-Legendre
 * rule on the whole kernel; closer pairs take 10 x 10 points after the static
 * parts of the kernels are integrated over the source segment in closed form (the
 * outer rule 20 points graded toward the shared vertex of neighbouring segments);
 * a segment with itself takes the logarithm over both copies in closed form.
 * k: complex wavenumber with Re k > 0 and Im k <= 0.  fp32: 0 = FP64 throughout
 * (Hankel functions from their ascending series below |k R| = 12 and Hankel's
 * expansion above); 1 = the well-separated pairs with |k R| >= 8 in FP32
 * (Hankel's expansion, the phase e^{-j k R} split into an FP64 midpoint part and
 * an FP32 offset part), about 1e-6 relative accuracy, the rest FP64.  S, D, N:
 * device complex128 n x n, row-major (element (i, j) at i * n + j), each may be
 * NULL.  Allocates 128 n^2 bytes of scratch; synchronises `stream`.  ctx (may be
 * NULL) only receives the error message.  No counterpart in the three-dimensional
 * path. */
bem_status bem_planar_operators(bem_ctx* ctx, const double* verts, int n, bem_c128 k, int fp32, void* S, void* D,
                                void* N, void* stream);

/* The paper's two-dimensional fast direct solver (Sec. III), FP64 on the GPU.
 * Polygons as in bem_planar_operators (n vertices, counter-clockwise, closed);
 * dense matrices device complex128 n x n row-major; U n x r column-major (column c
 * at U + c n); Vt r x n row-major; omega, b, x column-major with n rows.  Each call
 * synchronises `stream`; ctx (may be NULL) only receives the error message. */

/* Calderon-preconditioned CFIE of Eq. 16: Cp = N~ G^-1 S + (G/2 - D*~) G^-1 (G/2 + D*)
 * with S, D, N at k0 and D*~, N~ at k~ = k0 - 0.4 j k0^(1/3) a^(-2/3) (a <= 0: the
 * perimeter over 2 pi), G the Gram matrix of the hat functions (solved as a cyclic
 * tridiagonal system).  Le = N~ G^-1 and Lh = (G/2 - D*~) G^-1 (may be NULL) map the
 * right-hand side: rhs_p = Le (e / (j k0)) + Lh (eta0 h).  fp32: the operators'
 * form as in bem_planar_operators (the Gram solves and products stay FP64).
 * Allocates about 10 n^2 x 16 bytes of scratch. */
bem_status bem_planar_calderon(bem_ctx* ctx, const double* verts, int n, double k0, double a, int fp32, void* Cp,
                               void* Le, void* Lh, void* stream);

/* In-place FFT of `batch` vectors of length n (1..2048), vector b at x + b * batch_stride,
 * element stride `stride` (complex128 elements): forward sum_j x_j exp(-2 pi i jk/n),
 * inverse (inverse != 0) with exp(+2 pi i jk/n) / n.  Bluestein's chirp convolution
 * on radix-2 transforms, one CTA per vector. */
bem_status bem_fft(bem_ctx* ctx, void* x, int n, long long stride, int batch, long long batch_stride, int inverse,
                   void* stream);

/* Skeleton of Eq. 17 by the adaptive randomized range finder: orthonormal U with
 * |(I - U U^H) A w| <= tol * (largest |A w| of the first block) for the test vectors w,
 * taken `block` at a time from the p columns of omega (the random numbers are an
 * input), each block orthogonalised twice against U and among itself; Vt = U^H A.
 * A: the matrix to compress (C_p - C_p,c); U: capacity n x p; Vt: capacity p x n
 * (may be NULL); rank: host, the columns of U used.  BEM_ENOCONV if the test vectors
 * run out first. */
bem_status bem_planar_skeleton(bem_ctx* ctx, const void* A, int n, const void* omega, int p, double tol, int block,
                               void* U, void* Vt, int* rank, void* stream);

/* Woodbury solve of Eq. 18: x = (C_c + U Vt)^-1 b for nrhs right-hand sides, C_c the
 * circulant matrix whose first column is cc0 (device, n values; its eigenvalues by
 * FFT), U and Vt of rank r (r = 0: x = C_c^-1 b).  The r x r core is solved by LU
 * with partial pivoting (BEM_EINVAL if singular). */
bem_status bem_planar_woodbury_solve(bem_ctx* ctx, const void* cc0, int n, const void* U, const void* Vt, int r,
                                     const void* b, void* x, int nrhs, void* stream);

/* FMA throughput of the current device in TFLOP/s (2 FLOP per fused multiply-add),
 * FP64 if fp64 != 0 else FP32: the denominators of the arithmetic rooflines
 * (quadrature and ACA assembly, the complex128 product).  Runs a few short
 * launches of independent FMA chains on `stream` (about 5 ms in all) and returns
 * the best; changes no clock or power setting.  Allocates a few KB of device
 * memory for the duration of the call. */
bem_status bem_measure_fma_peak(int fp64, void* stream, double* tflops);

/* Test hook (host-side fault injection): after `after` further successful device
 * allocations by the library (any context), each allocation fails as if the
 * device were out of memory (cudaErrorMemoryAllocation, no CUDA call made), so
 * that the entry point that needed it returns BEM_ENOMEM.  after < 0 turns the
 * injection off (the default).  Not thread-safe against concurrent calls. */
void bem_debug_fail_alloc_after(long long after);

#ifdef __cplusplus
}
#endif

#endif /* BEM_H */
