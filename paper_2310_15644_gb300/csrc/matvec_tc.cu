// The compressed PMCHWT product y = Z x for many right-hand sides on the
// fifth-generation tensor cores (tcgen05): passes of 64 vectors, each pass one
// stream over the stored operator (Eq. 8's system matrix with its far blocks in
// the skeleton form U V^H of Eq. 17).
//
// Every stored block meets 64 vectors at once, so its entries enter a dense
// contraction.  Complex products are embedded in real ones on the operator side:
// a stored row i of Z (complex) becomes the two rows (i, re) and (i, im) of a real
// matrix over K = (column j, re/im),
//     (i, re): [ Re z_ij, -Im z_ij ],   (i, im): [ Im z_ij, Re z_ij ],
// so that this real matrix times the vector block X laid out as K = (j, re/im) by
// 64 columns gives Re and Im of Z X in the rows (i, re) and (i, im).  The real
// operator rows (128 per leaf of 64 rows) are the MMA's A operand in tensor
// memory; threads build them from the stored complex64 entries, so the stored
// layout serves the single-vector kernels and these alike.  The vector blocks are
// the B operand in shared memory.  FP32 accuracy comes from the three-term TF32
// split (tc.cuh): hi*hi + hi*lo + lo*hi, the main terms and the corrections in
// separate accumulators, both moved into FP32 registers every few K steps (the
// tensor core rounds its accumulation toward zero, which drifts over long chains).
//
// Kernels of one pass:
//   1. k_tc_gather  xp[pos][r] = x[r][edge(pos)]   (tree order, 64 vectors per position)
//   2. k_tc_vhx     t_b = W_b^T xp_sigma for every far block: tasks of up to 32 rank
//                   pairs of the blocks that share a column cluster (and a half J or
//                   M of the vector), accumulated over the cluster's columns;
//                   t[row][r] written through shared memory, one 512-byte row at a time
//   3. k_tc_rows    per work slot of a leaf (the single-vector product's schedule):
//                   y_J += A xJ + B xM,  y_M += C xM - B xJ over its dense items and
//                   y_J += U_A t_A + U_B t_BM, y_M += U_C t_C - U_B t_BJ over its far
//                   pieces (the minus sign rides on a negated copy of x_J / t_BJ);
//                   partial rows of a leaf split over several slots are summed by
//                   the last slot to finish (arrival counter).
// Both tensor kernels are persistent (one CTA per SM; CTA b takes work items b,
// b + #CTAs, ... of a heaviest-first list) and split their warps by role:
//   * a producer warp stages each chunk's operator and vector data by bulk copies
//     (cp.async.bulk) into a ring of shared-memory stages ahead of use;
//   * eight builder warps turn a staged chunk into the tensor-core operands
//     (operator rows, embedded and split, into tensor memory; vectors, split, into
//     shared tiles) and signal the issuer through the buffer's mbarrier;
//   * an issuer warp starts the chunk's MMAs and commits them to the chunk's
//     buffer barrier; operand buffers are double-buffered, so the builders prepare
//     chunk c + 1 while the tensor core runs chunk c.
// MMAs that share their A operand are merged along N: the vector tiles of a K step
// hold row groups [x_J hi, x_J lo, x_M hi, x_M lo, -x_J hi, -x_J lo, t_C hi, t_C lo]
// and the accumulators columns [J main, J corr, M main, M corr], so for instance
// B_hi x [x_M hi, x_M lo, -x_J hi, -x_J lo] is one N = 256 MMA into all four.
// Every wait is bounded: one that runs out makes the CTA stop at the next slot (or
// task) boundary, record *err, wait (bounded) for the copies and MMAs already
// issued, free its tensor memory and return.
#include "common.cuh"
#include "tc.cuh"

namespace bem {

namespace {

constexpr int NR = BEM_TC_NR;              // 64 right-hand sides per pass
constexpr uint32_t WAIT_LIMIT = 1u << 22;  // polls of an mbarrier before giving up
constexpr int NBUILD = 256;                // builder threads (warps 0-7)
constexpr int THREADS = 320;               // + producer warp 8 + issuer warp 9
constexpr uint32_t BAR_DECIDE = 1;         // builders + issuer: stop/continue decisions
constexpr uint32_t BAR_BUILD = 3;          // builders only
// (builders tell the issuer that a chunk's operands are ready through an mbarrier per
// operand buffer: the builders of chunk c + 2 first wait for chunk c's MMAs, so an
// arrival can never run ahead of the phase the issuer is waiting for)
constexpr int TILE_ROWS_BYTES = 64 * 16;   // 64 vector rows x 16 bytes (one row group, one K chunk)

// ---- rows kernel ---------------------------------------------------------------
constexpr int RKS = 2;                     // K steps (4 complex columns each) per chunk
constexpr int FLUSH_STEPS = 4;             // K steps between moves of the accumulators into registers
constexpr int R_GROUPS = 8;                // vector row groups per tile (see above)
constexpr int R_TILE_BYTES = 2 * R_GROUPS * TILE_ROWS_BYTES;       // one K step: 2 K chunks x 512 rows (16 KiB)
constexpr int R_TILES_BYTES = 2 * RKS * R_TILE_BYTES;              // 2 buffers (64 KiB)
constexpr int RSTAGES = 4;                                         // staged chunks in flight
constexpr int R_OP_BYTES = 3 * 4 * 64 * 16;                        // operator: 3 parts x 4 pairs x 64 rows
constexpr int R_STAGE_BYTES = R_OP_BYTES + 4 * 8 * NR * 8;         // + vectors: 4 slots x 8 rows x 64 (28 KiB)
constexpr int R_SMEM_BYTES = R_TILES_BYTES + RSTAGES * R_STAGE_BYTES + (RSTAGES + 2) * 64 + 256;  // one CTA per SM
// tensor-memory columns: accumulators [J main | J corr | M main | M corr], then two A
// buffers of RKS x 3 parts x (hi, lo) x 8
constexpr uint32_t COL_JH = 0, COL_JL = 64, COL_MH = 128, COL_ML = 192, COL_A = 256;
__device__ __forceinline__ uint32_t a_col(int buf, int s, int q, int h) {
    return COL_A + (uint32_t)((buf * RKS + s) * 48 + (q * 2 + h) * 8);
}

// ---- V^H x kernel --------------------------------------------------------------
constexpr int VKS = 8;                     // K steps per chunk
constexpr int VCOLS = 4 * VKS;             // columns per chunk
constexpr int V_TILE_BYTES = 2 * 2 * TILE_ROWS_BYTES;              // one K step: 2 K chunks x [hi, lo] rows (4 KiB)
constexpr int V_TILES_BYTES = 2 * VKS * V_TILE_BYTES;              // 2 buffers (64 KiB)
constexpr int V_W_BYTES = VCOLS * 32 * 16;                          // staged W: [column][32 pairs] x 16 bytes
constexpr int V_STAGE_BYTES = V_W_BYTES + VCOLS * NR * 8;          // + vector rows (32.5 KiB)
constexpr int VSTAGES = 3;
constexpr int V_OUT_ROW = NR * 2 + 2;                              // staged t row (floats; padded: no bank conflicts)
constexpr int V_OUT_FLOATS = 4 * 16 * V_OUT_ROW;                   // epilogue staging: 4 quadrants x 16 rank rows
constexpr int V_SMEM_BYTES = V_TILES_BYTES + VSTAGES * V_STAGE_BYTES + V_OUT_FLOATS * 4 + 128;
constexpr uint32_t VCOL_DH = 0, VCOL_DL = 64, VCOL_A = 128;
constexpr int VFLUSH_STEPS = 16;
__device__ __forceinline__ uint32_t va_col(int buf, int s, int h) {
    return VCOL_A + (uint32_t)((buf * VKS + s) * 16 + h * 8);
}

// the 8 real K values of one embedded operator row over 4 complex columns
// (z0..z3 = (re, im) pairs): row part d = 0 gives [re, -im] per column, d = 1 [im, re];
// split into TF32 hi and lo
__device__ __forceinline__ void embed_split(const float4& p0, const float4& p1, int d, uint32_t (&hi)[8],
                                            uint32_t (&lo)[8]) {
    const float z[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
        const float re = z[2 * jj], im = z[2 * jj + 1];
        const float a = d ? im : re, b = d ? re : -im;
        tc::tf32_split(a, hi[2 * jj], lo[2 * jj]);
        tc::tf32_split(b, hi[2 * jj + 1], lo[2 * jj + 1]);
    }
}

__device__ __forceinline__ float4 shfl4_xor(const float4& v, int m) {
    float4 r;
    r.x = __shfl_xor_sync(0xffffffffu, v.x, m);
    r.y = __shfl_xor_sync(0xffffffffu, v.y, m);
    r.z = __shfl_xor_sync(0xffffffffu, v.z, m);
    r.w = __shfl_xor_sync(0xffffffffu, v.w, m);
    return r;
}

__device__ __forceinline__ void split4(const float4& v, float4& h, float4& l) {
    uint32_t a, b;
    tc::tf32_split(v.x, a, b);
    h.x = __uint_as_float(a);
    l.x = __uint_as_float(b);
    tc::tf32_split(v.y, a, b);
    h.y = __uint_as_float(a);
    l.y = __uint_as_float(b);
    tc::tf32_split(v.z, a, b);
    h.z = __uint_as_float(a);
    l.z = __uint_as_float(b);
    tc::tf32_split(v.w, a, b);
    h.w = __uint_as_float(a);
    l.w = __uint_as_float(b);
}

// Vector tile rows of one K step from staged vector rows: K index (jj, re/im) over
// rows jl0 .. jl0 + 3 of the staged slot, whose first row has index jg0 in the
// numbering nvalid counts (zero at or beyond nvalid: rows never staged are not read).  Thread t (0..127) handles vector column r = t & 63 and K chunk t >> 6;
// it writes hi and lo to row groups gh and gh + 1 of the tile (K-major, 16 bytes per
// (K chunk, row); gh < 0 skips them) and, if gneg >= 0, the negated values to
// groups gneg, gneg + 1.
__device__ __forceinline__ void build_b_rows(unsigned char* tile, int ngroups, const float2* stv, int jl0, int jg0,
                                             int nvalid, int t, int gh, int gneg) {
    const int r = t & 63, kc = t >> 6;
    const int ja = 2 * kc, jb = ja + 1;
    float2 a = make_float2(0.f, 0.f), b = a;
    if (jg0 + ja < nvalid) a = stv[(jl0 + ja) * NR + r];
    if (jg0 + jb < nvalid) b = stv[(jl0 + jb) * NR + r];
    float4 h, l;
    split4(make_float4(a.x, a.y, b.x, b.y), h, l);
    float4* base = reinterpret_cast<float4*>(tile) + kc * ngroups * 64 + r;
    if (gh >= 0) {
        base[gh * 64] = h;
        base[(gh + 1) * 64] = l;
    }
    if (gneg >= 0) {
        base[gneg * 64] = make_float4(-h.x, -h.y, -h.z, -h.w);
        base[(gneg + 1) * 64] = make_float4(-l.x, -l.y, -l.z, -l.w);
    }
}

// Accumulators of the rows kernel moved into registers: warp w owns lanes
// 32 (w & 3) .. + 31 and columns 32 (w >> 2) .. + 31 of each accumulator; it adds
// main and correction terms into rj (y_J) and rm (y_M) and clears its part of
// tensor memory.  The tensor core must have finished (caller waited).
__device__ __forceinline__ void flush_rows(uint32_t tb, int warp, float (&rj)[32], float (&rm)[32]) {
    const uint32_t ln = 32 * (warp & 3), c0 = 32 * (warp >> 2);
    const uint32_t z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float a[16], b[16];
        tc::tmem_ld16(tc::taddr(tb, ln, COL_JH + c0 + 16 * h), a);
        tc::tmem_ld16(tc::taddr(tb, ln, COL_JL + c0 + 16 * h), b);
#pragma unroll
        for (int j = 0; j < 16; ++j) rj[16 * h + j] += a[j] + b[j];
        tc::tmem_ld16(tc::taddr(tb, ln, COL_MH + c0 + 16 * h), a);
        tc::tmem_ld16(tc::taddr(tb, ln, COL_ML + c0 + 16 * h), b);
#pragma unroll
        for (int j = 0; j < 16; ++j) rm[16 * h + j] += a[j] + b[j];
    }
#pragma unroll
    for (uint32_t c = 0; c < 32; c += 8) {
        tc::tmem_st8(tc::taddr(tb, ln, COL_JH + c0 + c), z);
        tc::tmem_st8(tc::taddr(tb, ln, COL_JL + c0 + c), z);
        tc::tmem_st8(tc::taddr(tb, ln, COL_MH + c0 + c), z);
        tc::tmem_st8(tc::taddr(tb, ln, COL_ML + c0 + c), z);
    }
    tc::tmem_st_wait();
}

}  // namespace

// One item of the rows kernel: 3 operator parts (A/U_A, B/U_B, C/U_C) as 16-byte
// column pairs (pair (k, i) at base + k * ld + i, npair pairs per part) and 4 vector
// slots (rows at vec[o] + j * NR, nvec[o] valid rows): dense items x_J, x_M (slots
// 2, 3 repeat them), far pieces t_A, t_BM, t_C, t_BJ.
struct TcItem {
    const float4* base[3];
    int ld, m, npair[3];
    const c64* vec[4];
    int nvec[4];
    bool far;
};

// Header of a staged chunk, written by the producer and copied by the builders for
// the issuer: kind 0 data, 1 end of slot; pairs per operator part and valid vector
// rows per slot in this chunk; K steps; far piece; pair stride.
struct __align__(16) TcHdr {
    int kind, ks, far, ld;
    int npr[4];   // [3] unused
    int nrow[4];
    int pad[4];
};

// Chunk c of an item: column (or rank) pairs [4c, 4c + 4) of each operator part
// and rows [8c, 8c + 8) of each vector slot, staged by bulk copies: part q at
// q * 4 KiB (pair k, row i at (k ld + i) * 16 bytes), vector slot o at
// R_OP_BYTES + o * 4 KiB (row j at j * 512 bytes).  Dense items stage slots 0 (x_J)
// and 1 (x_M); far pieces all four t segments.  Returns the chunk's header.
__device__ __forceinline__ void stage_chunk(const TcItem& it, int c, unsigned char* st, TcHdr* hdr, uint64_t* full,
                                            uint64_t pol) {
    uint32_t bytes = 0;
    TcHdr h;
    h.kind = 0;
    h.far = it.far ? 1 : 0;
    h.ld = it.ld;
    const int np = max(it.npair[0], max(it.npair[1], it.npair[2]));
    h.ks = min(RKS, ((np + 1) >> 1) - RKS * c);
    for (int q = 0; q < 3; ++q) {
        h.npr[q] = min(4, max(0, it.npair[q] - 4 * c));
        bytes += (uint32_t)(h.npr[q] * it.ld * 16);
    }
    h.npr[3] = 0;
    const int nslot = it.far ? 4 : 2;
    for (int o = 0; o < 4; ++o) {
        h.nrow[o] = o < nslot ? min(8, max(0, it.nvec[o] - 8 * c)) : 0;
        bytes += (uint32_t)(h.nrow[o] * NR * 8);
    }
    *hdr = h;
    tc::mbar_arrive_expect_tx(full, bytes);  // releases the header too
    for (int q = 0; q < 3; ++q)
        if (h.npr[q] > 0)
            tc::bulk_g2s_hint(st + q * 4096, it.base[q] + (int64_t)4 * c * it.ld, (uint32_t)(h.npr[q] * it.ld * 16),
                              full, pol);
    for (int o = 0; o < 4; ++o)
        if (h.nrow[o] > 0)
            tc::bulk_g2s(st + R_OP_BYTES + o * 4096, it.vec[o] + (int64_t)8 * c * NR, (uint32_t)(h.nrow[o] * NR * 8),
                         full);
}

// record i of the producer warp (held by lane i) as a TcItem
__device__ __forceinline__ void tc_item_from_rec(const int4 (&r)[4], int i, const MatvecPlan& p, const c64* near,
                                                 const c64* arena, const c64* xp, const c64* t, int m, TcItem& it,
                                                 int& kind) {
    int v[16];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        v[4 * q + 0] = __shfl_sync(0xffffffffu, r[q].x, i);
        v[4 * q + 1] = __shfl_sync(0xffffffffu, r[q].y, i);
        v[4 * q + 2] = __shfl_sync(0xffffffffu, r[q].z, i);
        v[4 * q + 3] = __shfl_sync(0xffffffffu, r[q].w, i);
    }
    auto i64 = [&](int k) { return (int64_t)(((uint64_t)(uint32_t)v[2 * k + 1] << 32) | (uint32_t)v[2 * k]); };
    kind = v[13];
    it.m = m;
    const int64_t b0 = i64(0), b1 = i64(1), b2 = i64(2), vec = i64(3);
    const int np0 = v[8], np1 = v[9], np2 = v[10];
    it.npair[0] = np0;
    it.npair[1] = np1;
    it.npair[2] = np2;
    if (kind == 0) {
        it.base[0] = reinterpret_cast<const float4*>(near + b0);
        it.base[1] = reinterpret_cast<const float4*>(near + b1);
        it.base[2] = reinterpret_cast<const float4*>(near + b2);
        it.ld = m;
        const int n = v[12];
        it.vec[0] = xp + vec * NR;
        it.vec[1] = xp + ((int64_t)p.ne + vec) * NR;
        it.vec[2] = it.vec[1];
        it.vec[3] = it.vec[0];
        it.nvec[0] = it.nvec[1] = it.nvec[2] = it.nvec[3] = n;
        it.far = false;
    } else {
        it.base[0] = reinterpret_cast<const float4*>(arena + b0);
        it.base[1] = reinterpret_cast<const float4*>(arena + b1);
        it.base[2] = reinterpret_cast<const float4*>(arena + b2);
        it.ld = v[11];
        const c64* tA = t + vec * NR;
        const c64* tBJ = tA + (int64_t)2 * np0 * NR;
        const c64* tBM = tBJ + (int64_t)2 * np1 * NR;
        const c64* tC = tBM + (int64_t)2 * np1 * NR;
        it.vec[0] = tA;
        it.vec[1] = tBM;
        it.vec[2] = tC;
        it.vec[3] = tBJ;
        it.nvec[0] = 2 * np0;
        it.nvec[1] = it.nvec[3] = 2 * np1;
        it.nvec[2] = 2 * np2;
        it.far = true;
    }
}

// The MMAs of one K step of the rows kernel (issuer thread): A parts in tensor
// memory (hi, lo), vector row groups of the step's tile (LBO: the tile's 512 rows
// of one K chunk), accumulators from column 0.
__device__ __forceinline__ void rows_step_mma(uint32_t tb, int buf, int s, const unsigned char* tile,
                                              const TcHdr& h) {
    const uint32_t id64 = tc::idesc_tf32(128, 64), id128 = tc::idesc_tf32(128, 128),
                   id256 = tc::idesc_tf32(128, 256);
    const uint32_t t0 = tc::smem_u32(tile);
    auto grp = [&](int g) { return tc::sdesc(t0 + g * TILE_ROWS_BYTES, R_GROUPS * TILE_ROWS_BYTES, 128); };
    const int gC = h.far ? 6 : 2;   // t_C, or x_M again for the dense C part
    if (2 * s < h.npr[0]) {         // A: x_J / t_A into J
        tc::mma_tf32_ts(tb + COL_JH, tb + a_col(buf, s, 0, 0), grp(0), id128, 1);  // hi x [hi, lo] -> J main, corr
        tc::mma_tf32_ts(tb + COL_JL, tb + a_col(buf, s, 0, 1), grp(0), id64, 1);   // lo x hi -> J corr
    }
    if (2 * s < h.npr[1]) {         // B: x_M / t_BM into J, -x_J / -t_BJ into M
        tc::mma_tf32_ts(tb + COL_JH, tb + a_col(buf, s, 1, 0), grp(2), id256, 1);
        tc::mma_tf32_ts(tb + COL_JL, tb + a_col(buf, s, 1, 1), grp(2), id64, 1);
        tc::mma_tf32_ts(tb + COL_ML, tb + a_col(buf, s, 1, 1), grp(4), id64, 1);
    }
    if (2 * s < h.npr[2]) {         // C: x_M / t_C into M
        tc::mma_tf32_ts(tb + COL_MH, tb + a_col(buf, s, 2, 0), grp(gC), id128, 1);
        tc::mma_tf32_ts(tb + COL_ML, tb + a_col(buf, s, 2, 1), grp(gC), id64, 1);
    }
}

struct TcRowsArgs {
    MatvecPlan p;
    TcPlan tp;
    const c64* near;
    const c64* arena;
    c64* y;            // caller layout, nr vectors
    int nr;
};

__global__ void __launch_bounds__(THREADS, 1) k_tc_rows(TcRowsArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* tiles = smem;
    unsigned char* stages = smem + R_TILES_BYTES;
    TcHdr* hdr = reinterpret_cast<TcHdr*>(stages + RSTAGES * R_STAGE_BYTES);  // RSTAGES: producer -> builders
    TcHdr* hdrb = hdr + RSTAGES;                                              // 2: builders -> issuer
    uint64_t* bar = reinterpret_cast<uint64_t*>(hdrb + 2);
    uint64_t* mma_bar = bar;              // 2: tensor core done with A/B buffer
    uint64_t* full = bar + 2;             // RSTAGES: stage loaded
    uint64_t* empty = full + RSTAGES;     // RSTAGES: stage consumed
    uint64_t* ready = empty + RSTAGES;    // 2: operands of the buffer's chunk built
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(ready + 2);
    int* s_fail = reinterpret_cast<int*>(s_tmem + 1);
    int* s_last = s_fail + 1;
    int* s_issued = s_fail + 2;
    int* s_consumed = s_fail + 3;
    const MatvecPlan& p = a.p;
    const TcPlan& tp = a.tp;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ne = p.ne;
    const int64_t nn = 2 * (int64_t)ne;
    const int sl0 = tp.cta_slot_ptr[blockIdx.x], sl1 = tp.cta_slot_ptr[blockIdx.x + 1];
    if (warp == 0) tc::tmem_alloc(s_tmem, 512);
    if (tid == 0) {
        tc::mbar_init(&mma_bar[0], 1);
        tc::mbar_init(&mma_bar[1], 1);
        tc::mbar_init(&ready[0], 8);
        tc::mbar_init(&ready[1], 8);
        for (int q = 0; q < RSTAGES; ++q) {
            tc::mbar_init(&full[q], 1);
            tc::mbar_init(&empty[q], 8);
        }
        tc::fence_mbar_init();
        *s_fail = 0;
        *s_issued = 0;
        *s_consumed = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tb = *s_tmem;

    if (warp == 8) {
        // producer: this CTA's item records, 32 at a time (one per lane), each chunk
        // staged RSTAGES ahead of its use, an end-of-slot marker after each slot
        const uint64_t pol = tc::policy_evict_first();
        const int r0 = tp.cta_rec_ptr[blockIdx.x], r1 = tp.cta_rec_ptr[blockIdx.x + 1];
        int si = sl0;
        int m = si < sl1 ? p.leaf_m[p.slot_leaf[tp.cta_slots[si]]] : 0;
        uint32_t g = 0;
        bool ok = true;
        for (int base = r0; base < r1 && ok; base += 32) {
            int4 rec[4] = {make_int4(0, 0, 0, 0), make_int4(0, 0, 0, 0), make_int4(0, 0, 0, 0),
                           make_int4(0, 0, 0, 0)};
            if (base + lane < r1) {
                const int4* rp = reinterpret_cast<const int4*>(tp.recs + base + lane);
#pragma unroll
                for (int q = 0; q < 4; ++q) rec[q] = __ldg(rp + q);
            }
            const int cnt = min(32, r1 - base);
            for (int i = 0; i < cnt && ok; ++i) {
                TcItem it;
                int kind;
                tc_item_from_rec(rec, i, p, a.near, a.arena, tp.xp, tp.t, m, it, kind);
                const int np = max(it.npair[0], max(it.npair[1], it.npair[2]));
                const int nch = kind == 2 ? 1 : (np + 3) >> 2;
                for (int c = 0; c < nch && ok; ++c, ++g) {
                    const int sidx = g % RSTAGES;
                    if (lane == 0) {
                        // s_fail is set once the builders have given up; a producer that
                        // stops leaves their bounded waits to run out
                        if (*(volatile int*)s_fail ||
                            !tc::mbar_wait(&empty[sidx], ((g / RSTAGES) & 1) ^ 1, WAIT_LIMIT)) {
                            ok = false;
                        } else if (kind == 2) {
                            TcHdr h = {};
                            h.kind = 1;
                            hdr[sidx] = h;
                            tc::mbar_arrive_expect_tx(&full[sidx], 0);
                        } else {
                            stage_chunk(it, c, stages + sidx * R_STAGE_BYTES, &hdr[sidx], &full[sidx], pol);
                        }
                        if (ok) *(volatile int*)s_issued = (int)(g + 1);
                    }
                    ok = __shfl_sync(0xffffffffu, ok, 0);
                }
                if (kind == 2 && ++si < sl1) m = p.leaf_m[p.slot_leaf[tp.cta_slots[si]]];
            }
        }
    } else if (warp == 9) {
        // issuer: waits for each chunk's operands (buffer header from the builders) and starts its MMAs
        uint32_t chunk = 0;
        bool failed = false;  // a wait ran out: issue nothing more (the builders' waits then run out too)
        for (int k = sl0; k < sl1; ++k) {
            for (;; ++chunk) {
                const int buf = chunk & 1;
                if (lane == 0 && !failed && !tc::mbar_wait(&ready[buf], (chunk >> 1) & 1, WAIT_LIMIT))
                    failed = true;
                int kind = 1;
                if (lane == 0 && !failed) {
                    tc::fence_after_sync();
                    const TcHdr h = hdrb[buf];
                    kind = h.kind;
                    if (kind == 0)
                        for (int s = 0; s < h.ks; ++s) rows_step_mma(tb, buf, s, tiles + (buf * RKS + s) * R_TILE_BYTES, h);
                    tc::mma_commit(&mma_bar[buf]);
                }
                kind = __shfl_sync(0xffffffffu, kind, 0);
                if (kind == 1) {
                    ++chunk;
                    break;
                }
            }
            if (tc::named_sync_or(BAR_DECIDE, NBUILD + 32, failed)) break;
        }
    } else {
        // builders (warps 0-7)
        uint32_t chunk = 0;  // chunks consumed (= stage sequence number; operand buffer = chunk & 1)
        const int row = 16 * (warp & 3) + (lane >> 1), dpart = lane & 1;
        bool failed = false;   // this thread's bounded wait ran out
        bool aborted = false;  // some builder's did (the same for all: barrier OR)
        for (int k = sl0; k < sl1; ++k) {
            const int slot = tp.cta_slots[k];
            const int leaf = p.slot_leaf[slot], part = p.slot_part[slot];
            const int P = p.leaf_parts[leaf];
            const int r0 = p.leaf_r0[leaf], m = p.leaf_m[leaf];
            float rj[32], rm[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) rj[j] = rm[j] = 0.f;
            flush_rows(tb, warp, rj, rm);  // clears the accumulators
#pragma unroll
            for (int j = 0; j < 32; ++j) rj[j] = rm[j] = 0.f;
            int since = 0;
            for (;; ++chunk) {
                const int buf = chunk & 1, sidx = chunk % RSTAGES;
                // move the accumulators into registers before this chunk's MMAs (after its
                // operands are built, so that the build overlaps the previous chunk's MMAs)
                const bool do_flush = since >= FLUSH_STEPS;
                if (do_flush) since = 0;
                // after a failure the builders keep the arrival protocol but do no work
                if (!failed && chunk >= 2 && !tc::mbar_wait(&mma_bar[buf], ((chunk >> 1) - 1) & 1, WAIT_LIMIT))
                    failed = true;
                if (!failed && !tc::mbar_wait(&full[sidx], (chunk / RSTAGES) & 1, WAIT_LIMIT)) failed = true;
                TcHdr h = {};
                h.kind = 1;
                if (!failed) h = hdr[sidx];
                const unsigned char* st = stages + sidx * R_STAGE_BYTES;
                if (!failed && h.kind == 0) {
                    const int ks = h.ks;
                    since += ks;
                    if (warp < 4) {
                        float4 v[RKS][3];
#pragma unroll
                        for (int s = 0; s < RKS; ++s)
#pragma unroll
                            for (int q = 0; q < 3; ++q) {
                                const int pl = 2 * s + dpart;  // this lane's pair within the chunk
                                v[s][q] = make_float4(0.f, 0.f, 0.f, 0.f);
                                if (s < ks && row < m && pl < h.npr[q])
                                    v[s][q] = reinterpret_cast<const float4*>(st + q * 4096)[pl * h.ld + row];
                            }
#pragma unroll
                        for (int s = 0; s < RKS; ++s) {
                            if (s >= ks) break;
#pragma unroll
                            for (int q = 0; q < 3; ++q) {
                                const float4 o = shfl4_xor(v[s][q], 1);
                                const float4 p0 = dpart ? o : v[s][q], p1 = dpart ? v[s][q] : o;
                                uint32_t hi[8], lo[8];
                                embed_split(p0, p1, dpart, hi, lo);
                                tc::tmem_st8(tc::taddr(tb, 32 * warp, a_col(buf, s, q, 0)), hi);
                                tc::tmem_st8(tc::taddr(tb, 32 * warp, a_col(buf, s, q, 1)), lo);
                            }
                        }
                        tc::tmem_st_wait();
                    } else {
                        const float2* sv = reinterpret_cast<const float2*>(st + R_OP_BYTES);
                        const int t = tid - 128;
                        for (int s = 0; s < ks; ++s) {
                            unsigned char* tile = tiles + (buf * RKS + s) * R_TILE_BYTES;
                            const int jl = 4 * s;
                            if (h.far) {
                                build_b_rows(tile, R_GROUPS, sv + 0 * 512, jl, jl, h.nrow[0], t, 0, -1);
                                build_b_rows(tile, R_GROUPS, sv + 1 * 512, jl, jl, h.nrow[1], t, 2, -1);
                                build_b_rows(tile, R_GROUPS, sv + 2 * 512, jl, jl, h.nrow[2], t, 6, -1);
                                build_b_rows(tile, R_GROUPS, sv + 3 * 512, jl, jl, h.nrow[3], t, -1, 4);
                            } else {
                                build_b_rows(tile, R_GROUPS, sv + 0 * 512, jl, jl, h.nrow[0], t, 0, 4);
                                build_b_rows(tile, R_GROUPS, sv + 1 * 512, jl, jl, h.nrow[1], t, 2, -1);
                            }
                        }
                        tc::fence_async_smem();
                    }
                }
                if (do_flush && h.kind == 0) {
                    if (!failed) {
                        const uint32_t last = chunk - 1;  // since > 0: an earlier chunk of this slot
                        if (!tc::mbar_wait(&mma_bar[last & 1], (last >> 1) & 1, WAIT_LIMIT)) failed = true;
                    }
                    tc::fence_after_sync();
                    if (!failed) flush_rows(tb, warp, rj, rm);
                }
                if (tid == 0) hdrb[buf] = h;  // for the issuer (kind 1 also after a failure: end of slot)
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) {
                    tc::mbar_arrive(&empty[sidx]);  // this warp is done with the stage
                    tc::mbar_arrive(&ready[buf]);   // and with the chunk's operands
                }
                if (h.kind == 1) {
                    ++chunk;
                    break;
                }
            }
            if (chunk > 0 && !failed) {
                const uint32_t last = chunk - 1;  // the end marker's commit: every MMA of the slot is done
                if (!tc::mbar_wait(&mma_bar[last & 1], (last >> 1) & 1, WAIT_LIMIT)) failed = true;
            }
            tc::fence_after_sync();
            if (tc::named_sync_or(BAR_DECIDE, NBUILD + 32, failed)) {
                aborted = true;
                break;
            }
            // epilogue: every builder warp adds its share of the accumulators (lanes of its
            // quadrant, 32 columns) to its register sums and writes rows (row, dpart)
            {
                float vj[32], vm[32];
                const uint32_t ln = 32 * (warp & 3), cb = 32 * (warp >> 2);
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    float x0[16], x1[16];
                    tc::tmem_ld16(tc::taddr(tb, ln, COL_JH + cb + 16 * hh), x0);
                    tc::tmem_ld16(tc::taddr(tb, ln, COL_JL + cb + 16 * hh), x1);
#pragma unroll
                    for (int j = 0; j < 16; ++j) vj[16 * hh + j] = rj[16 * hh + j] + (x0[j] + x1[j]);
                    tc::tmem_ld16(tc::taddr(tb, ln, COL_MH + cb + 16 * hh), x0);
                    tc::tmem_ld16(tc::taddr(tb, ln, COL_ML + cb + 16 * hh), x1);
#pragma unroll
                    for (int j = 0; j < 16; ++j) vm[16 * hh + j] = rm[16 * hh + j] + (x0[j] + x1[j]);
                }
                const bool act = row < m;
                const int64_t pos = r0 + row;
                const int64_t e = act ? p.perm[pos] : 0;
                float* yf = reinterpret_cast<float*>(a.y);
                float* pf = reinterpret_cast<float*>(tp.ypart);
                if (act) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int r = 32 * (warp >> 2) + j;
                        if (P == 1) {
                            if (r < a.nr) {
                                yf[2 * (r * nn + e) + dpart] = vj[j];
                                yf[2 * (r * nn + ne + e) + dpart] = vm[j];
                            }
                        } else {
                            pf[2 * (((int64_t)part * NR + r) * nn + pos) + dpart] = vj[j];
                            pf[2 * (((int64_t)part * NR + r) * nn + ne + pos) + dpart] = vm[j];
                        }
                    }
                }
            }
            if (P > 1) {
                __threadfence();
                tc::named_sync(BAR_BUILD, NBUILD);
                if (tid == 0) *s_last = (atomicAdd(p.arrive + leaf, 1u) == (unsigned)(P - 1));
                tc::named_sync(BAR_BUILD, NBUILD);
                if (*(volatile int*)s_last) {
                    __threadfence();
                    // sum the parts in index order (independent of which slot finished last)
                    for (int idx = tid; idx < 2 * m * a.nr; idx += NBUILD) {
                        const int i = idx % m, r = (idx / m) % a.nr, hh = idx / (m * a.nr);
                        const int64_t pos = (int64_t)hh * ne + r0 + i;
                        c64 sm = mk<float>(0.f, 0.f);
                        for (int q = 0; q < P; ++q) {
                            const float2 v =
                                __ldcg(reinterpret_cast<const float2*>(tp.ypart + ((int64_t)q * NR + r) * nn + pos));
                            sm.re += v.x;
                            sm.im += v.y;
                        }
                        a.y[r * nn + (int64_t)hh * ne + p.perm[r0 + i]] = sm;
                    }
                    if (tid == 0) p.arrive[leaf] = 0u;  // ready for the next pass
                }
                tc::named_sync(BAR_BUILD, NBUILD);
            }
            tc::fence_before_sync();
        }
        // the tensor core must have finished before its memory is released
        if (aborted && chunk > 0 && tid == 0) {
            const uint32_t last = chunk - 1;
            (void)tc::mbar_wait(&mma_bar[last & 1], (last >> 1) & 1, WAIT_LIMIT);
        }
        if (tid == 0) {
            *s_consumed = (int)chunk;
            if (aborted) *s_fail = 1;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (*(volatile int*)s_fail) {
        // stages issued but never consumed: wait (bounded) for their copies to land
        if (tid == 0) {
            atomicExch(tp.err, 1);
            for (int g = *s_consumed; g < *(volatile int*)s_issued; ++g)
                (void)tc::mbar_wait(&full[g % RSTAGES], (g / RSTAGES) & 1, WAIT_LIMIT);
        }
        __syncthreads();
    }
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tb, 512);
        tc::tmem_relinquish();
    }
}

// ---- t = W^T x -----------------------------------------------------------------
struct TcVhxArgs {
    TcPlan tp;
    int ne;
};

__global__ void __launch_bounds__(THREADS, 1) k_tc_vhx(TcVhxArgs va) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const TcPlan& a = va.tp;
    const int tk0 = a.vcta_ptr[blockIdx.x], tk1 = a.vcta_ptr[blockIdx.x + 1];
    unsigned char* tiles = smem;
    unsigned char* stages = smem + V_TILES_BYTES;
    float* out = reinterpret_cast<float*>(stages + VSTAGES * V_STAGE_BYTES);
    uint64_t* bar = reinterpret_cast<uint64_t*>(out + V_OUT_FLOATS);
    uint64_t* mma_bar = bar;
    uint64_t* full = bar + 2;
    uint64_t* empty = full + VSTAGES;
    uint64_t* ready = empty + VSTAGES;
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(ready + 2);
    int* s_fail = reinterpret_cast<int*>(s_tmem + 1);
    int* s_issued = s_fail + 1;
    int* s_consumed = s_fail + 2;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(s_tmem, 512);
    if (tid == 0) {
        tc::mbar_init(&mma_bar[0], 1);
        tc::mbar_init(&mma_bar[1], 1);
        tc::mbar_init(&ready[0], 8);
        tc::mbar_init(&ready[1], 8);
        for (int q = 0; q < VSTAGES; ++q) {
            tc::mbar_init(&full[q], 1);
            tc::mbar_init(&empty[q], 8);
        }
        tc::fence_mbar_init();
        *s_fail = 0;
        *s_issued = 0;
        *s_consumed = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tb = *s_tmem;
    if (warp == 8) {
        // producer: chunk c of a task stages columns [VCOLS c, VCOLS c + VCOLS) of its
        // W pairs from the task-major copy ([column][32 pairs] x 16 bytes, one copy)
        // and of its vector rows
        if (lane == 0) {
            const uint64_t pol = tc::policy_evict_first();
            uint32_t g = 0;
            bool ok = true;
            for (int k = tk0; k < tk1 && ok; ++k) {
                const TcVhxTask T = a.tasks[k];
                const int nch = (T.n + VCOLS - 1) / VCOLS;
                const c64* xv = a.xp + ((int64_t)T.g * va.ne + T.c0) * NR;
                for (int c = 0; c < nch; ++c, ++g) {
                    const int sidx = g % VSTAGES;
                    if (*(volatile int*)s_fail || !tc::mbar_wait(&empty[sidx], ((g / VSTAGES) & 1) ^ 1, WAIT_LIMIT)) {
                        ok = false;
                        break;
                    }
                    unsigned char* st = stages + sidx * V_STAGE_BYTES;
                    const int ncol = min(VCOLS, T.n - VCOLS * c);
                    const uint32_t xbytes = (uint32_t)ncol * NR * 8;
                    tc::mbar_arrive_expect_tx(&full[sidx], (uint32_t)V_W_BYTES + xbytes);
                    tc::bulk_g2s_hint(st, a.wcopy + T.wcopy + (int64_t)c * VCOLS * 32, (uint32_t)V_W_BYTES, &full[sidx],
                                      pol);
                    tc::bulk_g2s(st + V_W_BYTES, xv + (int64_t)VCOLS * c * NR, xbytes, &full[sidx]);
                    *(volatile int*)s_issued = (int)(g + 1);
                }
            }
        }
    } else if (warp == 9) {
        uint32_t chunk = 0;
        bool failed = false;
        const uint32_t id64 = tc::idesc_tf32(128, 64), id128 = tc::idesc_tf32(128, 128);
        for (int k = tk0; k < tk1; ++k) {
            const TcVhxTask T = a.tasks[k];
            const int nch = (T.n + VCOLS - 1) / VCOLS, nsteps = (T.n + 3) >> 2;
            for (int c = 0; c < nch; ++c, ++chunk) {
                const int buf = chunk & 1;
                if (lane == 0 && !failed && !tc::mbar_wait(&ready[buf], (chunk >> 1) & 1, WAIT_LIMIT)) failed = true;
                if (lane == 0 && !failed) {
                    tc::fence_after_sync();
                    const int ks = min(VKS, nsteps - VKS * c);
                    for (int s = 0; s < ks; ++s) {
                        // tile rows: [hi (64), lo (64)] per K chunk; LBO = 128 rows
                        const uint64_t d = tc::sdesc(tc::smem_u32(tiles + (buf * VKS + s) * V_TILE_BYTES),
                                                     2 * TILE_ROWS_BYTES, 128);
                        tc::mma_tf32_ts(tb + VCOL_DH, tb + va_col(buf, s, 0), d, id128, 1);  // hi x [hi, lo]
                        tc::mma_tf32_ts(tb + VCOL_DL, tb + va_col(buf, s, 1), d, id64, 1);   // lo x hi
                    }
                    tc::mma_commit(&mma_bar[buf]);
                }
                __syncwarp();
            }
            if (tc::named_sync_or(BAR_DECIDE, NBUILD + 32, failed)) break;
        }
    } else {
        uint32_t chunk = 0;
        bool failed = false, aborted = false;  // as in the rows kernel
        // warps 0-3: TMEM lane 32 warp + lane = (rank slot 16 warp + lane / 2, part lane & 1),
        // rank slot k = 2 pair + hh
        const int pr = 8 * (warp & 3) + (lane >> 2);
        const int hh = (lane >> 1) & 1, dpart = lane & 1;
        // warp w owns lanes 32 (w & 3) .. + 31 and columns 32 (w >> 2) .. + 31 of the accumulator
        const uint32_t ln = 32 * (warp & 3), cb = 32 * (warp >> 2);
        for (int k = tk0; k < tk1; ++k) {
            const TcVhxTask T = a.tasks[k];
            const int nch = (T.n + VCOLS - 1) / VCOLS;
            const int nsteps = (T.n + 3) >> 2;
            float acc[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[j] = 0.f;
            auto clear_d = [&]() {
                const uint32_t z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
                for (uint32_t c = 0; c < 32; c += 8) {
                    tc::tmem_st8(tc::taddr(tb, ln, VCOL_DH + cb + c), z);
                    tc::tmem_st8(tc::taddr(tb, ln, VCOL_DL + cb + c), z);
                }
                tc::tmem_st_wait();
            };
            auto take_d = [&]() {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float x0[16], x1[16];
                    tc::tmem_ld16(tc::taddr(tb, ln, VCOL_DH + cb + 16 * h), x0);
                    tc::tmem_ld16(tc::taddr(tb, ln, VCOL_DL + cb + 16 * h), x1);
#pragma unroll
                    for (int j = 0; j < 16; ++j) acc[16 * h + j] += x0[j] + x1[j];
                }
            };
            clear_d();
            int since = 0;
            for (int c = 0; c < nch; ++c, ++chunk) {
                const int ks = min(VKS, nsteps - VKS * c);
                const bool do_flush = since >= VFLUSH_STEPS;  // as in the rows kernel: after the build
                if (do_flush) since = 0;
                since += ks;
                const int buf = chunk & 1, sidx = chunk % VSTAGES;
                if (!failed && chunk >= 2 && !tc::mbar_wait(&mma_bar[buf], ((chunk >> 1) - 1) & 1, WAIT_LIMIT))
                    failed = true;
                if (!failed && !tc::mbar_wait(&full[sidx], (chunk / VSTAGES) & 1, WAIT_LIMIT)) failed = true;
                const unsigned char* st = stages + sidx * V_STAGE_BYTES;
                if (!failed) {
                    // warps w and w + 4 share TMEM quadrant w: w embeds the W rows of the even
                    // K steps and builds the vector tiles of the odd ones, w + 4 the reverse
                    const int par = warp < 4 ? 0 : 1;
                    const float4* wp = reinterpret_cast<const float4*>(st) + pr;  // column jl at wp[32 jl]
                    const bool pv = pr < T.npairs;
#pragma unroll
                    for (int s = 0; s < VKS; ++s) {
                        if (s >= ks) break;
                        if ((s & 1) != par) continue;
                        // W[j, 2 pair + hh] for the 4 columns j of this K step
                        float2 w4[4];
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) {
                            const int jl = 4 * s + jj;
                            w4[jj] = make_float2(0.f, 0.f);
                            if (pv && VCOLS * c + jl < T.n) {
                                const float4 v = wp[32 * jl];
                                w4[jj] = hh ? make_float2(v.z, v.w) : make_float2(v.x, v.y);
                            }
                        }
                        uint32_t hi[8], lo[8];
                        embed_split(make_float4(w4[0].x, w4[0].y, w4[1].x, w4[1].y),
                                    make_float4(w4[2].x, w4[2].y, w4[3].x, w4[3].y), dpart, hi, lo);
                        tc::tmem_st8(tc::taddr(tb, 32 * (warp & 3), va_col(buf, s, 0)), hi);
                        tc::tmem_st8(tc::taddr(tb, 32 * (warp & 3), va_col(buf, s, 1)), lo);
                    }
                    const float2* xs = reinterpret_cast<const float2*>(st + V_W_BYTES);
                    for (int s = 1 - par; s < ks; s += 2)
                        build_b_rows(tiles + (buf * VKS + s) * V_TILE_BYTES, 2, xs, 4 * s, VCOLS * c + 4 * s, T.n,
                                     tid & 127, 0, -1);
                    tc::tmem_st_wait();
                    tc::fence_async_smem();
                }
                if (do_flush) {
                    const uint32_t last = chunk - 1;
                    if (!failed && !tc::mbar_wait(&mma_bar[last & 1], (last >> 1) & 1, WAIT_LIMIT)) failed = true;
                    tc::fence_after_sync();
                    if (!failed) {
                        take_d();
                        clear_d();
                    }
                }
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) {
                    tc::mbar_arrive(&empty[sidx]);  // this warp is done with the stage
                    tc::mbar_arrive(&ready[buf]);   // and with the chunk's operands
                }
            }
            if (chunk > 0 && !failed) {
                const uint32_t last = chunk - 1;
                if (!tc::mbar_wait(&mma_bar[last & 1], (last >> 1) & 1, WAIT_LIMIT)) failed = true;
            }
            tc::fence_after_sync();
            if (tc::named_sync_or(BAR_DECIDE, NBUILD + 32, failed)) {
                aborted = true;
                break;
            }
            take_d();
            {
                // lane (rank slot, part) -> [16 slots of the quadrant][NR][re, im]
                float* so = out + (warp & 3) * 16 * V_OUT_ROW;
                const int kl = lane >> 1;
#pragma unroll
                for (int j = 0; j < 32; ++j) so[kl * V_OUT_ROW + (cb + j) * 2 + dpart] = acc[j];
            }
            tc::named_sync(BAR_BUILD, NBUILD);
            if (warp < 4) {
                const float* so = out + warp * 16 * V_OUT_ROW;
                // 16 rank rows of 512 bytes each, one row per step of the warp
                for (int kl2 = 0; kl2 < 16; ++kl2) {
                    const int pp = 8 * warp + (kl2 >> 1);
                    if (pp >= T.npairs) break;
                    const int64_t trow = a.pairs[T.pair0 + pp].trow + (kl2 & 1);
                    const float2* src = reinterpret_cast<const float2*>(so + kl2 * V_OUT_ROW) + 2 * lane;
                    const float2 u0 = src[0], u1 = src[1];
                    reinterpret_cast<float4*>(a.t + trow * NR)[lane] = make_float4(u0.x, u0.y, u1.x, u1.y);
                }
            }
            tc::fence_before_sync();
            tc::named_sync(BAR_BUILD, NBUILD);
        }
        if (aborted && chunk > 0 && tid == 0) {
            const uint32_t last = chunk - 1;
            (void)tc::mbar_wait(&mma_bar[last & 1], (last >> 1) & 1, WAIT_LIMIT);
        }
        if (tid == 0) {
            *s_consumed = (int)chunk;
            if (aborted) *s_fail = 1;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (*(volatile int*)s_fail) {
        if (tid == 0) {
            atomicExch(a.err, 1);
            for (int g = *s_consumed; g < *(volatile int*)s_issued; ++g)
                (void)tc::mbar_wait(&full[g % VSTAGES], (g / VSTAGES) & 1, WAIT_LIMIT);
        }
        __syncthreads();
    }
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tb, 512);
        tc::tmem_relinquish();
    }
}

// ---- task-major copy of the W factors -----------------------------------------------
// One CTA per task: chunk c, column j, pair p of the task at wcopy + (32 c + j) 32 + p
// (16 bytes: W[j, 2 kp], W[j, 2 kp + 1] of the pair's block and part); zero for
// columns at or beyond n and pairs at or beyond npairs.
__global__ void k_tc_wcopy(const TcVhxTask* __restrict__ tasks, const TcPair* __restrict__ pairs,
                           const c64* __restrict__ arena, float4* __restrict__ wcopy) {
    const TcVhxTask T = tasks[blockIdx.x];
    const int nch = (T.n + 31) / 32;
    float4* out = wcopy + T.wcopy;
    for (int64_t e = threadIdx.x; e < (int64_t)nch * 1024; e += blockDim.x) {
        const int p = (int)(e & 31), j = (int)(e >> 5);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (p < T.npairs && j < T.n) v = reinterpret_cast<const float4*>(arena + pairs[T.pair0 + p].w)[j];
        out[e] = v;
    }
}

cudaError_t tc_build_wcopy(const TcVhxTask* tasks, int ntask, const TcPair* pairs, const c64* arena, float4* wcopy,
                           cudaStream_t st) {
    if (ntask <= 0) return cudaSuccess;
    k_tc_wcopy<<<ntask, 256, 0, st>>>(tasks, pairs, arena, wcopy);
    return cudaGetLastError();
}

// ---- gather ----------------------------------------------------------------------
// xp[(h ne + pos) NR + r] = x[r 2ne + h ne + perm[pos]] for r < nr, zero for nr <= r < NR
__global__ void k_tc_gather(const c64* __restrict__ x, const int64_t* __restrict__ perm, c64* __restrict__ xp, int ne,
                            int nr) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nn = 2 * (int64_t)ne;
    if (idx >= nn * NR) return;
    const int r = (int)(idx % NR);
    const int64_t pos = idx / NR;
    const int64_t h = pos >= ne ? 1 : 0, pp = pos - h * ne;
    c64 v = mk<float>(0.f, 0.f);
    if (r < nr) v = x[r * nn + h * ne + perm[pp]];
    xp[idx] = v;
}

cudaError_t matvec_tc_run(const MatvecPlan& p, const TcPlan& tp, const void* near, const void* arena, const c64* x,
                          c64* y, int nrhs, cudaStream_t st, const cudaEvent_t* ev) {
    BEM_CUDA_TRY(cudaFuncSetAttribute(k_tc_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, R_SMEM_BYTES));
    BEM_CUDA_TRY(cudaFuncSetAttribute(k_tc_vhx, cudaFuncAttributeMaxDynamicSharedMemorySize, V_SMEM_BYTES));
    const int64_t nn = 2 * (int64_t)p.ne;
    int pass = 0;
    for (int r = 0; r < nrhs; r += NR, ++pass) {
        const int nr = std::min(NR, nrhs - r);
        const cudaEvent_t* e = ev ? ev + 6 * pass : nullptr;
        if (e) BEM_CUDA_TRY(cudaEventRecord(e[0], st));
        const int64_t total = nn * NR;
        k_tc_gather<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(x + r * nn, p.perm, tp.xp, p.ne, nr);
        BEM_CUDA_TRY(cudaGetLastError());
        if (e) BEM_CUDA_TRY(cudaEventRecord(e[1], st));
        if (e) BEM_CUDA_TRY(cudaEventRecord(e[2], st));
        if (tp.ntask > 0) {
            TcVhxArgs va{tp, p.ne};
            k_tc_vhx<<<tp.nsm, THREADS, V_SMEM_BYTES, st>>>(va);
            BEM_CUDA_TRY(cudaGetLastError());
        }
        if (e) BEM_CUDA_TRY(cudaEventRecord(e[3], st));
        if (e) BEM_CUDA_TRY(cudaEventRecord(e[4], st));
        TcRowsArgs ra{p, tp, (const c64*)near, (const c64*)arena, y + r * nn, nr};
        k_tc_rows<<<tp.nsm, THREADS, R_SMEM_BYTES, st>>>(ra);
        BEM_CUDA_TRY(cudaGetLastError());
        if (e) BEM_CUDA_TRY(cudaEventRecord(e[5], st));
    }
    return cudaSuccess;
}

}  // namespace bem
