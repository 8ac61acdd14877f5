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
// memory; threads build them from the stored complex64 entries in registers, so
// the stored layout serves the single-vector kernels and these alike.  The vector
// blocks are the B operand in shared memory.  FP32 accuracy comes from the
// three-term TF32 split (tc.cuh): hi*hi + hi*lo + lo*hi.
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
//                   the split's main terms hi*hi and its corrections hi*lo + lo*hi go
//                   to separate accumulators in tensor memory, so the small terms
//                   are not rounded against the running sum of the large ones;
//                   partial rows of a leaf split over several slots are summed by
//                   the last slot to finish (arrival counter).
// Both tensor kernels are persistent (one CTA per SM, work taken from a counter),
// pipeline their operands through two buffers (threads build chunk c + 1 while the
// tensor core runs chunk c), and bound every wait: a wait that runs out sets *err,
// waits (bounded) for the work already issued, frees its tensor memory and returns.
#include "common.cuh"
#include "tc.cuh"

namespace bem {

namespace {

constexpr int NR = BEM_TC_NR;          // 64 right-hand sides per pass
constexpr uint32_t WAIT_LIMIT = 1u << 22;  // polls of an mbarrier before giving up

// ---- rows kernel ---------------------------------------------------------------
constexpr int RKS = 2;                 // K steps (4 complex columns each) per chunk
// The tensor core rounds its FP32 accumulation toward zero, so a long chain of
// MMAs into one accumulator drifts (measured: about 1e-5 of |y| after ~1000 steps);
// the accumulators are moved into FP32 registers (round to nearest) and cleared
// once at least this many K steps have gone into them.
constexpr int FLUSH_STEPS = 8;
constexpr int R_TILE_FLOATS = 64 * 8;  // one B tile: 64 vector rows x 8 K elements
constexpr int R_SMEM_TILES = 2 * RKS * 4 * 2;           // buffers x steps x operand slots x (hi, lo)
constexpr int R_SMEM_BYTES_TILES = R_SMEM_TILES * R_TILE_FLOATS * 4;  // 64 KiB
constexpr int R_SMEM_BYTES = 120 * 1024;  // more than half an SM: one CTA per SM (tensor memory)
// tensor-memory columns: accumulators of y_J and y_M, main (hi*hi) and correction
// terms, then two A buffers of RKS x 3 parts x (hi, lo) x 8
constexpr uint32_t COL_JH = 0, COL_JL = 64, COL_MH = 128, COL_ML = 192, COL_A = 256;
__device__ __forceinline__ uint32_t a_col(int buf, int s, int q, int h) {
    return COL_A + (uint32_t)((buf * RKS + s) * 48 + (q * 2 + h) * 8);
}
__device__ __forceinline__ int b_tile(int buf, int s, int o, int h) { return ((buf * RKS + s) * 4 + o) * 2 + h; }

// ---- V^H x kernel --------------------------------------------------------------
constexpr int VKS = 8;                 // K steps per chunk
constexpr int V_SMEM_BYTES_TILES = 2 * VKS * 2 * R_TILE_FLOATS * 4;  // 64 KiB
constexpr int V_STAGE_FLOATS = 4 * 16 * NR * 2;                      // 32 KiB epilogue staging
constexpr int V_SMEM_BYTES = 120 * 1024;
constexpr uint32_t VCOL_DH = 0, VCOL_DL = 64, VCOL_A = 128;
constexpr int VFLUSH_STEPS = 16;       // K steps between moves of the accumulator into registers
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

__device__ __forceinline__ float4 shfl4(const float4& v, int src) {
    float4 r;
    r.x = __shfl_sync(0xffffffffu, v.x, src);
    r.y = __shfl_sync(0xffffffffu, v.y, src);
    r.z = __shfl_sync(0xffffffffu, v.z, src);
    r.w = __shfl_sync(0xffffffffu, v.w, src);
    return r;
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

// Vector block of one K step into its B tiles (hi, lo): K index (jj, re/im) over 4
// rows base[jj * NR + r] of the vector array (rows beyond nvalid are zero), negated
// if neg; this thread (0..127 of the builder group) fills vector column r = t & 63,
// K half t >> 6.
__device__ __forceinline__ void build_b(float* sh, float* sl, const c64* __restrict__ base, int j0, int nvalid,
                                        int t, bool neg) {
    const int r = t & 63, kc = t >> 6;
    const int ja = j0 + 2 * kc, jb = ja + 1;
    float2 a = make_float2(0.f, 0.f), b = a;
    if (ja < nvalid) a = __ldg(reinterpret_cast<const float2*>(base + (int64_t)ja * NR + r));
    if (jb < nvalid) b = __ldg(reinterpret_cast<const float2*>(base + (int64_t)jb * NR + r));
    const float sg = neg ? -1.f : 1.f;
    float4 h, l;
    split4(make_float4(sg * a.x, sg * a.y, sg * b.x, sg * b.y), h, l);
    reinterpret_cast<float4*>(sh)[kc * 64 + r] = h;
    reinterpret_cast<float4*>(sl)[kc * 64 + r] = l;
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
// operand slots (rows at vec[o] + j * NR, nvec[o] valid rows; slot 3 enters negated).
struct TcItem {
    const float4* base[3];
    int ld, m, npair[3];
    const c64* vec[4];
    int nvec[4];
    bool far;
};

__device__ __forceinline__ void tc_item_of(const MatvecPlan& p, const c64* near, const c64* arena, const c64* xp,
                                           const c64* t, int item, int m, TcItem& it) {
    it.m = m;
    if (item >= 0) {
        const int n = p.near_n[item], c0 = p.near_c0[item];
        const c64* a = near + p.near_off[item];
        for (int q = 0; q < 3; ++q) {
            it.base[q] = reinterpret_cast<const float4*>(a + q * p.near_op_stride);
            it.npair[q] = (n + 1) >> 1;
        }
        it.ld = m;
        it.vec[0] = xp + (int64_t)c0 * NR;               // x_J (A)
        it.vec[1] = xp + ((int64_t)p.ne + c0) * NR;      // x_M (B into y_J, and C)
        it.vec[2] = it.vec[1];
        it.vec[3] = it.vec[0];                           // -x_J (B into y_M)
        it.nvec[0] = it.nvec[1] = it.nvec[2] = it.nvec[3] = n;
        it.far = false;
    } else {
        const PieceDesc d = p.pieces[-1 - item];
        for (int q = 0; q < 3; ++q) {
            it.base[q] = reinterpret_cast<const float4*>(arena + d.base[q]);
            it.npair[q] = d.kp[q];
        }
        it.ld = d.ld;
        const c64* tA = t + d.t_off * NR;
        const c64* tBJ = tA + (int64_t)2 * d.kp[0] * NR;
        const c64* tBM = tBJ + (int64_t)2 * d.kp[1] * NR;
        const c64* tC = tBM + (int64_t)2 * d.kp[1] * NR;
        it.vec[0] = tA;
        it.vec[1] = tBM;
        it.vec[2] = tC;
        it.vec[3] = tBJ;
        it.nvec[0] = 2 * d.kp[0];
        it.nvec[1] = it.nvec[3] = 2 * d.kp[1];
        it.nvec[2] = 2 * d.kp[2];
        it.far = true;
    }
}

struct TcRowsArgs {
    MatvecPlan p;
    const c64* near;
    const c64* arena;
    const c64* xp;     // [2ne][NR] tree order
    const c64* t;      // [t_len][NR]
    c64* y;            // caller layout, nr vectors
    c64* ypart;        // [pmax][NR][2ne] tree order
    int* next;         // work counter (zero before the launch)
    int* err;          // set to 1 when a wait runs out
    int nr;
};

__global__ void __launch_bounds__(256, 1) k_tc_rows(TcRowsArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    float* sB = reinterpret_cast<float*>(smem);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + R_SMEM_BYTES_TILES);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bar + 2);
    int* s_work = reinterpret_cast<int*>(s_tmem + 1);
    int* s_fail = s_work + 1;
    int* s_last = s_work + 2;
    const MatvecPlan& p = a.p;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ne = p.ne;
    const int64_t nn = 2 * (int64_t)ne;
    if (warp == 0) tc::tmem_alloc(s_tmem, 512);
    if (tid == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
        tc::fence_mbar_init();
        *s_fail = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tb = *s_tmem;
    const uint32_t idesc = tc::idesc_tf32(128, 64);
    uint32_t chunk = 0;  // chunks issued by this CTA (buffer = chunk & 1)
    // operator-row role of warps 0-3: TMEM lane 32 warp + lane = (row i, part d)
    const int row = 16 * (warp & 3) + (lane >> 1), dpart = lane & 1;
    for (;;) {
        if (tid == 0) *s_work = atomicAdd(a.next, 1);
        __syncthreads();
        const int k = *s_work;
        if (k >= p.nslot || *s_fail) break;
        const int slot = p.slot_order[k];
        const int leaf = p.slot_leaf[slot], part = p.slot_part[slot];
        const int P = p.leaf_parts[leaf];
        const int r0 = p.leaf_r0[leaf], m = p.leaf_m[leaf];
        float rj[32], rm[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) rj[j] = rm[j] = 0.f;
        flush_rows(tb, warp, rj, rm);  // clears the accumulators (they hold the last slot's finished sums)
#pragma unroll
        for (int j = 0; j < 32; ++j) rj[j] = rm[j] = 0.f;
        int since = 0;  // K steps in the accumulators since they were last cleared
        const int w0 = p.work_ptr[slot], w1 = p.work_ptr[slot + 1];
        for (int w = w0; w < w1 && !*s_fail; ++w) {
            if (since >= FLUSH_STEPS) {
                // drain, then move the accumulators into registers
                if (chunk > 0) {
                    const uint32_t last = chunk - 1;
                    if (!tc::mbar_wait(&bar[last & 1], (last >> 1) & 1, WAIT_LIMIT)) atomicExch(s_fail, 1);
                }
                tc::fence_after_sync();
                flush_rows(tb, warp, rj, rm);
                since = 0;
            }
            TcItem it;
            tc_item_of(p, a.near, a.arena, a.xp, a.t, p.work_item[w], m, it);
            const int np = max(it.npair[0], max(it.npair[1], it.npair[2]));
            const int nsteps = (np + 1) >> 1;
            since += nsteps;
            for (int s0 = 0; s0 < nsteps; s0 += RKS) {
                const int ks = min(RKS, nsteps - s0);
                const int buf = chunk & 1;
                if (chunk >= 2) {
                    // the tensor core must be done with this buffer (chunk - 2)
                    if (!tc::mbar_wait(&bar[buf], ((chunk >> 1) - 1) & 1, WAIT_LIMIT)) atomicExch(s_fail, 1);
                }
                if (warp < 4) {
                    // operator rows: loads of the whole chunk first, then embedding and stores
                    float4 v[RKS][3];
#pragma unroll
                    for (int s = 0; s < RKS; ++s)
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            const int pr = 2 * (s0 + s) + dpart;  // this lane's column pair
                            v[s][q] = make_float4(0.f, 0.f, 0.f, 0.f);
                            if (s < ks && row < m && pr < it.npair[q])
                                v[s][q] = __ldcs(it.base[q] + (int64_t)pr * it.ld + row);
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
                    // dense items: x_J, x_M, -x_J (slot 2 unused); far pieces: t_A, t_BM, t_C, -t_BJ
                    for (int s = 0; s < ks; ++s)
                        for (int o = 0; o < 4; ++o) {
                            if (o == 2 && !it.far) continue;
                            build_b(sB + b_tile(buf, s, o, 0) * R_TILE_FLOATS, sB + b_tile(buf, s, o, 1) * R_TILE_FLOATS,
                                    it.vec[o], 4 * (s0 + s), it.nvec[o], tid - 128, o == 3);
                        }
                    tc::fence_async_smem();
                }
                tc::fence_before_sync();
                __syncthreads();
                if (*s_fail) break;
                if (tid == 0) {
                    tc::fence_after_sync();
                    // product table: (operator part, vector slot, accumulator of the main terms;
                    // the corrections go 64 columns further)
                    const int pq[4] = {0, 1, 2, 1};
                    const int po[4] = {0, 1, it.far ? 2 : 1, 3};
                    const uint32_t pd[4] = {COL_JH, COL_JH, COL_MH, COL_MH};
                    for (int s = 0; s < ks; ++s) {
                        const int st = s0 + s;
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int q = pq[u];
                            if (2 * st >= it.npair[q]) continue;  // part exhausted (far pieces)
                            const float* bh = sB + b_tile(buf, s, po[u], 0) * R_TILE_FLOATS;
                            const float* bl = sB + b_tile(buf, s, po[u], 1) * R_TILE_FLOATS;
                            const uint64_t dh = tc::sdesc(tc::smem_u32(bh), 1024, 128);
                            const uint64_t dl = tc::sdesc(tc::smem_u32(bl), 1024, 128);
                            const uint32_t ah = tb + a_col(buf, s, q, 0), al = tb + a_col(buf, s, q, 1);
                            tc::mma_tf32_ts(tb + pd[u], ah, dh, idesc, 1);
                            tc::mma_tf32_ts(tb + pd[u] + 64, ah, dl, idesc, 1);
                            tc::mma_tf32_ts(tb + pd[u] + 64, al, dh, idesc, 1);
                        }
                    }
                    tc::mma_commit(&bar[buf]);
                }
                ++chunk;
            }
        }
        // all of this slot's contractions done
        if (chunk > 0) {
            const uint32_t last = chunk - 1;
            if (!tc::mbar_wait(&bar[last & 1], (last >> 1) & 1, WAIT_LIMIT)) atomicExch(s_fail, 1);
        }
        tc::fence_after_sync();
        __syncthreads();
        if (*s_fail) break;
        // epilogue: every warp adds its share of the accumulators (lanes of its
        // quadrant, 32 columns) to its register sums and writes rows (row, dpart)
        {
            float vj[32], vm[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) vj[j] = vm[j] = 0.f;
            {
                const uint32_t ln = 32 * (warp & 3), cb = 32 * (warp >> 2);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float x0[16], x1[16];
                    tc::tmem_ld16(tc::taddr(tb, ln, COL_JH + cb + 16 * h), x0);
                    tc::tmem_ld16(tc::taddr(tb, ln, COL_JL + cb + 16 * h), x1);
#pragma unroll
                    for (int j = 0; j < 16; ++j) vj[16 * h + j] = rj[16 * h + j] + (x0[j] + x1[j]);
                    tc::tmem_ld16(tc::taddr(tb, ln, COL_MH + cb + 16 * h), x0);
                    tc::tmem_ld16(tc::taddr(tb, ln, COL_ML + cb + 16 * h), x1);
#pragma unroll
                    for (int j = 0; j < 16; ++j) vm[16 * h + j] = rm[16 * h + j] + (x0[j] + x1[j]);
                }
            }
            const bool act = row < m;
            const int64_t pos = r0 + row;
            const int64_t e = act ? p.perm[pos] : 0;
            float* yf = reinterpret_cast<float*>(a.y);
            float* pf = reinterpret_cast<float*>(a.ypart);
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
            __syncthreads();
            if (tid == 0) *s_last = (atomicAdd(p.arrive + leaf, 1u) == (unsigned)(P - 1));
            __syncthreads();
            if (*s_last) {
                __threadfence();
                // sum the parts in index order (independent of which slot finished last)
                for (int idx = tid; idx < 2 * m * a.nr; idx += blockDim.x) {
                    const int i = idx % m, r = (idx / m) % a.nr, h = idx / (m * a.nr);
                    const int64_t pos = (int64_t)h * ne + r0 + i;
                    c64 s = mk<float>(0.f, 0.f);
                    for (int q = 0; q < P; ++q) {
                        const float2 v =
                            __ldcg(reinterpret_cast<const float2*>(a.ypart + ((int64_t)q * NR + r) * nn + pos));
                        s.re += v.x;
                        s.im += v.y;
                    }
                    a.y[r * nn + (int64_t)h * ne + p.perm[r0 + i]] = s;
                }
                if (tid == 0) p.arrive[leaf] = 0u;  // ready for the next pass
            }
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    // leave: the tensor core must have finished before its memory is released
    if (*s_fail && chunk > 0) {
        const uint32_t last = chunk - 1;
        if (tid == 0) {
            atomicExch(a.err, 1);
            (void)tc::mbar_wait(&bar[last & 1], (last >> 1) & 1, WAIT_LIMIT);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tb, 512);
        tc::tmem_relinquish();
    }
}

// ---- t = W^T x -----------------------------------------------------------------
struct TcVhxArgs {
    const TcVhxTask* tasks;
    const TcPair* pairs;
    int ntask;
    const c64* arena;
    const c64* xp;
    c64* t;
    int ne;
    int* next;
    int* err;
};

__global__ void __launch_bounds__(256, 1) k_tc_vhx(TcVhxArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    float* sB = reinterpret_cast<float*>(smem);
    float* stage = sB + 2 * VKS * 2 * R_TILE_FLOATS;
    uint64_t* bar = reinterpret_cast<uint64_t*>(stage + V_STAGE_FLOATS);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bar + 2);
    int* s_work = reinterpret_cast<int*>(s_tmem + 1);
    int* s_fail = s_work + 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(s_tmem, 512);
    if (tid == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
        tc::fence_mbar_init();
        *s_fail = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tb = *s_tmem;
    const uint32_t idesc = tc::idesc_tf32(128, 64);
    uint32_t chunk = 0;
    // warps 0-3: TMEM lane 32 warp + lane = (rank slot 16 warp + lane / 2, part lane & 1);
    // rank slot k = 2 pair + h; the 4 lanes of a pair load columns j = 4 s + (lane & 3)
    const int pr = 8 * (warp & 3) + (lane >> 2);
    const int hh = (lane >> 1) & 1, dpart = lane & 1, jsub = lane & 3;
    for (;;) {
        if (tid == 0) *s_work = atomicAdd(a.next, 1);
        __syncthreads();
        const int k = *s_work;
        if (k >= a.ntask || *s_fail) break;
        const TcVhxTask T = a.tasks[k];
        const c64* xv = a.xp + ((int64_t)T.g * a.ne + T.c0) * NR;
        const c64* wb = (warp < 4 && pr < T.npairs) ? a.arena + a.pairs[T.pair0 + pr].w : nullptr;
        const int nsteps = (T.n + 3) >> 2;
        // warp w owns lanes 32 (w & 3) .. + 31 and columns 32 (w >> 2) .. + 31 of the
        // accumulator; its register sums acc[] take the accumulator every VFLUSH_STEPS
        const uint32_t ln = 32 * (warp & 3), cb = 32 * (warp >> 2);
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
        for (int s0 = 0; s0 < nsteps; s0 += VKS) {
            const int ks = min(VKS, nsteps - s0);
            if (since >= VFLUSH_STEPS) {
                const uint32_t last = chunk - 1;
                if (!tc::mbar_wait(&bar[last & 1], (last >> 1) & 1, WAIT_LIMIT)) atomicExch(s_fail, 1);
                tc::fence_after_sync();
                take_d();
                clear_d();
                since = 0;
            }
            since += ks;
            const int buf = chunk & 1;
            if (chunk >= 2) {
                if (!tc::mbar_wait(&bar[buf], ((chunk >> 1) - 1) & 1, WAIT_LIMIT)) atomicExch(s_fail, 1);
            }
            if (warp < 4) {
                float4 v[VKS];
#pragma unroll
                for (int s = 0; s < VKS; ++s) {
                    const int j = 4 * (s0 + s) + jsub;
                    v[s] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (s < ks && wb && j < T.n) v[s] = __ldcs(reinterpret_cast<const float4*>(wb) + j);
                }
#pragma unroll
                for (int s = 0; s < VKS; ++s) {
                    if (s >= ks) break;
                    // W[4 s + jj, 2 pair + hh] from the lane of the group that loaded column jj
                    float4 g[4];
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) g[jj] = shfl4(v[s], (lane & ~3) | jj);
                    const float4 p0 = hh ? make_float4(g[0].z, g[0].w, g[1].z, g[1].w)
                                         : make_float4(g[0].x, g[0].y, g[1].x, g[1].y);
                    const float4 p1 = hh ? make_float4(g[2].z, g[2].w, g[3].z, g[3].w)
                                         : make_float4(g[2].x, g[2].y, g[3].x, g[3].y);
                    uint32_t hi[8], lo[8];
                    embed_split(p0, p1, dpart, hi, lo);
                    tc::tmem_st8(tc::taddr(tb, 32 * warp, va_col(buf, s, 0)), hi);
                    tc::tmem_st8(tc::taddr(tb, 32 * warp, va_col(buf, s, 1)), lo);
                }
                tc::tmem_st_wait();
            } else {
                for (int s = 0; s < ks; ++s)
                    build_b(sB + ((buf * VKS + s) * 2 + 0) * R_TILE_FLOATS, sB + ((buf * VKS + s) * 2 + 1) * R_TILE_FLOATS,
                            xv, 4 * (s0 + s), T.n, tid - 128, false);
                tc::fence_async_smem();
            }
            tc::fence_before_sync();
            __syncthreads();
            if (*s_fail) break;
            if (tid == 0) {
                tc::fence_after_sync();
                for (int s = 0; s < ks; ++s) {
                    const float* bh = sB + ((buf * VKS + s) * 2 + 0) * R_TILE_FLOATS;
                    const float* bl = sB + ((buf * VKS + s) * 2 + 1) * R_TILE_FLOATS;
                    const uint64_t dh = tc::sdesc(tc::smem_u32(bh), 1024, 128);
                    const uint64_t dl = tc::sdesc(tc::smem_u32(bl), 1024, 128);
                    const uint32_t ah = tb + va_col(buf, s, 0), al = tb + va_col(buf, s, 1);
                    tc::mma_tf32_ts(tb + VCOL_DH, ah, dh, idesc, 1);
                    tc::mma_tf32_ts(tb + VCOL_DL, ah, dl, idesc, 1);
                    tc::mma_tf32_ts(tb + VCOL_DL, al, dh, idesc, 1);
                }
                tc::mma_commit(&bar[buf]);
            }
            ++chunk;
        }
        if (chunk > 0) {
            const uint32_t last = chunk - 1;
            if (!tc::mbar_wait(&bar[last & 1], (last >> 1) & 1, WAIT_LIMIT)) atomicExch(s_fail, 1);
        }
        tc::fence_after_sync();
        __syncthreads();
        if (*s_fail) break;
        take_d();
        {
            // lane (rank slot, part) -> staging [16 slots of the quadrant][NR][re, im]
            float* st = stage + (warp & 3) * 16 * NR * 2;
            const int kl = lane >> 1;
#pragma unroll
            for (int j = 0; j < 32; ++j) st[(kl * NR + cb + j) * 2 + dpart] = acc[j];
        }
        __syncthreads();
        if (warp < 4) {
            const float* st = stage + warp * 16 * NR * 2;
            // 16 rank rows of 512 bytes each, one row per step of the warp
            for (int kl2 = 0; kl2 < 16; ++kl2) {
                const int pp = 8 * warp + (kl2 >> 1);
                if (pp >= T.npairs) break;
                const int64_t trow = a.pairs[T.pair0 + pp].trow + (kl2 & 1);
                const float4 v = reinterpret_cast<const float4*>(st + kl2 * NR * 2)[lane];
                reinterpret_cast<float4*>(a.t + trow * NR)[lane] = v;
            }
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    if (*s_fail && chunk > 0) {
        const uint32_t last = chunk - 1;
        if (tid == 0) {
            atomicExch(a.err, 1);
            (void)tc::mbar_wait(&bar[last & 1], (last >> 1) & 1, WAIT_LIMIT);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tb, 512);
        tc::tmem_relinquish();
    }
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
        BEM_CUDA_TRY(cudaMemsetAsync(tp.counters, 0, 2 * sizeof(int), st));
        if (e) BEM_CUDA_TRY(cudaEventRecord(e[2], st));
        if (tp.ntask > 0) {
            TcVhxArgs va{tp.tasks, tp.pairs, tp.ntask, (const c64*)arena, tp.xp, tp.t, p.ne, tp.counters, tp.err};
            k_tc_vhx<<<tp.nsm, 256, V_SMEM_BYTES, st>>>(va);
            BEM_CUDA_TRY(cudaGetLastError());
        }
        if (e) BEM_CUDA_TRY(cudaEventRecord(e[3], st));
        if (e) BEM_CUDA_TRY(cudaEventRecord(e[4], st));
        TcRowsArgs ra{p, (const c64*)near, (const c64*)arena, tp.xp, tp.t, y + r * nn, tp.ypart, tp.counters + 1,
                      tp.err, nr};
        k_tc_rows<<<tp.nsm, 256, R_SMEM_BYTES, st>>>(ra);
        BEM_CUDA_TRY(cudaGetLastError());
        if (e) BEM_CUDA_TRY(cudaEventRecord(e[5], st));
    }
    return cudaSuccess;
}

}  // namespace bem
