// Cluster tree and block tree on the GPU.
//
// The compressed product needs a partition of the operator into dense (near) and
// low-rank (far) blocks; the paper's skeleton U V^T (Eq. 17) is the global form of
// the same idea.  The partition is defined exactly (so results can be compared for
// equality):
//   * clusters are contiguous ranges of a permutation of the RWG edges; a cluster
//     larger than the leaf size is split at floor(size/2) after ordering its edge
//     midpoints by (coordinate on the axis of largest bounding-box extent, first
//     axis on ties; original edge index);
//   * a pair of clusters is admissible when min(diam^2) <= (eta*eta) * dist^2 with
//     dist^2 > 0 and eta > 0, diam^2 and dist^2 the sums ((x*x + y*y) + z*z) of the
//     bounding-box extents and box gaps; admissible pairs become far blocks, leaf
//     pairs near blocks, and the others recurse into the children of every
//     non-leaf side.
// The split positions depend only on the sizes, so the host lays out the node
// ranges; the GPU computes bounding boxes and the ordering.  All floating-point
// decisions use round-to-nearest intrinsics (no fused multiply-add) so they match
// a plain float64 evaluation exactly.
#include "common.cuh"

namespace bem {

__global__ void k_bbox(const double* __restrict__ pts, const int64_t* __restrict__ perm, const int* __restrict__ lo,
                       const int* __restrict__ hi, double* __restrict__ bbmin, double* __restrict__ bbmax) {
    int c = blockIdx.x;
    int a = lo[c], b = hi[c];
    double mn[3] = {INFINITY, INFINITY, INFINITY};
    double mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int k = a + threadIdx.x; k < b; k += blockDim.x) {
        const double* p = pts + 3 * perm[k];
        for (int d = 0; d < 3; ++d) {
            mn[d] = fmin(mn[d], p[d]);
            mx[d] = fmax(mx[d], p[d]);
        }
    }
    __shared__ double smn[3][32], smx[3][32];
    for (int d = 0; d < 3; ++d) {
        for (int o = 16; o > 0; o >>= 1) {
            mn[d] = fmin(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
            mx[d] = fmax(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
        }
    }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0)
        for (int d = 0; d < 3; ++d) {
            smn[d][w] = mn[d];
            smx[d][w] = mx[d];
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        int nw = (blockDim.x + 31) >> 5;
        for (int d = 0; d < 3; ++d) {
            double a0 = smn[d][0], b0 = smx[d][0];
            for (int i = 1; i < nw; ++i) {
                a0 = fmin(a0, smn[d][i]);
                b0 = fmax(b0, smx[d][i]);
            }
            bbmin[3 * c + d] = a0;
            bbmax[3 * c + d] = b0;
        }
    }
}

cudaError_t tree_bbox_level(const double* pts, const int64_t* perm, const int* lo, const int* hi, int ncl,
                            double* bbmin, double* bbmax, cudaStream_t st) {
    if (ncl <= 0) return cudaSuccess;
    k_bbox<<<ncl, 256, 0, st>>>(pts, perm, lo, hi, bbmin, bbmax);
    return cudaGetLastError();
}

__device__ __forceinline__ int longest_axis(const double* mn, const double* mx) {
    double e0 = __dsub_rn(mx[0], mn[0]), e1 = __dsub_rn(mx[1], mn[1]), e2 = __dsub_rn(mx[2], mn[2]);
    int ax = 0;
    double best = e0;
    if (e1 > best) {
        best = e1;
        ax = 1;
    }
    if (e2 > best) ax = 2;
    return ax;
}

// Rank of every position inside its splitting cluster, by exact counting.
// pos_cl[k] = cluster (index into lo/hi/bbmin/bbmax) of position k, or -1 to copy.
__global__ void k_split(const double* __restrict__ pts, const int64_t* __restrict__ perm_in,
                        int64_t* __restrict__ perm_out, const int* __restrict__ lo, const int* __restrict__ hi,
                        const double* __restrict__ bbmin, const double* __restrict__ bbmax,
                        const int* __restrict__ splits, const int* __restrict__ pos_cl, int n) {
    __shared__ double skey[256];
    __shared__ int64_t sidx[256];
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    int c = (k < n) ? pos_cl[k] : -1;
    bool active = (c >= 0) && splits[c];
    int ax = 0, a = 0, b = 0;
    double key = 0.0;
    int64_t idx = 0;
    if (active) {
        ax = longest_axis(bbmin + 3 * c, bbmax + 3 * c);
        a = lo[c];
        b = hi[c];
        idx = perm_in[k];
        key = pts[3 * idx + ax];
    }
    // do all threads of this CTA share one cluster? then stage tiles in shared memory
    int c_first = pos_cl[min(blockIdx.x * blockDim.x, n - 1)];
    int c_last = pos_cl[min(blockIdx.x * blockDim.x + blockDim.x - 1, n - 1)];
    bool uniform = (c_first == c_last) && (c_first >= 0) && splits[c_first];
    int rank = 0;
    if (uniform) {
        int ua = lo[c_first], ub = hi[c_first];
        int uax = longest_axis(bbmin + 3 * c_first, bbmax + 3 * c_first);
        for (int t0 = ua; t0 < ub; t0 += blockDim.x) {
            int q = t0 + threadIdx.x;
            if (q < ub) {
                int64_t iq = perm_in[q];
                sidx[threadIdx.x] = iq;
                skey[threadIdx.x] = pts[3 * iq + uax];
            }
            __syncthreads();
            int cnt = min((int)blockDim.x, ub - t0);
            if (active)
                for (int j = 0; j < cnt; ++j) {
                    double kq = skey[j];
                    rank += (kq < key) || (kq == key && sidx[j] < idx);
                }
            __syncthreads();
        }
    } else if (active) {
        for (int q = a; q < b; ++q) {
            int64_t iq = perm_in[q];
            double kq = pts[3 * iq + ax];
            rank += (kq < key) || (kq == key && iq < idx);
        }
    }
    if (k < n) {
        if (active)
            perm_out[a + rank] = idx;
        else
            perm_out[k] = perm_in[k];
    }
}

cudaError_t tree_split_level(const double* pts, const int64_t* perm_in, int64_t* perm_out, const int* lo,
                             const int* hi, const double* bbmin, const double* bbmax, const int* split_cl,
                             int nsplit, const int* pos_cl, int npos_total, cudaStream_t st) {
    (void)nsplit;
    int blocks = (npos_total + 255) / 256;
    k_split<<<blocks, 256, 0, st>>>(pts, perm_in, perm_out, lo, hi, bbmin, bbmax, split_cl, pos_cl, npos_total);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// block tree: classify candidate pairs, then emit by exclusive-scan offsets
// ---------------------------------------------------------------------------
__device__ __forceinline__ double sq3(double a, double b, double c) {
    return __dadd_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)), __dmul_rn(c, c));
}

// kind: 0 far, 1 near, 2 split t, 3 split s, 4 split both
__global__ void k_block_classify(const int* __restrict__ cand, int ncand, const int* __restrict__ child0,
                                 const double* __restrict__ bbmin, const double* __restrict__ bbmax, double eta,
                                 int* __restrict__ kind, int* __restrict__ c_far, int* __restrict__ c_near,
                                 int* __restrict__ c_next) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncand) return;
    int t = cand[2 * i], s = cand[2 * i + 1];
    const double *tn = bbmin + 3 * t, *tx = bbmax + 3 * t, *sn = bbmin + 3 * s, *sx = bbmax + 3 * s;
    bool adm = false;
    if (eta > 0.0) {
        double g[3];
        for (int d = 0; d < 3; ++d) g[d] = fmax(0.0, fmax(__dsub_rn(sn[d], tx[d]), __dsub_rn(tn[d], sx[d])));
        double dist2 = sq3(g[0], g[1], g[2]);
        if (dist2 > 0.0) {
            double dt = sq3(__dsub_rn(tx[0], tn[0]), __dsub_rn(tx[1], tn[1]), __dsub_rn(tx[2], tn[2]));
            double ds = sq3(__dsub_rn(sx[0], sn[0]), __dsub_rn(sx[1], sn[1]), __dsub_rn(sx[2], sn[2]));
            adm = fmin(dt, ds) <= __dmul_rn(__dmul_rn(eta, eta), dist2);
        }
    }
    bool tl = child0[t] < 0, sl = child0[s] < 0;
    int k, nf = 0, nn = 0, nx = 0;
    if (adm) {
        k = 0;
        nf = 1;
    } else if (tl && sl) {
        k = 1;
        nn = 1;
    } else if (tl) {
        k = 3;
        nx = 2;
    } else if (sl) {
        k = 2;
        nx = 2;
    } else {
        k = 4;
        nx = 4;
    }
    kind[i] = k;
    c_far[i] = nf;
    c_near[i] = nn;
    c_next[i] = nx;
}

__global__ void k_block_emit(const int* __restrict__ cand, int ncand, const int* __restrict__ kind,
                             const int* __restrict__ child0, const int* __restrict__ o_far,
                             const int* __restrict__ o_near, const int* __restrict__ o_next,
                             int* __restrict__ next_cand, int* __restrict__ near_out, int* __restrict__ far_out,
                             const int* __restrict__ nlo, const int* __restrict__ nhi) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncand) return;
    int t = cand[2 * i], s = cand[2 * i + 1];
    int k = kind[i];
    if (k == 0 || k == 1) {
        int* o = (k == 0) ? far_out + 4 * o_far[i] : near_out + 4 * o_near[i];
        o[0] = nlo[t];
        o[1] = nhi[t] - nlo[t];
        o[2] = nlo[s];
        o[3] = nhi[s] - nlo[s];
        return;
    }
    int* o = next_cand + 2 * o_next[i];
    if (k == 2) {
        int c = child0[t];
        o[0] = c; o[1] = s;
        o[2] = c + 1; o[3] = s;
    } else if (k == 3) {
        int c = child0[s];
        o[0] = t; o[1] = c;
        o[2] = t; o[3] = c + 1;
    } else {
        int ct = child0[t], cs = child0[s];
        o[0] = ct; o[1] = cs;
        o[2] = ct; o[3] = cs + 1;
        o[4] = ct + 1; o[5] = cs;
        o[6] = ct + 1; o[7] = cs + 1;
    }
}

// single-CTA exclusive scan (deterministic); total written to total_dev
__global__ void k_scan(const int* __restrict__ in, int* __restrict__ out, int n, int* __restrict__ total) {
    __shared__ int warp_sums[32];
    __shared__ int carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < n; base += blockDim.x) {
        int i = base + threadIdx.x;
        int v = (i < n) ? in[i] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[w] = x;
        __syncthreads();
        if (w == 0) {
            int nw = blockDim.x >> 5;
            int s = (lane < nw) ? warp_sums[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            warp_sums[lane] = s;  // inclusive prefix of warp totals
        }
        __syncthreads();
        int warp_off = (w > 0) ? warp_sums[w - 1] : 0;
        int carry = carry_s;
        if (i < n) out[i] = carry + warp_off + x - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry_s = carry + warp_off + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry_s;
}

cudaError_t scan_exclusive(const int* in, int* out, int n, int* total_dev, cudaStream_t st) {
    k_scan<<<1, 1024, 0, st>>>(in, out, n, total_dev);
    return cudaGetLastError();
}

cudaError_t tree_block_level(const int* cand, int ncand, const int* nlo, const int* nhi, const int* child0,
                             const double* bbmin, const double* bbmax, double eta, int* kind, int* counts,
                             cudaStream_t st) {
    (void)nlo;
    (void)nhi;
    if (ncand <= 0) return cudaSuccess;
    int blocks = (ncand + 255) / 256;
    k_block_classify<<<blocks, 256, 0, st>>>(cand, ncand, child0, bbmin, bbmax, eta, kind, counts,
                                             counts + ncand, counts + 2 * ncand);
    return cudaGetLastError();
}

// offs holds the three exclusive scans (far, near, next) back to back, each ncand long
cudaError_t tree_block_emit(const int* cand, int ncand, const int* kind, const int* child0, const int* offs,
                            int* next_cand, int* near_out, int* far_out, const int* nlo, const int* nhi,
                            cudaStream_t st) {
    if (ncand <= 0) return cudaSuccess;
    int blocks = (ncand + 255) / 256;
    k_block_emit<<<blocks, 256, 0, st>>>(cand, ncand, kind, child0, offs, offs + ncand, offs + 2 * ncand, next_cand,
                                         near_out, far_out, nlo, nhi);
    return cudaGetLastError();
}

}  // namespace bem
