// The compressed PMCHWT product y = Z x (Eq. 8's system matrix applied to a
// vector, with its far blocks in the skeleton form U V^H of Eq. 17).
//
// Data layout (all in HBM, written once by assembly):
//   near items   one per (leaf row cluster, dense column range); A, B, C arrays
//                op_stride apart; element (i, 2cp + h) at 2 (cp m + i) + h, so
//                that thread i of a 64-thread group reads one 16-byte (complex64)
//                pair per column pair and a warp reads 512 contiguous bytes;
//   far factors  per block and operator: U (m rows) and W = conj(V) (n rows),
//                the same column-pair layout; t = W^T x = V^H x.
// Kernels per product (one stream, in order):
//   1. gather  xp = x[perm]           (tree order; complex vector, L2-resident)
//   2. vhx     t_b = V_b^H xp_sigma   64-thread CTAs of 8 column-pair items (8 lanes
//                                      each), largest blocks first
//   3. rows    per leaf cluster tau:  y_tau = sum_near Z_{tau,sigma} xp_sigma
//                                             + sum_far U_b[tau rows] t_b
//              with the 2x2 PMCHWT structure [[A, B], [-B, C]] (B read once,
//              used in both rows); four 64-thread groups split the leaf's items
//              and are reduced in shared memory; y written once per row, in
//              edge order (deterministic, no atomics).
#include "common.cuh"

namespace bem {

// Double-float numbers: value hi + lo with two FP32 numbers (|lo| <= ulp(hi) / 2
// after each operation), about 44 significant bits.  They carry the FP64-sum form
// of the complex64 operator (BEM_FORM_C64_IN_FP64, the residuals of iterative
// refinement): FP32 entries times vectors kept to ~2^-44, summed with error-free
// transformations (Knuth's TwoSum, Dekker's FastTwoSum, the product error of one
// fused multiply-add) on the FP32 pipe instead of the GPU's much narrower FP64
// pipe.  A product a b keeps a.hi b.hi exactly and the cross terms to FP32; the
// lo * lo term (2^-48 relative) is dropped.
struct df {
    float hi, lo;
    df() = default;
    __host__ __device__ df(float h) : hi(h), lo(0.f) {}
    __host__ __device__ df(float h, float l) : hi(h), lo(l) {}
};
__device__ __forceinline__ df operator+(df a, df b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b.hi - bb);  // TwoSum: s + e = a.hi + b.hi exactly
    e += a.lo + b.lo;
    const float h = s + e;                     // FastTwoSum (|s| >= |e|)
    return df(h, e - (h - s));
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);            // exact rounding error of p
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float h = p + e;
    return df(h, e - (h - p));
}
__device__ __forceinline__ df& operator+=(df& a, df b) { return a = a + b; }
__device__ __forceinline__ df& operator-=(df& a, df b) { return a = a - b; }

// Products with a stored entry.  In every product below the entry is the left
// operand of `*` and the middle operand of cfma, and an entry is an FP32 value
// widened with lo = 0: these overloads skip its lo terms and keep each entry x
// vector product exact up to the vector's lo part (e = fma(b, hi, -p) is the exact
// error of p = b hi), accumulating with one TwoSum per term and one renormalisation
// per component.
__device__ __forceinline__ void df_acc(df& a, float b, df c, bool neg) {
    float p = b * c.hi;
    float e = fmaf(b, c.hi, -p);
    e = fmaf(b, c.lo, e);
    if (neg) {
        p = -p;
        e = -e;
    }
    const float s = a.hi + p;
    const float bb = s - a.hi;
    const float t = (a.hi - (s - bb)) + (p - bb);  // TwoSum
    a.hi = s;
    a.lo += t + e;
}
__device__ __forceinline__ void df_norm(df& a) {
    const float h = a.hi + a.lo;  // FastTwoSum
    a.lo = a.lo - (h - a.hi);
    a.hi = h;
}
__device__ __forceinline__ void cfma(cx<df>& a, cx<df> b, cx<df> c) {
    df_acc(a.re, b.re.hi, c.re, false);
    df_acc(a.re, b.im.hi, c.im, true);
    df_acc(a.im, b.re.hi, c.im, false);
    df_acc(a.im, b.im.hi, c.re, false);
    df_norm(a.re);
    df_norm(a.im);
}
__device__ __forceinline__ cx<df> operator*(cx<df> b, cx<df> c) {
    cx<df> a = mk<df>(df(0.f), df(0.f));
    cfma(a, b, c);
    return a;
}

// warp shuffles of the arithmetic types (a double-float moves as two floats)
template <typename T>
__device__ __forceinline__ T xshfl(unsigned mask, T v, int o) {
    return __shfl_xor_sync(mask, v, o);
}
template <>
__device__ __forceinline__ df xshfl<df>(unsigned mask, df v, int o) {
    return df(__shfl_xor_sync(mask, v.hi, o), __shfl_xor_sync(mask, v.lo, o));
}

// Element type of the caller's vectors for a product arithmetic R (double-float
// products read and write complex128) and the conversions at the boundary.
template <typename R>
struct Caller {
    using T = cx<R>;
    static __device__ __forceinline__ cx<R> in(T v) { return v; }
    static __device__ __forceinline__ T out(cx<R> v) { return v; }
};
template <>
struct Caller<df> {
    using T = c128;
    static __device__ __forceinline__ df split(double v) {
        const float h = (float)v;
        return df(h, (float)(v - (double)h));
    }
    static __device__ __forceinline__ cx<df> in(c128 v) { return mk<df>(split(v.re), split(v.im)); }
    static __device__ __forceinline__ c128 out(cx<df> v) {
        return mk<double>((double)v.re.hi + (double)v.re.lo, (double)v.im.hi + (double)v.im.lo);
    }
};

// Loads of two consecutive complex values of the stored operator, converted to
// the arithmetic R of the product.  Storage F: complex64 (one 16-byte load),
// complex128 (two), or BF16 pairs (one 8-byte load; far factors of the complex64
// product only).  The operator is read once per product, so the loads are marked
// streaming (evict-first): they must not push the reused vectors (x, t) out of L1
// and L2.
template <typename F>
struct FPair;
template <>
struct FPair<c64> {
    template <typename R>
    static __device__ __forceinline__ void ld(const c64* base, int64_t idx, cx<R>& a, cx<R>& b) {
        const float4 v = __ldcs(reinterpret_cast<const float4*>(base) + idx);
        a = mk<R>((R)v.x, (R)v.y);
        b = mk<R>((R)v.z, (R)v.w);
    }
};
template <>
struct FPair<c128> {
    template <typename R>
    static __device__ __forceinline__ void ld(const c128* base, int64_t idx, cx<R>& a, cx<R>& b) {
        const double2* p = reinterpret_cast<const double2*>(base) + 2 * idx;
        const double2 u = __ldcs(p), v = __ldcs(p + 1);
        a = mk<R>((R)u.x, (R)u.y);
        b = mk<R>((R)v.x, (R)v.y);
    }
};
template <>
struct FPair<bf16c> {
    template <typename R>
    static __device__ __forceinline__ void ld(const bf16c* base, int64_t idx, cx<R>& a, cx<R>& b) {
        const uint2 u = __ldcs(reinterpret_cast<const uint2*>(base) + idx);
        const float2 fa = bf16c_to_float2(u.x), fb = bf16c_to_float2(u.y);
        a = mk<R>((R)fa.x, (R)fa.y);
        b = mk<R>((R)fb.x, (R)fb.y);
    }
};

// load bypassing L1 (data written by other CTAs of the same launch)
__device__ __forceinline__ c64 ld_cg(const c64* q) {
    float2 v = __ldcg(reinterpret_cast<const float2*>(q));
    return mk<float>(v.x, v.y);
}
__device__ __forceinline__ c128 ld_cg(const c128* q) {
    double2 v = __ldcg(reinterpret_cast<const double2*>(q));
    return mk<double>(v.x, v.y);
}
__device__ __forceinline__ cx<df> ld_cg(const cx<df>* q) {
    const float4 v = __ldcg(reinterpret_cast<const float4*>(q));
    return mk<df>(df(v.x, v.y), df(v.z, v.w));
}

// NR consecutive complex values (one vector entry for NR right-hand sides)
template <typename R, int NR>
__device__ __forceinline__ void ldv(const cx<R>* __restrict__ q, cx<R> (&v)[NR]) {
    if constexpr (sizeof(R) == 4 && NR % 2 == 0) {
#pragma unroll
        for (int r = 0; r < NR; r += 2) {
            const float4 f = __ldg(reinterpret_cast<const float4*>(q + r));
            v[r] = mk<R>(f.x, f.y);
            v[r + 1] = mk<R>(f.z, f.w);
        }
    } else {
#pragma unroll
        for (int r = 0; r < NR; ++r) v[r] = q[r];
    }
}

// xp[(pos) * NR + r] = x[r * 2ne + edge(pos)] for both halves (J: pos < ne, M: ne + pos),
// conjugated for the adjoint product
template <typename R, int NR, bool CONJ>
__global__ void k_gather(const typename Caller<R>::T* __restrict__ x, const int64_t* __restrict__ perm,
                         cx<R>* __restrict__ xp, int ne) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    const int64_t e = perm[i];
    const int64_t nn = 2 * (int64_t)ne;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        cx<R> a = Caller<R>::in(x[r * nn + e]), b = Caller<R>::in(x[r * nn + ne + e]);
        if (CONJ) {
            a.im = -a.im;
            b.im = -b.im;
        }
        xp[(int64_t)i * NR + r] = a;
        xp[(int64_t)(ne + i) * NR + r] = b;
    }
}

#define VHX_THREADS 64   // 8 items of 8 lanes

// t = W^T x for a slice of one far block's items.  An item is one column pair kp
// of one operator's W (A and C use x_J and x_M respectively; B uses both and gives
// the two t segments of B).  Unit u covers items [8 lo, 8 lo + 8) of block b; an
// item is handled by 8 lanes (rows jj, jj+8, ...) and its t values are written by
// the group's first lane -- no shared memory, no barrier, no cross-CTA sum.
// Every loaded pair of W is applied to NR right-hand sides.
template <typename R, typename F, int NR>
__device__ __forceinline__ void vhx_unit(const FarRec* __restrict__ far, int2 un, const F* __restrict__ arena,
                                         const cx<R>* __restrict__ xp, cx<R>* __restrict__ t, int ne) {
    // BF16 factors move half the bytes per load: twice as many loads in flight
    constexpr int UN = (NR == 1 ? 4 : (NR == 2 ? 2 : 1)) * (sizeof(F) == 4 ? 2 : 1);
    const FarRec* Fp = far + un.x;
    const int n = Fp->n;
    const int kpA = (Fp->rk[0] + 1) >> 1, kpB = (Fp->rk[1] + 1) >> 1, kpC = (Fp->rk[2] + 1) >> 1;
    const int it = un.y * 8 + (threadIdx.x >> 3);
    const int jj = threadIdx.x & 7;
    if (it >= kpA + kpB + kpC) return;  // whole 8-lane group leaves this unit together
    int op, kp;
    if (it < kpA) {
        op = 0;
        kp = it;
    } else if (it < kpA + kpB) {
        op = 1;
        kp = it - kpA;
    } else {
        op = 2;
        kp = it - kpA - kpB;
    }
    // column pair kp of W, all rows: pair index kp*n + row (two complex values per pair)
    const F* V = arena + Fp->off_v[op] + 2 * (int64_t)kp * n;
    const cx<R>* xs = xp + ((int64_t)((op == 2) ? ne : 0) + Fp->c0) * NR;  // J for A and B, M for C
    const cx<R>* xm = xp + ((int64_t)ne + Fp->c0) * NR;
    cx<R> a0[NR], a1[NR], b0[NR], b1[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) a0[r] = a1[r] = b0[r] = b1[r] = mk<R>(0, 0);
    auto step = [&](const cx<R>& w0, const cx<R>& w1, int j) {
        cx<R> xv[NR];
        ldv<R, NR>(xs + (int64_t)j * NR, xv);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            cfma(a0[r], w0, xv[r]);
            cfma(a1[r], w1, xv[r]);
        }
        if (op == 1) {
            ldv<R, NR>(xm + (int64_t)j * NR, xv);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                cfma(b0[r], w0, xv[r]);
                cfma(b1[r], w1, xv[r]);
            }
        }
    };
    int j = jj;
    for (; j + 8 * (UN - 1) < n; j += 8 * UN) {
        cx<R> w0[UN], w1[UN];
#pragma unroll
        for (int q = 0; q < UN; ++q) FPair<F>::template ld<R>(V, j + 8 * q, w0[q], w1[q]);
#pragma unroll
        for (int q = 0; q < UN; ++q) step(w0[q], w1[q], j + 8 * q);
    }
    if (j < n) {
        // the remaining (< UN) rows of this lane: loads first, then the sums
        cx<R> w0[UN], w1[UN];
#pragma unroll
        for (int q = 0; q < UN; ++q) {
            if (j + 8 * q < n) {
                FPair<F>::template ld<R>(V, j + 8 * q, w0[q], w1[q]);
            } else {
                w0[q] = w1[q] = mk<R>(0, 0);
            }
        }
#pragma unroll
        for (int q = 0; q < UN; ++q)
            if (j + 8 * q < n) step(w0[q], w1[q], j + 8 * q);
    }
    // sum over the 8 lanes of the group (xor offsets stay inside the group)
    const unsigned mask = 0xffu << (threadIdx.x & 24);
#pragma unroll
    for (int r = 0; r < NR; ++r)
        for (int o = 4; o > 0; o >>= 1) {
            a0[r].re += xshfl(mask, a0[r].re, o);
            a0[r].im += xshfl(mask, a0[r].im, o);
            a1[r].re += xshfl(mask, a1[r].re, o);
            a1[r].im += xshfl(mask, a1[r].im, o);
            if (op == 1) {
                b0[r].re += xshfl(mask, b0[r].re, o);
                b0[r].im += xshfl(mask, b0[r].im, o);
                b1[r].re += xshfl(mask, b1[r].re, o);
                b1[r].im += xshfl(mask, b1[r].im, o);
            }
        }
    if (jj == 0) {
        // t segments of the block: [tA | tB(J) | tB(M) | tC], 2 values per column pair, NR each
        cx<R>* tb = t + Fp->off_t * NR;
        const int seg = (op == 0) ? 0 : ((op == 1) ? 2 * kpA : 2 * (kpA + 2 * kpB));
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            tb[(seg + 2 * kp) * NR + r] = a0[r];
            tb[(seg + 2 * kp + 1) * NR + r] = a1[r];
            if (op == 1) {
                tb[(2 * (kpA + kpB) + 2 * kp) * NR + r] = b0[r];
                tb[(2 * (kpA + kpB) + 2 * kp + 1) * NR + r] = b1[r];
            }
        }
    }
}

// The same for 4 or 8 right-hand sides, with lanes over right-hand sides: lane l
// of an item's 8 handles right-hand side l mod NR over the rows j = l / NR,
// l / NR + 8 / NR, ...; the W pair of a row is
// one broadcast load for the lanes that share it, each lane keeps four complex
// sums, and the lanes of one right-hand side are summed by shuffles.
template <typename R, typename F, int NR>
__device__ __forceinline__ void vhx_unit_rhs(const FarRec* __restrict__ far, int2 un, const F* __restrict__ arena,
                                             const cx<R>* __restrict__ xp, cx<R>* __restrict__ t, int ne) {
    constexpr int LPR = 8 / NR;  // lanes per right-hand side (rows split among them)
    constexpr int UN = 4;
    const FarRec* Fp = far + un.x;
    const int n = Fp->n;
    const int kpA = (Fp->rk[0] + 1) >> 1, kpB = (Fp->rk[1] + 1) >> 1, kpC = (Fp->rk[2] + 1) >> 1;
    const int it = un.y * 8 + (threadIdx.x >> 3);
    const int ll = threadIdx.x & 7;
    const int r = ll % NR, j0 = ll / NR;
    if (it >= kpA + kpB + kpC) return;  // whole 8-lane group leaves this unit together
    int op, kp;
    if (it < kpA) {
        op = 0;
        kp = it;
    } else if (it < kpA + kpB) {
        op = 1;
        kp = it - kpA;
    } else {
        op = 2;
        kp = it - kpA - kpB;
    }
    const F* V = arena + Fp->off_v[op] + 2 * (int64_t)kp * n;
    const cx<R>* xs = xp + ((int64_t)((op == 2) ? ne : 0) + Fp->c0) * NR + r;
    const cx<R>* xm = xp + ((int64_t)ne + Fp->c0) * NR + r;
    cx<R> a0 = mk<R>(0, 0), a1 = a0, b0 = a0, b1 = a0;
    int j = j0;
    for (; j + LPR * (UN - 1) < n; j += LPR * UN) {
        cx<R> w0[UN], w1[UN], xv[UN];
#pragma unroll
        for (int q = 0; q < UN; ++q) {
            FPair<F>::template ld<R>(V, j + LPR * q, w0[q], w1[q]);
            xv[q] = xs[(int64_t)(j + LPR * q) * NR];
        }
#pragma unroll
        for (int q = 0; q < UN; ++q) {
            cfma(a0, w0[q], xv[q]);
            cfma(a1, w1[q], xv[q]);
        }
        if (op == 1) {
#pragma unroll
            for (int q = 0; q < UN; ++q) {
                const cx<R> xw = xm[(int64_t)(j + LPR * q) * NR];
                cfma(b0, w0[q], xw);
                cfma(b1, w1[q], xw);
            }
        }
    }
    if (j < n) {
        cx<R> w0[UN], w1[UN], xv[UN];
#pragma unroll
        for (int q = 0; q < UN; ++q) {
            if (j + LPR * q < n) {
                FPair<F>::template ld<R>(V, j + LPR * q, w0[q], w1[q]);
                xv[q] = xs[(int64_t)(j + LPR * q) * NR];
            } else {
                w0[q] = w1[q] = xv[q] = mk<R>(0, 0);
            }
        }
#pragma unroll
        for (int q = 0; q < UN; ++q) {
            cfma(a0, w0[q], xv[q]);
            cfma(a1, w1[q], xv[q]);
        }
        if (op == 1) {
#pragma unroll
            for (int q = 0; q < UN; ++q)
                if (j + LPR * q < n) {
                    const cx<R> xw = xm[(int64_t)(j + LPR * q) * NR];
                    cfma(b0, w0[q], xw);
                    cfma(b1, w1[q], xw);
                }
        }
    }
    if (LPR > 1) {
        // lanes of one right-hand side differ in the bits above log2(NR)
        const unsigned mask = 0xffu << (threadIdx.x & 24);
#pragma unroll
        for (int o = NR; o < 8; o <<= 1) {
            a0.re += xshfl(mask, a0.re, o);
            a0.im += xshfl(mask, a0.im, o);
            a1.re += xshfl(mask, a1.re, o);
            a1.im += xshfl(mask, a1.im, o);
            if (op == 1) {
                b0.re += xshfl(mask, b0.re, o);
                b0.im += xshfl(mask, b0.im, o);
                b1.re += xshfl(mask, b1.re, o);
                b1.im += xshfl(mask, b1.im, o);
            }
        }
    }
    if (j0 == 0) {
        cx<R>* tb = t + Fp->off_t * NR;
        const int seg = (op == 0) ? 0 : ((op == 1) ? 2 * kpA : 2 * (kpA + 2 * kpB));
        tb[(seg + 2 * kp) * NR + r] = a0;
        tb[(seg + 2 * kp + 1) * NR + r] = a1;
        if (op == 1) {
            tb[(2 * (kpA + kpB) + 2 * kp) * NR + r] = b0;
            tb[(2 * (kpA + kpB) + 2 * kp + 1) * NR + r] = b1;
        }
    }
}

// one CTA per unit; the hardware scheduler balances the (largest-first) units
template <typename R, typename F, int NR>
__global__ void __launch_bounds__(VHX_THREADS, (NR == 1 && sizeof(R) == 4 && sizeof(F) == 8) ? 24 : 1) k_vhx(const FarRec* __restrict__ far, const int2* __restrict__ units,
                                                     int nunits, const F* __restrict__ arena,
                                                     const cx<R>* __restrict__ xp, cx<R>* __restrict__ t, int ne) {
    if ((int)blockIdx.x < nunits) {
        if constexpr (NR >= 4)
            vhx_unit_rhs<R, F, NR>(far, units[blockIdx.x], arena, xp, t, ne);
        else
            vhx_unit<R, F, NR>(far, units[blockIdx.x], arena, xp, t, ne);
    }
}

// Adjoint product, first pass: t' = U^T xp over the block's rows (A and C use x_J
// and x_M of the row cluster; B gives both segments), the same units and t layout
// as vhx.  U is slice-major, so each row's pair index depends on its leaf: the leaf
// start and size of every tree position come from pos_leaf_lo / pos_leaf_m.
template <typename R, typename F, int NR>
__device__ __forceinline__ void uhx_unit(const FarRec* __restrict__ far, int2 un, const F* __restrict__ arena,
                                         const cx<R>* __restrict__ xp, cx<R>* __restrict__ t, int ne,
                                         const int* __restrict__ pos_leaf_lo, const int* __restrict__ pos_leaf_m) {
    const FarRec* Fp = far + un.x;
    const int m = Fp->m, r0 = Fp->r0;
    const int kpA = (Fp->rk[0] + 1) >> 1, kpB = (Fp->rk[1] + 1) >> 1, kpC = (Fp->rk[2] + 1) >> 1;
    const int it = un.y * 8 + (threadIdx.x >> 3);
    const int jj = threadIdx.x & 7;
    if (it >= kpA + kpB + kpC) return;  // whole 8-lane group leaves this unit together
    int op, kp, kpc;
    if (it < kpA) {
        op = 0;
        kp = it;
        kpc = kpA;
    } else if (it < kpA + kpB) {
        op = 1;
        kp = it - kpA;
        kpc = kpB;
    } else {
        op = 2;
        kp = it - kpA - kpB;
        kpc = kpC;
    }
    const F* Ub = arena + Fp->off_u[op];
    const cx<R>* xs = xp + ((int64_t)((op == 2) ? ne : 0) + r0) * NR;  // J for A and B, M for C
    const cx<R>* xm = xp + ((int64_t)ne + r0) * NR;
    cx<R> a0[NR], a1[NR], b0[NR], b1[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) a0[r] = a1[r] = b0[r] = b1[r] = mk<R>(0, 0);
    constexpr int UN = NR == 1 ? 4 : (NR == 2 ? 2 : 1);
    for (int i0 = jj; i0 < m; i0 += 8 * UN) {
        // UN rows of this lane: loads first (predicated at the end of the block)
        cx<R> u0[UN], u1[UN];
#pragma unroll
        for (int q = 0; q < UN; ++q) {
            const int i = i0 + 8 * q;
            if (i < m) {
                const int ro = pos_leaf_lo[r0 + i] - r0, ms = pos_leaf_m[r0 + i];
                FPair<F>::template ld<R>(Ub, (int64_t)ro * kpc + (int64_t)kp * ms + (i - ro), u0[q], u1[q]);
            } else {
                u0[q] = u1[q] = mk<R>(0, 0);
            }
        }
#pragma unroll
        for (int q = 0; q < UN; ++q) {
            const int i = i0 + 8 * q;
            if (i >= m) continue;
            cx<R> xv[NR];
            ldv<R, NR>(xs + (int64_t)i * NR, xv);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                cfma(a0[r], u0[q], xv[r]);
                cfma(a1[r], u1[q], xv[r]);
            }
            if (op == 1) {
                ldv<R, NR>(xm + (int64_t)i * NR, xv);
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    cfma(b0[r], u0[q], xv[r]);
                    cfma(b1[r], u1[q], xv[r]);
                }
            }
        }
    }
    const unsigned mask = 0xffu << (threadIdx.x & 24);
#pragma unroll
    for (int r = 0; r < NR; ++r)
        for (int o = 4; o > 0; o >>= 1) {
            a0[r].re += xshfl(mask, a0[r].re, o);
            a0[r].im += xshfl(mask, a0[r].im, o);
            a1[r].re += xshfl(mask, a1[r].re, o);
            a1[r].im += xshfl(mask, a1[r].im, o);
            if (op == 1) {
                b0[r].re += xshfl(mask, b0[r].re, o);
                b0[r].im += xshfl(mask, b0[r].im, o);
                b1[r].re += xshfl(mask, b1[r].re, o);
                b1[r].im += xshfl(mask, b1[r].im, o);
            }
        }
    if (jj == 0) {
        cx<R>* tb = t + Fp->off_t * NR;
        const int seg = (op == 0) ? 0 : ((op == 1) ? 2 * kpA : 2 * (kpA + 2 * kpB));
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            tb[(seg + 2 * kp) * NR + r] = a0[r];
            tb[(seg + 2 * kp + 1) * NR + r] = a1[r];
            if (op == 1) {
                tb[(2 * (kpA + kpB) + 2 * kp) * NR + r] = b0[r];
                tb[(2 * (kpA + kpB) + 2 * kp + 1) * NR + r] = b1[r];
            }
        }
    }
}

template <typename R, typename F, int NR>
__global__ void __launch_bounds__(VHX_THREADS) k_uhx(const FarRec* __restrict__ far, const int2* __restrict__ units,
                                                     int nunits, const F* __restrict__ arena,
                                                     const cx<R>* __restrict__ xp, cx<R>* __restrict__ t, int ne,
                                                     const int* __restrict__ pos_leaf_lo,
                                                     const int* __restrict__ pos_leaf_m) {
    if ((int)blockIdx.x < nunits)
        uhx_unit<R, F, NR>(far, units[blockIdx.x], arena, xp, t, ne, pos_leaf_lo, pos_leaf_m);
}

#define ROW_THREADS (64 * BEM_ROW_GROUPS)
#define ROW_GROUPS BEM_ROW_GROUPS

// One dense item (leaf rows x n columns): y_J += A xJ + B xM, y_M += C xM - B xJ
// for NR right-hand sides (xJ, xM: NR values per column).  ADJ: the item holds the
// transposed blocks and B enters with the opposite signs (Z^T = [[A^T, -B^T],
// [B^T, C^T]]).
template <typename R, typename NS, int NR, bool ADJ>
__device__ __forceinline__ void dense_item(const NS* __restrict__ A, int64_t stride, int m, int i, int n,
                                           const cx<R>* __restrict__ xJ, const cx<R>* __restrict__ xM,
                                           cx<R> (&aJ)[NR], cx<R> (&aM)[NR]) {
    constexpr int UN = NR == 1 ? 4 : (NR == 2 ? 2 : 1);
    const NS* B = A + stride;
    const NS* C = B + stride;
    const int nfull = n >> 1;  // column pairs with both columns inside the item
    auto apply = [&](const cx<R>& a0, const cx<R>& a1, const cx<R>& b0, const cx<R>& b1, const cx<R>& c0,
                     const cx<R>& c1, int j) {
        cx<R> xj0[NR], xm0[NR], xj1[NR], xm1[NR];
        ldv<R, NR>(xJ + (int64_t)j * NR, xj0);
        ldv<R, NR>(xJ + (int64_t)(j + 1) * NR, xj1);
        ldv<R, NR>(xM + (int64_t)j * NR, xm0);
        ldv<R, NR>(xM + (int64_t)(j + 1) * NR, xm1);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            cfma(aJ[r], a0, xj0[r]);
            cfma(aJ[r], a1, xj1[r]);
            cfma(aM[r], c0, xm0[r]);
            cfma(aM[r], c1, xm1[r]);
            if (ADJ) {
                cx<R> bm = b0 * xm0[r];
                cfma(bm, b1, xm1[r]);
                cx<R> bx = b0 * xj0[r];
                cfma(bx, b1, xj1[r]);
                aJ[r] = aJ[r] - bm;
                aM[r] = aM[r] + bx;
            } else {
                cfma(aJ[r], b0, xm0[r]);
                cfma(aJ[r], b1, xm1[r]);
                cx<R> bx = b0 * xj0[r];
                cfma(bx, b1, xj1[r]);
                aM[r] = aM[r] - bx;
            }
        }
    };
    int cp = 0;
    for (; cp + UN <= nfull; cp += UN) {
        cx<R> a0[UN], a1[UN], b0[UN], b1[UN], c0[UN], c1[UN];
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            const int64_t idx = (int64_t)(cp + u) * m + i;
            FPair<NS>::template ld<R>(A, idx, a0[u], a1[u]);
            FPair<NS>::template ld<R>(B, idx, b0[u], b1[u]);
            FPair<NS>::template ld<R>(C, idx, c0[u], c1[u]);
        }
#pragma unroll
        for (int u = 0; u < UN; ++u) apply(a0[u], a1[u], b0[u], b1[u], c0[u], c1[u], 2 * (cp + u));
    }
    if (cp < nfull) {
        // the remaining (< UN) column pairs: all loads issued before any is used
        cx<R> a0[UN], a1[UN], b0[UN], b1[UN], c0[UN], c1[UN];
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            if (cp + u < nfull) {
                const int64_t idx = (int64_t)(cp + u) * m + i;
                FPair<NS>::template ld<R>(A, idx, a0[u], a1[u]);
                FPair<NS>::template ld<R>(B, idx, b0[u], b1[u]);
                FPair<NS>::template ld<R>(C, idx, c0[u], c1[u]);
            } else {
                a0[u] = a1[u] = b0[u] = b1[u] = c0[u] = c1[u] = mk<R>(0, 0);
            }
        }
#pragma unroll
        for (int u = 0; u < UN; ++u)
            if (cp + u < nfull) apply(a0[u], a1[u], b0[u], b1[u], c0[u], c1[u], 2 * (cp + u));
        cp = nfull;
    }
    if (n & 1) {  // last column; its pair partner is a stored zero column
        cx<R> a0, a1, b0, b1, c0, c1;
        const int64_t idx = (int64_t)nfull * m + i;
        FPair<NS>::template ld<R>(A, idx, a0, a1);
        FPair<NS>::template ld<R>(B, idx, b0, b1);
        FPair<NS>::template ld<R>(C, idx, c0, c1);
        cx<R> xj0[NR], xm0[NR];
        ldv<R, NR>(xJ + (int64_t)(n - 1) * NR, xj0);
        ldv<R, NR>(xM + (int64_t)(n - 1) * NR, xm0);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            cfma(aJ[r], a0, xj0[r]);
            cfma(aM[r], c0, xm0[r]);
            if (ADJ) {
                aJ[r] = aJ[r] - b0 * xm0[r];
                aM[r] = aM[r] + b0 * xj0[r];
            } else {
                cfma(aJ[r], b0, xm0[r]);
                aM[r] = aM[r] - b0 * xj0[r];
            }
        }
    }
}

// y_J += U_A tA + U_B tBM, y_M += U_C tC - U_B tBJ for rows ro + i of one far block.
// U is slice-major: the leaf's slice (ms rows starting at ro) of operator q is one
// contiguous run, pair (kp, i) at ro * kpc + kp * ms + i (stride ms).  t values: NR
// per column.  ADJ (rows of the block's column cluster): the factor is W, pair
// (kp, i) at kp * n + so + i (stride n), and the B terms change sign.
template <typename R, typename F, int NR, int MODE, bool ADJ>
__device__ __forceinline__ void far_slice(const F* __restrict__ U, int kpc, int ms, int i,
                                          const cx<R>* __restrict__ tv, const cx<R>* __restrict__ tv2,
                                          cx<R> (&aJ)[NR], cx<R> (&aM)[NR]) {
    // MODE 0: aJ += U tv; 1: aJ += U tv (tBM), aM -= U tv2 (tBJ); 2: aM += U tv
    // (slices are short runs: eight loads in flight per thread for one right-hand side)
    constexpr int UN = NR == 1 ? 8 : (NR == 2 ? 4 : (NR == 4 ? 2 : 1));
    auto apply = [&](const cx<R>& u0, const cx<R>& u1, int kp) {
        const int k2 = 2 * kp;
        cx<R> p0[NR], p1[NR];
        ldv<R, NR>(tv + (int64_t)k2 * NR, p0);
        ldv<R, NR>(tv + (int64_t)(k2 + 1) * NR, p1);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            cx<R> sum = u0 * p0[r];
            cfma(sum, u1, p1[r]);
            if (MODE == 2)
                aM[r] = aM[r] + sum;
            else if (MODE == 1 && ADJ)
                aJ[r] = aJ[r] - sum;
            else
                aJ[r] = aJ[r] + sum;
        }
        if (MODE == 1) {
            ldv<R, NR>(tv2 + (int64_t)k2 * NR, p0);
            ldv<R, NR>(tv2 + (int64_t)(k2 + 1) * NR, p1);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                cx<R> bx = u0 * p0[r];
                cfma(bx, u1, p1[r]);
                aM[r] = ADJ ? aM[r] + bx : aM[r] - bx;
            }
        }
    };
    int kp = 0;
    for (; kp + UN <= kpc; kp += UN) {
        cx<R> u0[UN], u1[UN];
#pragma unroll
        for (int u = 0; u < UN; ++u) FPair<F>::template ld<R>(U, (int64_t)(kp + u) * ms + i, u0[u], u1[u]);
#pragma unroll
        for (int u = 0; u < UN; ++u) apply(u0[u], u1[u], kp + u);
    }
    if (kp < kpc) {
        // the remaining (< UN) pairs: all loads issued before any is used (short
        // slices, e.g. low-rank blocks of small leaves, are mostly tail)
        cx<R> u0[UN], u1[UN];
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            if (kp + u < kpc) {
                FPair<F>::template ld<R>(U, (int64_t)(kp + u) * ms + i, u0[u], u1[u]);
            } else {
                u0[u] = u1[u] = mk<R>(0, 0);
            }
        }
#pragma unroll
        for (int u = 0; u < UN; ++u)
            if (kp + u < kpc) apply(u0[u], u1[u], kp + u);
    }
}

// One far piece: the three factor slices of a leaf's rows with the 2 x 2 PMCHWT
// structure (ADJ: the factors are W rows and the B terms change sign).
template <typename R, typename FS, int NR, bool ADJ>
__device__ __forceinline__ void far_piece(const PieceDesc& d, int i, const FS* __restrict__ arena,
                                          const cx<R>* __restrict__ t, cx<R> (&aJ)[NR], cx<R> (&aM)[NR]) {
    const int kpA = d.kp[0], kpB = d.kp[1], kpC = d.kp[2];
    const cx<R>* tA = t + d.t_off * NR;
    const cx<R>* tBJ = tA + 2 * kpA * NR;
    const cx<R>* tBM = tBJ + 2 * kpB * NR;
    const cx<R>* tC = tBM + 2 * kpB * NR;
    far_slice<R, FS, NR, 0, ADJ>(arena + d.base[0], kpA, d.ld, i, tA, nullptr, aJ, aM);
    far_slice<R, FS, NR, 1, ADJ>(arena + d.base[1], kpB, d.ld, i, tBM, tBJ, aJ, aM);
    far_slice<R, FS, NR, 2, ADJ>(arena + d.base[2], kpC, d.ld, i, tC, nullptr, aJ, aM);
}

// Grid: one 64-thread CTA per work slot (a leaf's dense items and far pieces are
// split at assembly into parts proportional to its share of the work; CTAs take
// the slots heaviest first).  With one part the CTA writes y; with several, each
// writes its partial rows, and the last CTA of the leaf to finish (arrival
// counter, after a memory fence) adds the parts in index order and writes y -- the
// sum does not depend on which CTA finishes last.
// y is in the caller's layout: right-hand side r at y + r * 2ne.
template <typename R, typename NS, typename FS, int NR, bool ADJ>
__global__ void __launch_bounds__(ROW_THREADS, (NR == 1 && sizeof(R) == 4) ? 16 : 1) k_rows(MatvecPlan p, const NS* __restrict__ near,
                                                      const FS* __restrict__ arena,
                                                      const cx<R>* __restrict__ xp, const cx<R>* __restrict__ t,
                                                      typename Caller<R>::T* __restrict__ y,
                                                      cx<R>* __restrict__ ypart, unsigned int* __restrict__ arrive) {
    __shared__ bool s_last;
    const int slot = p.slot_order[blockIdx.x];
    const int leaf = p.slot_leaf[slot], part = p.slot_part[slot];
    const int P = p.leaf_parts[leaf];
    const int r0 = p.leaf_r0[leaf], m = p.leaf_m[leaf];
    const int i = threadIdx.x & 63;
    const bool act = i < m;
    const int ne = p.ne;
    const int64_t nn = 2 * (int64_t)ne;
    cx<R> aJ[NR], aM[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) aJ[r] = aM[r] = mk<R>(0, 0);
    const int w0 = p.work_ptr[slot], w1 = p.work_ptr[slot + 1];
    if (act) {
        for (int w = w0; w < w1; ++w) {
            const int item = p.work_item[w];
            if (item >= 0) {
                const int c0 = p.near_c0[item];
                dense_item<R, NS, NR, ADJ>(near + p.near_off[item], p.near_op_stride, m, i, p.near_n[item],
                                  xp + (int64_t)c0 * NR, xp + ((int64_t)ne + c0) * NR, aJ, aM);
            } else {
                const PieceDesc d = p.pieces[-1 - item];
                far_piece<R, FS, NR, ADJ>(d, i, arena, t, aJ, aM);
            }
        }
    }
    if (P == 1) {
        if (act) {
            const int64_t e = p.perm[r0 + i];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                if (ADJ) {
                    aJ[r].im = -aJ[r].im;
                    aM[r].im = -aM[r].im;
                }
                y[r * nn + e] = Caller<R>::out(aJ[r]);
                y[r * nn + ne + e] = Caller<R>::out(aM[r]);
            }
        }
        return;
    }
    if (act) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            ypart[(part * nn + r0 + i) * NR + r] = aJ[r];
            ypart[(part * nn + ne + r0 + i) * NR + r] = aM[r];
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(arrive + leaf, 1u) == (unsigned)(P - 1));
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (act) {
        const int64_t e = p.perm[r0 + i];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            cx<R> sj = mk<R>(0, 0), sm = sj;
            for (int q = 0; q < P; ++q) {
                sj = sj + ld_cg(ypart + (q * nn + r0 + i) * NR + r);
                sm = sm + ld_cg(ypart + (q * nn + ne + r0 + i) * NR + r);
            }
            if (ADJ) {
                sj.im = -sj.im;
                sm.im = -sm.im;
            }
            y[r * nn + e] = Caller<R>::out(sj);
            y[r * nn + ne + e] = Caller<R>::out(sm);
        }
    }
    if (threadIdx.x == 0) arrive[leaf] = 0u;  // ready for the next product
}

template <typename R, typename NS, typename FS, int NR, bool ADJ>
static cudaError_t product_chunk(const MatvecPlan& p, const void* near_entries, const void* arena,
                                 const typename Caller<R>::T* x, typename Caller<R>::T* y, cx<R>* xp, cx<R>* t,
                                 cudaStream_t st, const cudaEvent_t* e) {
    if (e) BEM_CUDA_TRY(cudaEventRecord(e[0], st));
    k_gather<R, NR, ADJ><<<(p.ne + 255) / 256, 256, 0, st>>>(x, p.perm, xp, p.ne);
    BEM_CUDA_TRY(cudaGetLastError());
    if (e) BEM_CUDA_TRY(cudaEventRecord(e[1], st));
    if (e) BEM_CUDA_TRY(cudaEventRecord(e[2], st));
    if (p.nvhx > 0) {
        if (ADJ)
            k_uhx<R, FS, NR><<<p.nvhx, VHX_THREADS, 0, st>>>(p.far, p.vhx_units, p.nvhx, (const FS*)arena, xp, t, p.ne,
                                                             p.pos_leaf_lo, p.pos_leaf_m);
        else
            k_vhx<R, FS, NR><<<p.nvhx, VHX_THREADS, 0, st>>>(p.far, p.vhx_units, p.nvhx, (const FS*)arena, xp, t, p.ne);
        BEM_CUDA_TRY(cudaGetLastError());
    }
    if (e) BEM_CUDA_TRY(cudaEventRecord(e[3], st));
    if (e) BEM_CUDA_TRY(cudaEventRecord(e[4], st));
    k_rows<R, NS, FS, NR, ADJ><<<p.nslot, ROW_THREADS, 0, st>>>(p, (const NS*)near_entries, (const FS*)arena, xp, t,
                                                                 y, (cx<R>*)p.ypart, p.arrive);
    BEM_CUDA_TRY(cudaGetLastError());
    if (e) BEM_CUDA_TRY(cudaEventRecord(e[5], st));
    return cudaSuccess;
}

// Right-hand sides are processed in chunks of 8 (at most MAXC), 4, 2, 1: every
// chunk streams the operator once and applies each loaded entry to all of its
// right-hand sides.
template <typename R, typename NS, typename FS, bool ADJ, int MAXC = 8>
static cudaError_t matvec_chunks(const MatvecPlan& p, const void* near_entries, const void* arena,
                                 const typename Caller<R>::T* x, typename Caller<R>::T* y, cx<R>* xp, cx<R>* t,
                                 int nrhs, cudaStream_t st, const cudaEvent_t* ev) {
    const int64_t nn = 2 * (int64_t)p.ne;
    int r = 0, chunk = 0;
    while (r < nrhs) {
        const int left = nrhs - r;
        const int nr = (left >= 8 && MAXC >= 8) ? 8 : (left >= 4 ? 4 : (left >= 2 ? 2 : 1));
        const cudaEvent_t* e = ev ? ev + 6 * chunk : nullptr;
        const typename Caller<R>::T* xr = x + r * nn;
        typename Caller<R>::T* yr = y + r * nn;
        cudaError_t err;
        switch (nr) {
            case 8:
                if constexpr (MAXC >= 8) {
                    err = product_chunk<R, NS, FS, 8, ADJ>(p, near_entries, arena, xr, yr, xp, t, st, e);
                    break;
                }
                [[fallthrough]];
            case 4: err = product_chunk<R, NS, FS, 4, ADJ>(p, near_entries, arena, xr, yr, xp, t, st, e); break;
            case 2: err = product_chunk<R, NS, FS, 2, ADJ>(p, near_entries, arena, xr, yr, xp, t, st, e); break;
            default: err = product_chunk<R, NS, FS, 1, ADJ>(p, near_entries, arena, xr, yr, xp, t, st, e); break;
        }
        if (err != cudaSuccess) return err;
        r += nr;
        ++chunk;
    }
    return cudaSuccess;
}

template <typename R>
cudaError_t matvec_run(const MatvecPlan& p, const void* near_entries, const void* arena, const cx<R>* x, cx<R>* y,
                       cx<R>* xp, cx<R>* t, int nrhs, int64_t t_len, cudaStream_t st, const cudaEvent_t* ev,
                       int form, bool adjoint) {
    (void)t_len;
    if constexpr (sizeof(R) == 4) {
        if (form == BEM_FORM_BF16F) {
            if (adjoint) return cudaErrorInvalidValue;
            return matvec_chunks<float, c64, bf16c, false>(p, near_entries, arena, x, y, xp, t, nrhs, st, ev);
        }
        if (form != BEM_FORM_NATIVE) return cudaErrorInvalidValue;
    } else {
        if (form == BEM_FORM_C64_IN_FP64) {
            // complex64 operator applied to complex128 vectors with double-float
            // products and sums (residuals of iterative refinement); the complex64
            // workspaces (8 values of 8 bytes per unknown) hold 4 right-hand sides
            cx<df>* xd = reinterpret_cast<cx<df>*>(xp);
            cx<df>* td = reinterpret_cast<cx<df>*>(t);
            if (adjoint) return matvec_chunks<df, c64, c64, true, 4>(p, near_entries, arena, x, y, xd, td, nrhs, st, ev);
            return matvec_chunks<df, c64, c64, false, 4>(p, near_entries, arena, x, y, xd, td, nrhs, st, ev);
        }
        if (form != BEM_FORM_NATIVE) return cudaErrorInvalidValue;
    }
    if (adjoint) return matvec_chunks<R, cx<R>, cx<R>, true>(p, near_entries, arena, x, y, xp, t, nrhs, st, ev);
    return matvec_chunks<R, cx<R>, cx<R>, false>(p, near_entries, arena, x, y, xp, t, nrhs, st, ev);
}

// Transposed copy of the dense items for the adjoint product: item k (m rows x n
// columns at offF[k], element (i, j) at 2 ((j / 2) m + i) + j mod 2, an odd n padded
// with a zero column) becomes an item of n rows x m columns at offT[k] in the same
// layout (an odd m padded with a zero column).  One CTA per item.
template <typename R>
__global__ void k_transpose_items(const BlockDesc* __restrict__ items, const int64_t* __restrict__ offF,
                                  const int64_t* __restrict__ offT, const cx<R>* __restrict__ near, int64_t strideF,
                                  cx<R>* __restrict__ nearT, int64_t strideT) {
    const BlockDesc b = items[blockIdx.x];
    const int m = b.m, n = b.n, mpad = m + (m & 1);
    for (int q = 0; q < 3; ++q) {
        const cx<R>* src = near + q * strideF + offF[blockIdx.x];
        cx<R>* dst = nearT + q * strideT + offT[blockIdx.x];
        for (int e = threadIdx.x; e < n * mpad; e += blockDim.x) {
            const int j = e % n, i = e / n;  // destination row j (a column of the item), column i
            const cx<R> v = i < m ? src[2 * ((int64_t)(j >> 1) * m + i) + (j & 1)] : mk<R>(0, 0);
            dst[2 * ((int64_t)(i >> 1) * n + j) + (i & 1)] = v;
        }
    }
}

template <typename R>
cudaError_t transpose_items(const BlockDesc* items, const int64_t* offF, const int64_t* offT, int nitems,
                            const cx<R>* near, int64_t strideF, cx<R>* nearT, int64_t strideT, cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    k_transpose_items<R><<<nitems, 256, 0, st>>>(items, offF, offT, near, strideF, nearT, strideT);
    return cudaGetLastError();
}

// BF16 copy of complex64 factors (round to nearest even per component)
__global__ void k_to_bf16(const c64* __restrict__ in, bf16c* __restrict__ out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = float2_to_bf16c(in[i].re, in[i].im);
}

cudaError_t factors_to_bf16(const c64* in, bf16c* out, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
    k_to_bf16<<<(unsigned)blocks, 256, 0, st>>>(in, out, n);
    return cudaGetLastError();
}

template cudaError_t matvec_run<float>(const MatvecPlan&, const void*, const void*, const c64*, c64*, c64*, c64*, int,
                                       int64_t, cudaStream_t, const cudaEvent_t*, int, bool);
template cudaError_t matvec_run<double>(const MatvecPlan&, const void*, const void*, const c128*, c128*, c128*,
                                        c128*, int, int64_t, cudaStream_t, const cudaEvent_t*, int, bool);
template cudaError_t transpose_items<float>(const BlockDesc*, const int64_t*, const int64_t*, int, const c64*, int64_t,
                                            c64*, int64_t, cudaStream_t);
template cudaError_t transpose_items<double>(const BlockDesc*, const int64_t*, const int64_t*, int, const c128*,
                                             int64_t, c128*, int64_t, cudaStream_t);

}  // namespace bem
