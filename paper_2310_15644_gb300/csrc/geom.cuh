// Device geometry helpers shared by the quadrature kernels.
#pragma once

#include "common.cuh"

namespace bem {

// slot of the singular pair (a, b) in the table (partners of a sorted ascending), or -1
__device__ __forceinline__ int find_singular(const GeomDev& g, int a, int b) {
    int lo = g.sing_ptr[a], hi = g.sing_ptr[a + 1];
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        int v = g.sing_b[mid];
        if (v == b) return mid;
        if (v < b)
            lo = mid + 1;
        else
            hi = mid;
    }
    return -1;
}

// 7-point degree-5 rule: barycentric points and weights (closed form with sqrt(15))
__device__ __forceinline__ void rule7_d(int q, double& l0, double& l1, double& l2, double& w) {
    const double s = 3.872983346207416885;  // sqrt(15)
    const double a1 = (6.0 - s) / 21.0, b1 = 1.0 - 2.0 * a1;
    const double a2 = (6.0 + s) / 21.0, b2 = 1.0 - 2.0 * a2;
    const double w1 = (155.0 - s) / 1200.0, w2 = (155.0 + s) / 1200.0;
    switch (q) {
        case 0: l0 = l1 = l2 = 1.0 / 3.0; w = 9.0 / 40.0; break;
        case 1: l0 = b1; l1 = a1; l2 = a1; w = w1; break;
        case 2: l0 = a1; l1 = b1; l2 = a1; w = w1; break;
        case 3: l0 = a1; l1 = a1; l2 = b1; w = w1; break;
        case 4: l0 = b2; l1 = a2; l2 = a2; w = w2; break;
        case 5: l0 = a2; l1 = b2; l2 = a2; w = w2; break;
        default: l0 = a2; l1 = a2; l2 = b2; w = w2; break;
    }
}

// the same rule in the arithmetic R (constants folded at compile time)
template <typename R>
__device__ __forceinline__ void rule7(int q, R& l0, R& l1, R& l2, R& w) {
    constexpr double s = 3.872983346207416885;  // sqrt(15)
    constexpr double a1 = (6.0 - s) / 21.0, b1 = 1.0 - 2.0 * a1;
    constexpr double a2 = (6.0 + s) / 21.0, b2 = 1.0 - 2.0 * a2;
    constexpr double w1 = (155.0 - s) / 1200.0, w2 = (155.0 + s) / 1200.0;
    constexpr R third = (R)(1.0 / 3.0), w0 = (R)(9.0 / 40.0);
    constexpr R A1 = (R)a1, B1 = (R)b1, A2 = (R)a2, B2 = (R)b2, W1 = (R)w1, W2 = (R)w2;
    switch (q) {
        case 0: l0 = l1 = l2 = third; w = w0; break;
        case 1: l0 = B1; l1 = A1; l2 = A1; w = W1; break;
        case 2: l0 = A1; l1 = B1; l2 = A1; w = W1; break;
        case 3: l0 = A1; l1 = A1; l2 = B1; w = W1; break;
        case 4: l0 = B2; l1 = A2; l2 = A2; w = W2; break;
        case 5: l0 = A2; l1 = B2; l2 = A2; w = W2; break;
        default: l0 = A2; l1 = A2; l2 = B2; w = W2; break;
    }
}

struct d3 {
    double x, y, z;
};
__device__ __forceinline__ d3 D3(double x, double y, double z) { return {x, y, z}; }
__device__ __forceinline__ d3 operator+(d3 a, d3 b) { return D3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ d3 operator-(d3 a, d3 b) { return D3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ d3 operator*(double s, d3 a) { return D3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ double dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ d3 cross(d3 a, d3 b) {
    return D3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ d3 ld3(const double* p) { return D3(p[0], p[1], p[2]); }

// complex 3-vector
struct z3 {
    c128 x, y, z;
};
__device__ __forceinline__ z3 Z3(c128 x, c128 y, c128 z) { return {x, y, z}; }
__device__ __forceinline__ z3 zscale(c128 s, d3 a) { return Z3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ z3 zadd(z3 a, z3 b) { return Z3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ z3 zsub(z3 a, z3 b) { return Z3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ c128 zdot(d3 a, z3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
// real x complex cross product
__device__ __forceinline__ z3 rzcross(d3 a, z3 b) {
    return Z3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ z3 zrcross(z3 a, d3 b) {
    return Z3(b.z * a.y - b.y * a.z, b.x * a.z - b.z * a.x, b.y * a.x - b.x * a.y);
}


}  // namespace bem
