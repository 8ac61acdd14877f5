// Absorbed power without any device allocation.
//
// bem_power sums the absorbed power through per-block partial sums kept in a
// device buffer that it allocates (and grows) on first use.  Some callers cannot
// let a library call cudaMalloc: a framework that owns all device memory through
// its own pool allocator and budget, or a latency-critical loop that must not
// take the implicit device-wide synchronisation that cudaMalloc and cudaFree can
// cause.  This file gives them bem_absorbed_power_static: the same reduction,
// with its partial sums in a fixed array that is part of the library image on
// each device, so the call itself allocates nothing.
#include <cstdio>
#include <mutex>

#include "common.cuh"

// Partial sums of the absorbed-power reduction: one double per (256-triangle
// block, right-hand side).  512 KiB on every device that loads the library, held
// until the process exits.
#define BEM_STATIC_PARTIALS 65536
static __device__ __align__(256) double g_power_partials[BEM_STATIC_PARTIALS];

namespace {

// Device address of g_power_partials, per device ordinal.  In host code the name
// g_power_partials is only a host-side stand-in for the symbol, never a device
// address, so the address is looked up with cudaGetSymbolAddress on that device.
const int kMaxDevices = 64;
double* g_partials_dev[kMaxDevices] = {nullptr};
std::mutex g_partials_mu;

cudaError_t partials_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_partials_mu);
    if (!g_partials_dev[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_power_partials);
        if (e != cudaSuccess) return e;
        g_partials_dev[dev] = (double*)p;
    }
    *out = g_partials_dev[dev];
    return cudaSuccess;
}

}  // namespace

// Helper shared with bem_api.cu: the context's device geometry (no allocation).
GeomDev bem_geom_view_for_static(const bem_ctx* c);
bool bem_ctx_has_geometry(const bem_ctx* c);
bool bem_ctx_is_layered(const bem_ctx* c);
void bem_ctx_set_error(bem_ctx* c, const char* msg);

extern "C" bem_status bem_absorbed_power_static(bem_ctx* c, const void* x, int nrhs, double* p_abs, void* stream) {
    if (!c) return BEM_EINVAL;
    if (!bem_ctx_has_geometry(c)) {
        bem_ctx_set_error(c, "bem_absorbed_power_static needs bem_assemble");
        return BEM_ESTATE;
    }
    if (bem_ctx_is_layered(c)) {
        bem_ctx_set_error(c, "bem_absorbed_power_static is not available on a layered context");
        return BEM_ESTATE;
    }
    if (nrhs < 1 || !x || !p_abs) {
        bem_ctx_set_error(c, "bem_absorbed_power_static: bad arguments");
        return BEM_EINVAL;
    }
    if (nrhs > BEM_MAX_NRHS) {
        char buf[160];
        snprintf(buf, sizeof buf, "bem_absorbed_power_static: %d right-hand sides in one call; at most %d", nrhs,
                 BEM_MAX_NRHS);
        bem_ctx_set_error(c, buf);
        return BEM_EINVAL;
    }
    GeomDev g = bem_geom_view_for_static(c);
    const int nblk = (g.nt + 255) / 256;  // partial sums per right-hand side (blocks of power_abs)
    if ((int64_t)nblk * nrhs > BEM_STATIC_PARTIALS) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "bem_absorbed_power_static: %d right-hand sides x %d triangle blocks need %lld partial sums; "
                 "the fixed scratch holds %d (use bem_power, or fewer right-hand sides per call)",
                 nrhs, nblk, (long long)nblk * nrhs, BEM_STATIC_PARTIALS);
        bem_ctx_set_error(c, buf);
        return BEM_EINVAL;
    }
    double* partials = nullptr;
    cudaError_t e = partials_address(&partials);
    if (e == cudaSuccess) {
        // every partial sum is written before it is read, so nothing needs clearing
        e = bem::power_abs(g, (const c128*)x, nrhs, nullptr, partials, nblk, (cudaStream_t)stream);
    }
    if (e == cudaSuccess) e = bem::kv_reduce_real(partials, nblk, nrhs, p_abs, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        bem_ctx_set_error(c, cudaGetErrorString(e));
        return BEM_ECUDA;
    }
    return BEM_OK;
}
