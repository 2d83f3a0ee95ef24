// Debug bounds checks on the kernels' computed gather / scatter indices.
//
// Built with GVS_BOUNDS_CHECK, GVS_IN_BOUNDS(i, n, site) is true for 0 <= i < n;
// otherwise it records the first offender of this translation unit as
// (site << 48 | low 48 bits of i) and is false, so the caller skips the
// access.  Nothing traps or waits.  Without the macro it is the constant true
// and costs nothing.  gvs_debug_bounds_error (api.cu) collects and clears the
// record of every translation unit.
#pragma once

#include <cuda_runtime.h>

#ifdef GVS_BOUNDS_CHECK
namespace {
__device__ unsigned long long g_bounds_error = 0;  // one per translation unit
__device__ __forceinline__ bool gvs_in_bounds(long long i, long long n, unsigned long long site) {
    if (i >= 0 && i < n) return true;
    atomicCAS(&g_bounds_error, 0ull, (site << 48) | ((unsigned long long)i & 0xffffffffffffull));
    return false;
}
// host side: read and clear this translation unit's record
inline unsigned long long bounds_error_take() {
    unsigned long long v = 0, z = 0;
    cudaMemcpyFromSymbol(&v, g_bounds_error, sizeof(v));
    cudaMemcpyToSymbol(g_bounds_error, &z, sizeof(z));
    return v;
}
}  // namespace
#define GVS_IN_BOUNDS(i, n, site) gvs_in_bounds((long long)(i), (long long)(n), (site))
#define GVS_BOUNDS_TAKE_FN(name) \
    unsigned long long name() { return bounds_error_take(); }
#else
#define GVS_IN_BOUNDS(i, n, site) true
#define GVS_BOUNDS_TAKE_FN(name) \
    unsigned long long name() { return 0ull; }
#endif

// Per translation unit: read and clear its record (0 without GVS_BOUNDS_CHECK).
namespace gvs {
unsigned long long bounds_take_fuse();
unsigned long long bounds_take_fuse_batch();
unsigned long long bounds_take_fuse_bwd();
unsigned long long bounds_take_sphere();
unsigned long long bounds_take_splat();
unsigned long long bounds_take_gauss();
}  // namespace gvs

// Sites (the top 16 bits of a record).
#define GVS_SITE_FUSE_MAP 1ull      // (d, omega) gather of a fusion sample
#define GVS_SITE_FUSE_BOUNDS 2ull   // depth-bound tile of a slab test
#define GVS_SITE_SPLAT_KEY 3ull     // z-buffer atomic of the splat scatter
#define GVS_SITE_SPLAT_SRC 4ull     // winner's colour gather of the resolve
#define GVS_SITE_GAUSS_REC 5ull     // Gaussian record gather of the render
#define GVS_SITE_GAUSS_KEY 6ull     // tile-list write of the fill
#define GVS_SITE_SOFT_ACC 7ull      // key / accumulator of the differentiable splat
