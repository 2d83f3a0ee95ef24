// Sphere-tracing raymarch (Supplement A.1): arguments and launch entry shared
// by sphere.cu and the C ABI.
#pragma once

#include "gvs_internal.cuh"

namespace gvs {

struct SphereArgs {
    FuseArgs f;        // map (float2, correctly rounded weights), views, target, zn, inv_mu, fused
    float zf;          // march ends past z_far (FP32)
    float c08mu;       // 0.8 mu rounded once to FP32
    float min_frac;    // smallest normalised step
    int max_steps;
    int32_t *evals;    // [Ht][Wt] samples evaluated per ray, or null
};

cudaError_t launch_sphere(const SphereArgs &s, cudaStream_t st);

}  // namespace gvs
