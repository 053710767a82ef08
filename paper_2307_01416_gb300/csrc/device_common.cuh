// Device primitives shared by the transport and surrogate kernels: the
// counter-based generator, its uniform and normal variates, and the
// beam's-eye-view to patient transform.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "vpmc_internal.cuh"

namespace vpmc {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32 -> 64-bit
// multiplications with the published multipliers and Weyl key increments.
// Each product is formed once as a 64-bit value (one wide multiply gives
// both halves).
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k.x, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k.y, (uint32_t)p0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// ((x >> 9) + 1/2) * 2^-23: 23-bit uniform in (0, 1), exact in FP32.
__device__ __forceinline__ float u01(uint32_t x) { return fmaf(__uint2float_rn(x >> 9), 0x1p-23f, 0x1p-24f); }

// (v + 1/2) * 2^-21 for a 21-bit v: the per-step uniforms, exact in FP32.
__device__ __forceinline__ float u21(uint32_t v) { return fmaf(__uint2float_rn(v), 0x1p-21f, 0x1p-22f); }

// Box-Muller with accurate functions (source sampling, once per history).
__device__ __forceinline__ float2 box_muller(float u1, float u2)
{
    const float r = sqrtf(-2.0f * logf(u1));
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    return make_float2(r * c, r * s);
}

// Beam's-eye view (a, b, t) -> patient coordinates with the scenario's shift.
__device__ __forceinline__ void bev_to_patient(const DevBeam& B, const DevScen& sc, const float pb[3], float out[3])
{
#pragma unroll
    for (int k = 0; k < 3; ++k)
        out[k] = B.iso[k] + sc.shift[k] + pb[0] * B.u[k] + pb[1] * B.v[k] + pb[2] * B.w[k];
}

}  // namespace dev
}  // namespace vpmc
