// gelu.cuh -- the surrogate network's activation on the GPU, used by the
// GEMM epilogues (mlp_gemm.cu).
#pragma once

#include <cuda_runtime.h>

namespace paam_gelu {

// The network's activation: GELU in its tanh form (Hendrycks and Gimpel,
// "Gaussian Error Linear Units", 2016),
//   gelu(z) = z (1 + tanh(u)) / 2,  u = sqrt(2 / pi) (z + 0.044715 z^3),
// evaluated through (1 + tanh(u)) / 2 = 1 / (1 + exp(-2u)) with one base-2
// exponential and one reciprocal (PTX ex2.approx / rcp.approx, relative error
// near 2^-22), so the result is the tanh form to about 1e-6 relative: far below
// the bf16 step (2^-8) of the stored activations.  The exponent is clamped so
// the reciprocal never sees infinity.
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// sigmoid(2u) for the activation at z
__device__ __forceinline__ float gelu_gate(float z)
{
    // -2u log2(e) = z (k0 + k1 z^2), k0 = -2 sqrt(2/pi) log2(e), k1 = 0.044715 k0
    constexpr float k0 = -2.3022082f, k1 = -0.10294324f;
    const float w = fminf(z * fmaf(k1, z * z, k0), 126.0f);
    return rcp_approx(1.0f + ex2_approx(w));
}

__device__ __forceinline__ float gelu(float z) { return z * gelu_gate(z); }

// d/dz z s(z), s = sigmoid(2u): s + z s (1 - s) d(2u)/dz, d(2u)/dz = c0 + 3 c1 z^2
__device__ __forceinline__ float gelu_grad(float z)
{
    constexpr float c0 = 1.5957691f, c1x3 = 0.21406444f; // 2 sqrt(2/pi), 3 * 0.044715 * c0
    const float g = gelu_gate(z);
    return fmaf(z * g * (1.0f - g), fmaf(c1x3, z * z, c0), g);
}

} // namespace paam_gelu
