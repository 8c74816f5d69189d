// Real (odd) cube root used by the FP32 stencil kernel.
//
// cbrt(z) = sign(z) * 2^(log2|z| / 3), with the hardware approximations of
// the base-2 logarithm and exponential (PTX lg2.approx.ftz.f32 and
// ex2.approx.ftz.f32). Applied to z' = z * 2^(-3k) and rescaled by 2^k, which
// is exact (powers of two) and keeps |log2 z'| small, so the FP32 logarithm
// does not lose absolute precision on the very small z of the method
// (z ~ beta^(-3/2)). Relative error ~2^-22 for normal z'; z' = 0 and
// subnormal z' give 0. Tested against cbrtf through ising_selftest_cbrt.
#pragma once

#include <cmath>

namespace doch {

__device__ __forceinline__ float cbrt_pow2(float z) {
    float l, y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(fabsf(z)));
    l *= (1.0f / 3.0f);
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(l));
    return copysignf(y, z);
}

// exponent k of the prescale: 2^(3k) / beta puts z 2^(3k) near 1 at the
// attractor scale x ~ beta^(-1/2) of Eq. alphabeta's beta
inline int cbrt_prescale_exp(double inv_beta) {
    int k = static_cast<int>(std::lround(-0.5 * std::log2(inv_beta)));
    if (k > 40) k = 40;
    if (k < -40) k = -40;
    return k;
}

}  // namespace doch
