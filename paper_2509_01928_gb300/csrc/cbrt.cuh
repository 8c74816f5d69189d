// Real (odd) cube roots of the FP32 kernels: cbrt_pow2 (CSR, batched, dense,
// procedural and ADOCH kernels) and cbrt_log (the lattice DOCH kernels).
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

// cbrt(z / beta) as sign(z) 2^(log2|z| / 3 + c3) with c3 = -log2(beta) / 3 given:
// one FMA joins the division by three and the scale, and no products by the
// power-of-two prescale are needed (two instructions fewer than cbrt_pow2 with
// its scales). The FP32 value l = log2|z| / 3 + c3 carries an absolute rounding
// of (|log2 z| / 3 + |l|) 2^-24, which exp2 turns into a relative error of at
// most ln 2 times that; with the hardware log2/exp2 approximations the error is
// within 2^-21 + (0.25 |log2 z| + 0.75 |l|) 2^-24. In the lattice iteration |l|
// and |log2 z| stay near the attractor scale. z = 0 and subnormal z give 0.
// Tested against cbrt through ising_selftest_cbrt_log.
__device__ __forceinline__ float cbrt_log(float z, float c3) {
    float l, y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(fabsf(z)));
    l = fmaf(l, 1.0f / 3.0f, c3);
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
