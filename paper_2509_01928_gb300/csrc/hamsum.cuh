// Compensated per-thread sums of the fused H monitor (Eq. Hamilton terms).
#pragma once

namespace doch {

// One running sum: compensated (Kahan) in FP32 for FP32 iterates, plain FP64
// for FP64 iterates.
template <typename XT>
struct HamSum {
    XT s = XT(0), c = XT(0);
    __device__ __forceinline__ void add(XT v) {
        if constexpr (sizeof(XT) == 4) {
            const XT y = v - c;
            const XT t = s + y;
            c = (t - s) - y;
            s = t;
        } else {
            s += v;
        }
    }
    __device__ __forceinline__ double value() const { return static_cast<double>(s) - static_cast<double>(c); }
};

// Compensated FP32 sum of terms or of products a_i b_i. Each product is rounded once
// (__fmul_rn, so that no FMA contraction moves it) and its rounding error,
// recovered exactly by an FMA (a b = p + e), joins the Kahan compensation c;
// value() = s - c in FP64. Error ~2^-44 of sum |a_i b_i| for a few hundred
// terms, on the FP32 pipes: FP64 throughput on this part is a small fraction
// of FP32's.
struct DotSum32 {
    float s = 0.f, c = 0.f;
    // one term v (Kahan)
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    // one product a b, split exactly
    __device__ __forceinline__ void add(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float e = fmaf(a, b, -p);
        const float y = p - c;
        const float t = s + y;
        c = ((t - s) - y) - e;
        s = t;
    }
    __device__ __forceinline__ double value() const { return static_cast<double>(s) - static_cast<double>(c); }
};

}  // namespace doch
