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

}  // namespace doch
