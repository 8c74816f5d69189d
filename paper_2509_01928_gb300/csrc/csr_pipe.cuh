// Loads of the CSR row pipeline. A thread that owns rows i, i + S, i + 2S, ...
// keeps the next row's first batch of column / value entries and the entry range
// of the row after it in flight while the current row's neighbours are gathered,
// so a row waits for one round of memory latency instead of three
// (row_ptr -> col -> gather).
#pragma once

#include <cstdint>

namespace doch {

// entry range [e0, e1) of row i (empty past the last row), in the kernel's index type IT
// (32-bit where the rows and entries allow it: fewer registers, more resident warps)
template <typename IT>
__device__ __forceinline__ void pipe_row_range(const int64_t *__restrict__ row_ptr, IT i, IT n, IT &e0, IT &e1) {
    if (i < n) {
        e0 = static_cast<IT>(__ldg(row_ptr + i));
        e1 = static_cast<IT>(__ldg(row_ptr + i + 1));
    } else {
        e0 = e1 = 0;
    }
}

// the first B entries of [e0, e1): columns and values as AT (0 past the end)
template <int B, typename AT, typename VT, typename IT>
__device__ __forceinline__ void pipe_first_batch(const int32_t *__restrict__ col, const VT *__restrict__ val,
                                                 IT e0, IT e1, int32_t (&js)[B], AT (&ws)[B]) {
    const int m = e1 - e0 < B ? static_cast<int>(e1 - e0) : B;
    const int32_t *c = col + e0;
    const VT *v = val + e0;
#pragma unroll
    for (int t = 0; t < B; ++t) {
        js[t] = t < m ? __ldg(c + t) : 0;
        ws[t] = t < m ? static_cast<AT>(__ldg(v + t)) : AT(0);
    }
}

}  // namespace doch
