// Dense coupling matrix, plain FP32 form: the DOCH step of Eq. FPE,
//   U = J X  (n x n by n x R),  X' = cbrt((U + alpha X + h) / beta),
// with FP32 iterates, FP32 products and FP32 accumulation on the CUDA cores
// (no tensor cores, no reduced-precision state). It is the reference form the
// BF16 tensor-core kernel (k_dense_tc.cu) is compared with at equal final
// energy; both read the same device copy of J.
//
// J is read from the handle's tensor-core tile order (128 rows x 64 columns
// per tile, [m_tile][k_block] order): packed 2-bit codes when every entry is
// -1, 0 or +1 (2 KB per tile, row-major, 4 codes per byte from the low bits:
// 0 -> 0, 1 -> +1, 2 -> -1), BF16 otherwise (16 KB per tile, 16-byte chunk c
// of row r stored at chunk c ^ (r & 7)). Both are exact integers, decoded to
// FP32 in shared memory.
//
// Tiling: one CTA (256 threads) per 128 rows of J x 128 replicas; each thread
// owns an 8 x 8 block of U (rows ty*4 + {0..3} and 64 + ty*4 + {0..3}, columns
// tx*4 + {0..3} and 64 + tx*4 + {0..3}, so the shared-memory fragment loads
// are 16-byte vectors without bank conflicts). K advances one 64-column tile
// of J per stage: two shared-memory stages (A = J tile transposed to [k][m],
// B = X rows [k][r], FP32), the next stage's global data is loaded into
// registers while the current one is multiplied. The epilogue applies the
// update in FP32 with CUDA's cbrtf and writes the new iterate [n][R].
#include <cuda_bf16.h>

#include <cmath>

#include "internal.cuh"

namespace doch {
namespace {

constexpr int kFM = 128;       // rows of J per CTA
constexpr int kFN = 128;       // replicas per CTA
constexpr int kFK = 64;        // columns of J per stage (one tile of the handle's layout)
constexpr int kFThreads = 256;

struct F32Smem {
    float a[2][kFK][kFM];  // J tile, transposed: a[s][k][m]
    float b[2][kFK][kFN];  // X rows: b[s][k][r]
};

__device__ __forceinline__ float tern_value(uint32_t code) {
    return code == 1u ? 1.f : (code == 2u ? -1.f : 0.f);
}

// Raw A data of one tile held in registers between load and store: thread t
// owns row m = t % 128 and columns 32 * (t / 128) .. + 31 of the tile.
template <bool TERN> struct ARaw;
template <> struct ARaw<true> { uint2 w; };            // 32 codes = 8 bytes
template <> struct ARaw<false> { uint4 c[4]; };        // 32 BF16 = 4 chunks of 16 bytes

__device__ __forceinline__ void load_a(const unsigned char *__restrict__ J, int64_t tile, ARaw<true> &raw) {
    const int t = threadIdx.x, m = t & 127, half = t >> 7;
    raw.w = __ldg(reinterpret_cast<const uint2 *>(J + tile * (kFM * kFK / 4) + m * 16 + half * 8));
}

__device__ __forceinline__ void load_a(const unsigned char *__restrict__ J, int64_t tile, ARaw<false> &raw) {
    const int t = threadIdx.x, m = t & 127, half = t >> 7;
    const uint4 *row = reinterpret_cast<const uint4 *>(J + tile * (kFM * kFK * 2) + m * 128);
#pragma unroll
    for (int q = 0; q < 4; ++q) raw.c[q] = __ldg(row + ((half * 4 + q) ^ (m & 7)));
}

__device__ __forceinline__ void store_a(float (*a)[kFM], const ARaw<true> &raw) {
    const int t = threadIdx.x, m = t & 127, k0 = (t >> 7) * 32;
#pragma unroll
    for (int j = 0; j < 16; ++j) a[k0 + j][m] = tern_value((raw.w.x >> (2 * j)) & 3u);
#pragma unroll
    for (int j = 0; j < 16; ++j) a[k0 + 16 + j][m] = tern_value((raw.w.y >> (2 * j)) & 3u);
}

__device__ __forceinline__ void store_a(float (*a)[kFM], const ARaw<false> &raw) {
    const int t = threadIdx.x, m = t & 127, k0 = (t >> 7) * 32;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const __nv_bfloat162 *v = reinterpret_cast<const __nv_bfloat162 *>(&raw.c[q]);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float2 f = __bfloat1622float2(v[e]);
            a[k0 + q * 8 + 2 * e][m] = f.x;
            a[k0 + q * 8 + 2 * e + 1][m] = f.y;
        }
    }
}

// B: 64 rows of X (spins kb*64 ..) x 128 replicas (c0 ..); thread t loads
// rows 8 * (t / 32) .. + 7, columns 4 * (t % 32) .. + 3 (zero beyond n or R).
struct BRaw { float4 v[8]; };

__device__ __forceinline__ void load_b(const float *__restrict__ x, int n, int R, int k_base, int c0, bool vec,
                                       BRaw &raw) {
    const int t = threadIdx.x, r0 = (t >> 5) * 8, col = c0 + (t & 31) * 4;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int row = k_base + r0 + i;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row < n) {
            const float *p = x + static_cast<int64_t>(row) * R + col;
            if (vec && col + 3 < R) {
                v = __ldg(reinterpret_cast<const float4 *>(p));
            } else {
                if (col < R) v.x = __ldg(p);
                if (col + 1 < R) v.y = __ldg(p + 1);
                if (col + 2 < R) v.z = __ldg(p + 2);
                if (col + 3 < R) v.w = __ldg(p + 3);
            }
        }
        raw.v[i] = v;
    }
}

__device__ __forceinline__ void store_b(float (*b)[kFN], const BRaw &raw) {
    const int t = threadIdx.x, r0 = (t >> 5) * 8, c = (t & 31) * 4;
#pragma unroll
    for (int i = 0; i < 8; ++i) *reinterpret_cast<float4 *>(&b[r0 + i][c]) = raw.v[i];
}

template <bool TERN>
__global__ void __launch_bounds__(kFThreads, 1)
dense_f32_step(const unsigned char *__restrict__ J, const float *__restrict__ x, float *__restrict__ xo,
               const float *__restrict__ h, int n, int kblocks, int R, float alpha, float inv_beta) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    F32Smem &sm = *reinterpret_cast<F32Smem *>(smem_raw);
    const int mt = blockIdx.x, m0 = mt * kFM, c0 = blockIdx.y * kFN;
    const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
    const bool vec = (R & 3) == 0;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    ARaw<TERN> ar;
    BRaw br;
    load_a(J, static_cast<int64_t>(mt) * kblocks, ar);
    load_b(x, n, R, 0, c0, vec, br);
    store_a(sm.a[0], ar);
    store_b(sm.b[0], br);
    __syncthreads();
    for (int kb = 0; kb < kblocks; ++kb) {
        const int s = kb & 1;
        const bool more = kb + 1 < kblocks;
        if (more) {  // next stage's global data, held in registers during the products
            load_a(J, static_cast<int64_t>(mt) * kblocks + kb + 1, ar);
            load_b(x, n, R, (kb + 1) * kFK, c0, vec, br);
        }
#pragma unroll 8
        for (int k = 0; k < kFK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&sm.a[s][k][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&sm.a[s][k][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&sm.b[s][k][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&sm.b[s][k][64 + tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (more) {  // the other stage was last read before the previous barrier
            store_a(sm.a[s ^ 1], ar);
            store_b(sm.b[s ^ 1], br);
        }
        __syncthreads();
    }
    // epilogue: z = (u + alpha x + h) / beta, x' = cbrt(z), all in FP32
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int row = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
        if (row >= n) continue;
        const float hr = h ? h[row] : 0.f;
#pragma unroll
        for (int jh = 0; jh < 2; ++jh) {
            const int col = c0 + jh * 64 + tx * 4;
            const int64_t base = static_cast<int64_t>(row) * R + col;
            if (vec && col + 3 < R) {
                const float4 xv = __ldg(reinterpret_cast<const float4 *>(x + base));
                float4 o;
                o.x = cbrtf((acc[i][jh * 4 + 0] + alpha * xv.x + hr) * inv_beta);
                o.y = cbrtf((acc[i][jh * 4 + 1] + alpha * xv.y + hr) * inv_beta);
                o.z = cbrtf((acc[i][jh * 4 + 2] + alpha * xv.z + hr) * inv_beta);
                o.w = cbrtf((acc[i][jh * 4 + 3] + alpha * xv.w + hr) * inv_beta);
                *reinterpret_cast<float4 *>(xo + base) = o;
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (col + j < R)
                        xo[base + j] = cbrtf((acc[i][jh * 4 + j] + alpha * x[base + j] + hr) * inv_beta);
            }
        }
    }
}

}  // namespace

ising_status_t dense_iterate_f32(ising_context *c, float *x, int R, const double *alpha_h, int alpha_len,
                                 double beta, int iters, cudaStream_t st) {
    if (iters <= 0) return ISING_OK;
    const int n = static_cast<int>(c->n);
    const int kblocks = static_cast<int>(c->dense_ld / kFK);
    const size_t xbytes = static_cast<size_t>(n) * R * sizeof(float);
    DOCH_CHECK(c->ping.ensure(xbytes));
    float *buf[2] = {x, c->ping.as<float>()};
    auto kern = c->dense_ternary ? dense_f32_step<true> : dense_f32_step<false>;
    const int smem = static_cast<int>(sizeof(F32Smem));
    DOCH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    dim3 grid(static_cast<unsigned>((n + kFM - 1) / kFM), static_cast<unsigned>((R + kFN - 1) / kFN));
    const float inv_beta = static_cast<float>(1.0 / beta);
    int cur = 0;
    for (int k = 0; k < iters; ++k) {
        const float a = static_cast<float>(alpha_h[alpha_len == 1 ? 0 : k]);
        kern<<<grid, kFThreads, smem, st>>>(static_cast<const unsigned char *>(c->dense), buf[cur], buf[1 - cur],
                                            c->h_f32, n, kblocks, R, a, inv_beta);
        DOCH_CUDA(cudaGetLastError());
        cur = 1 - cur;
    }
    if (cur != 0) DOCH_CUDA(cudaMemcpyAsync(x, buf[cur], xbytes, cudaMemcpyDeviceToDevice, st));
    return ISING_OK;
}

}  // namespace doch
