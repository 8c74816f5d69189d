// Dense coupling matrix on the tcgen05 tensor cores.
//
// One DOCH step (Eq. FPE) for dense J and R replicas is a GEMM followed by a
// pointwise update:  U = J X  (n x n by n x R),  X' = cbrt((U + alpha X + h) / beta).
// The energy readout is the same GEMM with the spins S = sign(X):
// q_r = sum_i s_ir (J S)_ir, E_r = -q_r/2 - h^T s_r, cut_r = -(J_sum - q_r)/2
// (Eq. IsingModel; Supplementary Note 5 with W = -2J). Integer J with |J| <= 256
// is exact in BF16 and every (J S) entry is an integer below 2^24, so the FP32
// accumulator and the int64 reduction are exact.
//
// Layout: both operands are stored in HBM as the exact shared-memory images
// the MMA reads, so every pipeline stage is two contiguous bulk copies
// (DRAM pages are read whole, no tensor maps):
//   J  : [m_tiles][kblocks][128 rows][64 columns] BF16, each 16 KB block
//        128-byte swizzled (16-byte chunk c of row r stored at chunk
//        c ^ (r & 7)); rows >= n and columns >= n are zero.
//   X  : replica-major [kblocks][R_pad][64] BF16 with the same swizzle, so
//        the rows r0 .. r0+N-1 of one K block are one contiguous N x 128 B
//        image; spins >= n are zero.
// Tiles: one CTA per (128 rows of J) x (N = up to 256 replicas).
//
// Pipeline per CTA (256 threads):
//   warp 0, one lane: producer. K-block kb (64 columns of J = 64 spins of
//     X) goes to ring stage it % kStages by two cp.async.bulk copies: A tile
//     128 x 64 (16 KB), B tile N x 64 (N x 128 B); arrival tracked by the
//     stage's "full" mbarrier (complete_tx).
//   warp 1, one lane: MMA issuer. Waits "full", issues four
//     tcgen05.mma.kind::f16 (K = 16 each) into the TMEM accumulator, and
//     tcgen05.commit's the stage's "empty" mbarrier (the producer may reuse
//     it once the MMAs that read it complete). After the last block it
//     commits the "accumulator ready" mbarrier.
//   warp 2: allocates and frees the TMEM columns.
//   epilogue, all eight warps once the accumulator is ready: warp w owns
//     TMEM lanes (rows) 32 (w % 4) .. +31 and every other 32-column block
//     from block w / 4; it reads 32 columns at a time (tcgen05.ld 32x32b.x32)
//     and writes the new iterate (cube root as sign(z) 2^(log2|z|/3) with the
//     hardware lg2/ex2 on a power-of-two prescaled z; BF16 output) or the
//     energy partials.
// Every mbarrier wait is bounded (~1 s of %globaltimer); on expiry the CTA
// sets the error word, drains its TMA copies (bounded), frees TMEM, returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>

#include "cbrt.cuh"
#include "internal.cuh"
#include "mbar.cuh"

namespace doch {
namespace {

// Ring stages: 4 with BF16 A and B tiles in shared memory (48 KB per stage);
// 6 in ternary mode, where only B (32 KB) lives in shared memory and A in TMEM.
template <bool TERN> constexpr int kStagesOf = TERN ? 6 : 4;
constexpr int kBM = 128;           // rows of J per tile (MMA M)
constexpr int kBK = 64;            // K per stage: 64 BF16 = 128 bytes = one swizzle row
constexpr int kThreadsTC = 256;

constexpr uint32_t kTernTile = kBM * kBK / 4;  // bytes of one packed ternary J tile (2 bits per entry)
constexpr int kJStages = 8;                      // packed ternary tiles staged ahead

template <bool TERN>
struct DenseSmem {
    static constexpr int kS = kStagesOf<TERN>;
    alignas(1024) unsigned char b[kS][256 * kBK * 2];
    alignas(1024) unsigned char a[TERN ? 1 : kS][TERN ? 1024 : kBM * kBK * 2];  // BF16 A tiles (unused if ternary)
    alignas(16) unsigned char jp[kJStages][kTernTile];  // packed ternary J (ternary mode)
    alignas(8) unsigned long long full[kS];             // B (and BF16 A) landed
    alignas(8) unsigned long long empty[kS];            // MMAs of the stage done
    alignas(8) unsigned long long conv[kS];             // ternary: A tile expanded
    alignas(8) unsigned long long jfull[kJStages];      // ternary: packed tile landed
    alignas(8) unsigned long long jempty[kJStages];     // ternary: packed tile read
    alignas(8) unsigned long long acc_ready;
    uint32_t tmem_base;
    int abort_flag;
};

// contiguous global -> shared copy (16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     saddr(dst)),
                 "l"(src), "r"(bytes), "r"(saddr(bar))
                 : "memory");
}

// element offset of (replica r, spin i) in the swizzled replica-major layout
__host__ __device__ __forceinline__ size_t xs_index(int r, int i, int R_pad) {
    const int kb = i >> 6, c = i & 63;
    return (static_cast<size_t>(kb) * R_pad + r) * 64 + ((((c >> 3) ^ r) & 7) << 3) + (c & 7);
}

// K-major, 128-byte swizzled operand tile: rows are 128 bytes apart, groups of
// 8 rows 1024 bytes apart (stride byte offset); descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc_sw128(const void *tile) {
    const uint64_t start = (saddr(tile) & 0x3FFFFu) >> 4;
    uint64_t d = start;
    d |= static_cast<uint64_t>(1) << 16;           // leading byte offset (unused for swizzled K-major)
    d |= static_cast<uint64_t>(1024 >> 4) << 32;   // stride byte offset
    d |= static_cast<uint64_t>(1) << 46;           // descriptor version
    d |= static_cast<uint64_t>(2) << 61;           // SWIZZLE_128B
    return d;
}

// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// the same MMA with A read from tensor memory (rows in lanes, two BF16 per 32-bit column)
__device__ __forceinline__ void mma_bf16_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem_d),
        "r"(tmem_a), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// 32 consecutive 32-bit columns of this warp's 32 TMEM lanes from registers
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
        "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
        "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void mma_commit(unsigned long long *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}

// BF16 bits of a 2-bit ternary code: 0 -> 0, 1 -> +1, 2 -> -1 (3 unused -> 0)
__device__ __forceinline__ uint32_t tern_bf16(uint32_t code) {
    return code == 1 ? 0x3F80u : (code == 2 ? 0xBF80u : 0u);
}

// MODE 0: DOCH step into Xt_out. MODE 1: energy partials q_r into q_out (int64).
// TERN: J is stored as packed 2-bit codes (entries in {-1, 0, +1}); warps 4-7
// expand each K block into BF16 and store it in tensor memory (columns a_col +
// 32 s for stage s), from where the MMA reads A; shared memory then carries
// only the B tiles, the packed codes and the barriers.
template <int MODE, bool TERN>
__global__ void __launch_bounds__(kThreadsTC, 1)
dense_tc_kernel(const void *__restrict__ jt, const __nv_bfloat16 *__restrict__ xt_in,
                __nv_bfloat16 *__restrict__ xt_out, const float *__restrict__ h, int n, int kblocks, int R,
                int R_pad, int n_tile, uint32_t tmem_cols, uint32_t a_col, float alpha, float zscale,
                float xscale,
                long long *__restrict__ q_out, int *__restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint32_t lut[16];  // ternary: two 2-bit codes -> two BF16
    using Smem = DenseSmem<TERN>;
    constexpr int kStages = Smem::kS;
    Smem &sm = *reinterpret_cast<Smem *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kBM;
    const int r0 = blockIdx.y * n_tile;
    // bytes of J per K block: a BF16 tile, or a packed ternary tile expanded on chip
    constexpr uint32_t a_bytes = TERN ? kTernTile : kBM * kBK * 2;
    const uint32_t b_bytes = static_cast<uint32_t>(n_tile) * kBK * 2;
    const unsigned char *a_src = static_cast<const unsigned char *>(jt) + static_cast<size_t>(blockIdx.x) * kblocks * a_bytes;
    const __nv_bfloat16 *b_src = xt_in + static_cast<size_t>(r0) * kBK;
    volatile int *abort_flag = &sm.abort_flag;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], 1);
        }
        mbar_init(&sm.acc_ready, 1);
        for (int s = 0; s < kStages; ++s) mbar_init(&sm.conv[s], 128);
        for (int p = 0; p < kJStages; ++p) {
            mbar_init(&sm.jfull[p], 1);
            mbar_init(&sm.jempty[p], 128);
        }
        sm.abort_flag = 0;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (TERN && threadIdx.x < 16)
        lut[threadIdx.x] = tern_bf16(threadIdx.x & 3) | (tern_bf16(threadIdx.x >> 2) << 16);
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&sm.tmem_base)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = sm.tmem_base;

    int issued = 0;  // producers: K-blocks whose copies were issued
    // Each CTA walks K from its own starting block kb0 and wraps around, so at
    // any moment the CTAs stream different parts of J (equal 4 MB-aligned
    // offsets in lockstep would queue on the same DRAM channels) and read
    // different blocks of X from L2. Sum order only changes FP32 rounding.
    const int kb0 = static_cast<int>(static_cast<int64_t>(blockIdx.x) * kblocks / gridDim.x);
    if (warp == 0 && lane == 0) {
        for (int it = 0; it < kblocks; ++it) {
            const int s = it % kStages;
            int kb = kb0 + it;
            if (kb >= kblocks) kb -= kblocks;
            if (it >= kStages && !mbar_wait(&sm.empty[s], ((it / kStages) - 1) & 1, err, abort_flag)) break;
            if (TERN) {
                mbar_expect_tx(&sm.full[s], b_bytes);
            } else {
                mbar_expect_tx(&sm.full[s], a_bytes + b_bytes);
                bulk_load(sm.a[s], a_src + static_cast<size_t>(kb) * a_bytes, a_bytes, &sm.full[s]);
            }
            bulk_load(sm.b[s], b_src + static_cast<size_t>(kb) * R_pad * kBK, b_bytes, &sm.full[s]);
            issued = it + 1;
        }
    } else if (warp == 1 && lane == 0) {
        const uint32_t idesc = idesc_bf16(kBM, n_tile);
        bool ok = true;
        for (int it = 0; it < kblocks; ++it) {
            const int s = it % kStages;
            // ternary: A is ready when the converters arrived on conv[s]; B when full[s] completed
            if ((TERN && !mbar_wait(&sm.conv[s], (it / kStages) & 1, err, abort_flag)) ||
                !mbar_wait(&sm.full[s], (it / kStages) & 1, err, abort_flag)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t ad = smem_desc_sw128(sm.a[s]);
            const uint64_t bd = smem_desc_sw128(sm.b[s]);
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k)  // K = 16 per MMA: +32 bytes = +2 in the descriptor
                if (TERN)  // K = 16 BF16 = 8 TMEM columns per MMA
                    mma_bf16_ta(tmem, tmem + a_col + 32 * s + 8 * k, bd + 2 * k, idesc, (it | k) != 0);
                else
                    mma_bf16(tmem, ad + 2 * k, bd + 2 * k, idesc, (it | k) != 0);
            mma_commit(&sm.empty[s]);
        }
        // the accumulator barrier also tracks completion of every MMA issued so far
        mma_commit(&sm.acc_ready);
        if (!ok) {  // error path: let the issued MMAs finish before TMEM is freed
            const uint64_t t0 = gtime();
            while (!mbar_test(&sm.acc_ready, 0) && gtime() - t0 < kWaitNs) {
            }
        }
    } else if (TERN && warp == 3 && lane == 0) {
        // producer of the packed ternary tiles (2 KB each), kJStages ahead
        for (int it = 0; it < kblocks; ++it) {
            const int p = it % kJStages;
            int kb = kb0 + it;
            if (kb >= kblocks) kb -= kblocks;
            if (it >= kJStages && !mbar_wait(&sm.jempty[p], ((it / kJStages) - 1) & 1, err, abort_flag)) break;
            mbar_expect_tx(&sm.jfull[p], a_bytes);
            bulk_load(sm.jp[p], a_src + static_cast<size_t>(kb) * a_bytes, a_bytes, &sm.jfull[p]);
            issued = it + 1;
        }
    } else if (TERN && warp >= 4) {
        // Converters: thread t expands row t of each K block, 64 codes (16 bytes)
        // into 32 columns of two BF16 each and stores them in its TMEM lane t,
        // once the packed tile has landed and the MMAs freed the A stage. The
        // waits are made warp-uniform: tcgen05.st is a .sync.aligned instruction.
        const int t = threadIdx.x - 128;
        const uint32_t a_lane = tmem + (static_cast<uint32_t>(32 * (warp & 3)) << 16) + a_col;
        for (int it = 0; it < kblocks; ++it) {
            const int s = it % kStages, p = it % kJStages;
            if (!__all_sync(0xffffffffu, mbar_wait(&sm.jfull[p], (it / kJStages) & 1, err, abort_flag))) break;
            const uint4 codes = *reinterpret_cast<const uint4 *>(sm.jp[p] + 16 * t);
            mbar_arrive(&sm.jempty[p]);
            if (it >= kStages &&
                !__all_sync(0xffffffffu, mbar_wait(&sm.empty[s], ((it / kStages) - 1) & 1, err, abort_flag)))
                break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t words[4] = {codes.x, codes.y, codes.z, codes.w};
            uint32_t v[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = lut[(words[j >> 3] >> (4 * (j & 7))) & 15];
            tmem_st32(a_lane + 32 * s, v);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(&sm.conv[s]);
        }
    }
    __syncwarp();
    // Epilogue, all eight warps: warp w reads TMEM lanes 32 (w % 4) .. +31 (its
    // 32 rows) and every other 32-column block starting at block w / 4.
    {
        const int q = warp & 3, half = warp >> 2;
        const int row = m0 + 32 * q + lane;
        // warp-uniform decision: tcgen05.ld below is a .sync.aligned warp instruction
        const bool ok = __all_sync(0xffffffffu, mbar_wait_idle(&sm.acc_ready, 0, err, abort_flag) && !*abort_flag);
        if (ok) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const float hv = (h && row < n) ? h[row] : 0.f;
            for (int c0 = 32 * half; c0 < n_tile; c0 += 64) {
                float acc[32];
                tmem_ld32(tmem + (static_cast<uint32_t>(32 * q) << 16) + c0, acc);
                if (MODE == 0) {
                    float xo[32];
#pragma unroll
                    for (int k = 0; k < 32; ++k) {  // all loads first
                        const int r = r0 + c0 + k;
                        xo[k] = (row < n && r < R) ? __bfloat162float(xt_in[xs_index(r, row, R_pad)]) : 0.f;
                    }
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        const int r = r0 + c0 + k;
                        if (row < n && r < R) {
                            const float z = (acc[k] + alpha * xo[k] + hv) * zscale;
                            xt_out[xs_index(r, row, R_pad)] = __float2bfloat16_rn(cbrt_pow2(z) * xscale);
                        }
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        const int r = r0 + c0 + k;
                        long long contrib = 0;
                        if (row < n && r < R) {
                            const float s = __bfloat162float(xt_in[xs_index(r, row, R_pad)]);
                            contrib = static_cast<long long>(s) * static_cast<long long>(acc[k]);
                        }
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, o);
                        if (lane == 0 && r < R && contrib != 0) atomicAdd(reinterpret_cast<unsigned long long *>(q_out + r),
                                                                      static_cast<unsigned long long>(contrib));
                    }
                }
            }
        }
    }
    // drain: the producer waits (bounded) until every copy it issued has landed
    if (warp == 0 && lane == 0 && *abort_flag) {
        for (int it = (issued > kStages ? issued - kStages : 0); it < issued; ++it) {
            const uint64_t t0 = gtime();
            while (!mbar_test(&sm.full[it % kStages], (it / kStages) & 1) && gtime() - t0 < kWaitNs) {
            }
        }
    }
    if (TERN && warp == 3 && lane == 0 && *abort_flag) {
        for (int it = (issued > kJStages ? issued - kJStages : 0); it < issued; ++it) {
            const uint64_t t0 = gtime();
            while (!mbar_test(&sm.jfull[it % kJStages], (it / kJStages) & 1) && gtime() - t0 < kWaitNs) {
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 2) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
    }
}

// x [n][R] (caller layout, BF16) <-> the swizzled replica-major layout
__global__ void to_replica_major(const __nv_bfloat16 *__restrict__ x, __nv_bfloat16 *__restrict__ xt, int n,
                                 int R, int R_pad) {
    __shared__ __nv_bfloat16 tile[32][33];
    const int i0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int i = i0 + k, r = r0 + threadIdx.x;
        tile[k][threadIdx.x] = (i < n && r < R) ? x[static_cast<size_t>(i) * R + r] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, i = i0 + threadIdx.x;
        if (r < R && i < n) xt[xs_index(r, i, R_pad)] = tile[threadIdx.x][k];
    }
}

__global__ void from_replica_major(const __nv_bfloat16 *__restrict__ xt, __nv_bfloat16 *__restrict__ x, int n,
                                   int R, int R_pad) {
    __shared__ __nv_bfloat16 tile[32][33];
    const int i0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, i = i0 + threadIdx.x;
        tile[k][threadIdx.x] = (r < R && i < n) ? xt[xs_index(r, i, R_pad)] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int i = i0 + k, r = r0 + threadIdx.x;
        if (i < n && r < R) x[static_cast<size_t>(i) * R + r] = tile[threadIdx.x][k];
    }
}

// spins (BF16 +1/-1, sign(0) = +1) of iterates of any supported type, replica-major
template <typename XT>
__global__ void spins_replica_major(const XT *__restrict__ x, __nv_bfloat16 *__restrict__ st, int n, int R,
                                    int R_pad) {
    const int64_t total = static_cast<int64_t>(n) * R;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = t / R;
        const int r = static_cast<int>(t - i * R);
        float v;
        if constexpr (sizeof(XT) == 2) v = __bfloat162float(x[t]);
        else v = static_cast<float>(x[t]);
        st[xs_index(r, static_cast<int>(i), R_pad)] = __float2bfloat16_rn(v >= 0.f ? 1.f : -1.f);
    }
}

__global__ void field_dot_spins(const __nv_bfloat16 *__restrict__ st, const int64_t *__restrict__ h, int n,
                                int R_pad, long long *__restrict__ hs) {
    const int r = blockIdx.y;
    long long acc = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        acc += h[i] * static_cast<long long>(__bfloat162float(st[xs_index(r, i, R_pad)]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(reinterpret_cast<unsigned long long *>(hs + r),
                                                  static_cast<unsigned long long>(acc));
}

__global__ void dense_energy_finish(const long long *__restrict__ q, const long long *__restrict__ hs,
                                    long long j_sum, int R, int64_t *E_i, int64_t *cut_i, double *E_d,
                                    double *cut_d) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const long long E = -(q[r] / 2) - hs[r];
    const long long cut = -((j_sum - q[r]) / 2);
    if (E_i) E_i[r] = E;
    if (cut_i) cut_i[r] = cut;
    if (E_d) E_d[r] = static_cast<double>(E);
    if (cut_d) cut_d[r] = static_cast<double>(cut);
}

struct DenseGeom {
    int n, kblocks, R, R_pad, n_tile, m_tiles, r_tiles;
    uint32_t tmem_cols, a_col;  // TMEM columns allocated; first column of the A stages (ternary)
};

DenseGeom geometry(const ising_context *c, int R) {
    DenseGeom g;
    g.n = static_cast<int>(c->n);
    g.kblocks = static_cast<int>(c->dense_ld / kBK);
    g.R = R;
    g.R_pad = R <= 256 ? ((R + 15) / 16) * 16 : ((R + 255) / 256) * 256;
    g.n_tile = g.R_pad < 256 ? g.R_pad : 256;
    g.m_tiles = (g.n + kBM - 1) / kBM;
    g.r_tiles = g.R_pad / g.n_tile;
    uint32_t cols = 32;
    while (cols < static_cast<uint32_t>(g.n_tile)) cols <<= 1;
    g.a_col = cols;
    if (c->dense_ternary) {  // + one 32-column A tile per stage, rounded up to a power of two
        cols += kStagesOf<true> * 32;
        uint32_t p2 = 32;
        while (p2 < cols) p2 <<= 1;
        cols = p2;
    }
    g.tmem_cols = cols;
    return g;
}

template <bool TERN>
size_t smem_bytes() { return sizeof(DenseSmem<TERN>) + 1024; }

template <int MODE>
ising_status_t launch_dense(const ising_context *c, const DenseGeom &g, const __nv_bfloat16 *xt_in,
                            __nv_bfloat16 *xt_out, const float *h, float alpha, float zscale, float xscale,
                            long long *q_out, cudaStream_t st) {
    auto kern = c->dense_ternary ? dense_tc_kernel<MODE, true> : dense_tc_kernel<MODE, false>;
    const size_t smem = c->dense_ternary ? smem_bytes<true>() : smem_bytes<false>();
    DOCH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    dim3 grid(static_cast<unsigned>(g.m_tiles), static_cast<unsigned>(g.r_tiles));
    kern<<<grid, kThreadsTC, smem, st>>>(c->dense, xt_in, xt_out, h, g.n,
                                                 g.kblocks, g.R, g.R_pad, g.n_tile, g.tmem_cols, g.a_col, alpha,
                                                 zscale, xscale, q_out, c->err_word);
    DOCH_CUDA(cudaGetLastError());
    return ISING_OK;
}

}  // namespace

ising_status_t dense_iterate(ising_context *c, void *x, int R, const double *alpha_h, int alpha_len,
                             double beta, int iters, cudaStream_t st) {
    const DenseGeom g = geometry(c, R);
    const size_t xt_bytes = static_cast<size_t>(g.R_pad) * g.kblocks * kBK * 2;
    DOCH_CHECK(c->work.ensure(2 * xt_bytes));
    __nv_bfloat16 *xt[2] = {c->work.as<__nv_bfloat16>(),
                            reinterpret_cast<__nv_bfloat16 *>(c->work.as<unsigned char>() + xt_bytes)};
    DOCH_CUDA(cudaMemsetAsync(c->work.ptr, 0, 2 * xt_bytes, st));
    dim3 tb(32, 8), tg((g.n + 31) / 32, (R + 31) / 32);
    to_replica_major<<<tg, tb, 0, st>>>(static_cast<const __nv_bfloat16 *>(x), xt[0], g.n, R, g.R_pad);
    DOCH_CUDA(cudaGetLastError());
    // cube root on (z 2^(3k)) / beta, rescaled by 2^-k (exact powers of two, k from beta)
    const double inv_beta = 1.0 / beta;
    const int ks = cbrt_prescale_exp(inv_beta);
    const float zscale = static_cast<float>(std::ldexp(inv_beta, 3 * ks));
    const float xscale = std::ldexp(1.0f, -ks);
    int cur = 0;
    for (int k = 0; k < iters; ++k) {
        const float a = static_cast<float>(alpha_h[alpha_len == 1 ? 0 : k]);
        DOCH_CHECK(launch_dense<0>(c, g, xt[cur], xt[1 - cur], c->h_f32, a, zscale, xscale, nullptr, st));
        cur = 1 - cur;
    }
    from_replica_major<<<tg, tb, 0, st>>>(xt[cur], static_cast<__nv_bfloat16 *>(x), g.n, R, g.R_pad);
    DOCH_CUDA(cudaGetLastError());
    return ISING_OK;
}

ising_status_t dense_energy(ising_context *c, const void *x, int xtype, int R, int64_t *E_i, int64_t *cut_i,
                            double *E_d, double *cut_d, cudaStream_t st) {
    const DenseGeom g = geometry(c, R);
    const size_t st_bytes = static_cast<size_t>(g.R_pad) * g.kblocks * kBK * 2;
    DOCH_CHECK(c->partials.ensure(st_bytes + 2 * sizeof(long long) * R + 256));
    __nv_bfloat16 *sp = c->partials.as<__nv_bfloat16>();
    long long *q = reinterpret_cast<long long *>(c->partials.as<unsigned char>() + ((st_bytes + 255) & ~size_t(255)));
    long long *hs = q + R;
    DOCH_CUDA(cudaMemsetAsync(c->partials.ptr, 0, c->partials.bytes, st));
    const int64_t total = static_cast<int64_t>(g.n) * R;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 16LL * c->num_sms) blocks = 16LL * c->num_sms;
    switch (xtype) {
        case ISING_BF16: spins_replica_major<<<blocks, 256, 0, st>>>(static_cast<const __nv_bfloat16 *>(x), sp, g.n, R, g.R_pad); break;
        case ISING_F32: spins_replica_major<<<blocks, 256, 0, st>>>(static_cast<const float *>(x), sp, g.n, R, g.R_pad); break;
        case ISING_F64: spins_replica_major<<<blocks, 256, 0, st>>>(static_cast<const double *>(x), sp, g.n, R, g.R_pad); break;
        case ISING_I8: spins_replica_major<<<blocks, 256, 0, st>>>(static_cast<const int8_t *>(x), sp, g.n, R, g.R_pad); break;
        default: return fail(ISING_ERR_INVALID_ARG, "dense energy: x type");
    }
    DOCH_CUDA(cudaGetLastError());
    DOCH_CHECK(launch_dense<1>(c, g, sp, nullptr, nullptr, 0.f, 0.f, 0.f, q, st));
    if (c->h_i64) {
        dim3 fg(static_cast<unsigned>((g.n + 255) / 256 < 64 ? (g.n + 255) / 256 : 64), static_cast<unsigned>(R));
        field_dot_spins<<<fg, 256, 0, st>>>(sp, c->h_i64, g.n, g.R_pad, hs);
        DOCH_CUDA(cudaGetLastError());
    }
    dense_energy_finish<<<(R + 127) / 128, 128, 0, st>>>(q, hs, c->dense_jsum, R, E_i, cut_i, E_d, cut_d);
    DOCH_CUDA(cudaGetLastError());
    return ISING_OK;
}

}  // namespace doch
