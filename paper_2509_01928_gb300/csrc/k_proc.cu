// Procedural dense couplings (Supplementary Note 9, on one GPU the block
// product of Algorithm S6): J_ij = sin(i j + c) for 1-based i != j, J_ii = 0,
// generated where they are used and never stored.
//
// Phase. With F = floor(2^96 / (2 pi)), the 96-bit integer (a F) mod 2^96 is
// frac(a / (2 pi)) 2^96 to within a units (a fixed-point argument reduction in
// the manner of Payne and Hanek, exact in integers). Along row i the phase of
// column j + 1 is that of column j plus (i F) mod 2^96; the kernels keep the top
// 64 bits of both (the truncation adds at most one 2^-64 turn per column) and
// advance four columns at a time on four independent chains.
// Coupling. Between resynchronisations from the 64-bit phase (every 32
// columns) a column's top 32 bits advance by the rounded top 32 bits of the
// increment (at most 16 units of 2^-32 turn of drift). With s those bits as a
// signed integer, the angle is pi y for y = s / 2^31 in [-1, 1), and
// sin(pi y) = sign(y) cos(pi (|y| - 1/2)) with pi (|y| - 1/2) in
// [-pi/2, pi/2]; the cosine is an even polynomial of degree 8 whose
// coefficients minimise the largest absolute error on the interval (Remez
// exchange). Measured against the FP64 sine of the exact phase, the FP32
// couplings are within 3.3e-7 (rms 6.0e-8), about one FP32 unit in the last
// place of a coupling of size 1/2 to 1.
// Product. One thread per row, CTAs of kPT rows, the columns in tiles of kPN
// staged in shared memory (each value read by all threads: a broadcast);
// per-tile sums, then a sum over the tiles of a column split. The splits
// (blockIdx.y) give enough CTAs to fill the GPU for any n; their partial sums
// go to a scratch array [split][n][R] that a finishing kernel adds in split
// order, so results do not depend on the schedule.
// The sums of J and of J^2 over i != j (for the cut and the Wigner estimate)
// come in closed form from geometric series of the sines, in FP64 on the host;
// the rows' sums of |J_ij| (Eq. alphabeta) from the symmetric product with |J|.
#include <algorithm>
#include <cmath>
#include <vector>

#include "cbrt.cuh"
#include "internal.cuh"

namespace doch {
namespace {

constexpr int kPT = 256;  // rows per CTA (one per thread)
constexpr int kPN = 256;  // columns per shared-memory tile (kPN == kPT: one diagonal tile per CTA)

// top 64 bits of (a G) mod 2^96 for the 96-bit constant G = (g2, g1, g0)
__host__ __device__ __forceinline__ uint64_t mulmod96_top(uint64_t a, uint32_t g2, uint32_t g1, uint32_t g0) {
    const uint64_t a0 = a & 0xFFFFFFFFull, a1 = a >> 32;
    const uint64_t c0 = a0 * g0;
    const uint64_t s1 = a0 * g1 + (c0 >> 32);
    const uint64_t s2 = a1 * g0 + (s1 & 0xFFFFFFFFull);
    const uint32_t w2 = static_cast<uint32_t>(a0 * g2 + a1 * g1 + (s1 >> 32) + (s2 >> 32));
    return (static_cast<uint64_t>(w2) << 32) | (s2 & 0xFFFFFFFFull);
}

// floor(2^96 / (2 pi)): the phase of an integer argument in turns
__host__ __device__ __forceinline__ uint64_t phase64(uint64_t a) {
    return mulmod96_top(a, 0x28BE60DBu, 0x9391054Au, 0x7F09D5F4u);
}

// J for the top 32 bits t of the phase: with s = (int32) t and y = s / 2^31,
// sin(pi y) = sign(y) cos(pi (|y| - 1/2)); the argument pi |y| - pi/2 is one
// multiply-add from the float of |s| (whose rounding, and that of the two
// constants, moves it by at most 2.4e-7 where |y| is near 1 and sin(pi y) is
// near 0), the cosine a minimax even polynomial of degree 8 (4.7e-8 before
// rounding)
__device__ __forceinline__ float coupling(uint32_t t) {
    const float a = static_cast<float>(abs(static_cast<int32_t>(t)));  // |INT_MIN| wraps to the same angle
    const float x = fmaf(a, 1.4629180792671596e-09f, -1.5707963267948966f);
    const float u = x * x;
    float q = 2.3153931635876185e-05f;
    q = fmaf(q, u, -0.0013853704307259674f);
    q = fmaf(q, u, 0.041663584693001555f);
    q = fmaf(q, u, -0.49999905347077034f);
    q = fmaf(q, u, 0.9999999534666968f);
    return __uint_as_float(__float_as_uint(q) ^ (t & 0x80000000u));
}

// the top 32 bits of a phase increment, rounded
__device__ __forceinline__ uint32_t top32_rounded(uint64_t d) {
    return static_cast<uint32_t>((d + 0x80000000ull) >> 32);
}

// One kPN-column tile for RC replicas: tacc[r] = sum_j J_ij x_jr. P[4] are
// the phases of the next four columns (64-bit, advanced by D4 = 4 D per group
// and resynchronised into 32-bit chains every 8 groups). For
// RC <= 2 each of the four column chains has its own sums (64 terms each,
// added pairwise at the end), which shortens the FP32 summation; wider
// replica groups sum the tile in one chain per replica.
template <int RC, bool DIAG>
__device__ __forceinline__ void tile_pass(const float *__restrict__ tf, uint64_t (&P)[4], uint64_t D4,
                                          float (&tacc)[RC], int diag_col) {
    constexpr int kCh = RC <= 2 ? 4 : 1;
    float ch[kCh][RC];
#pragma unroll
    for (int k = 0; k < kCh; ++k)
#pragma unroll
        for (int r = 0; r < RC; ++r) ch[k][r] = 0.f;
    const uint32_t d4 = top32_rounded(D4);
    for (int j8 = 0; j8 < kPN; j8 += 32) {
        uint32_t t[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            t[u] = static_cast<uint32_t>(P[u] >> 32);
            P[u] += 8 * D4;
        }
#pragma unroll
        for (int jj = j8; jj < j8 + 32; jj += 4) {
            float w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                w[u] = coupling(t[u]);
                t[u] += d4;
                if (DIAG && jj + u == diag_col) w[u] = 0.f;
            }
            if constexpr (RC < 4) {
                float v[4 * RC];
#pragma unroll
                for (int q = 0; q < RC; ++q) {
                    const float4 g = reinterpret_cast<const float4 *>(tf + jj * RC)[q];
                    v[4 * q] = g.x;
                    v[4 * q + 1] = g.y;
                    v[4 * q + 2] = g.z;
                    v[4 * q + 3] = g.w;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int r = 0; r < RC; ++r) ch[u % kCh][r] = fmaf(w[u], v[u * RC + r], ch[u % kCh][r]);
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
#pragma unroll
                    for (int q = 0; q < RC / 4; ++q) {
                        const float4 g = reinterpret_cast<const float4 *>(tf + (jj + u) * RC)[q];
                        ch[0][4 * q] = fmaf(w[u], g.x, ch[0][4 * q]);
                        ch[0][4 * q + 1] = fmaf(w[u], g.y, ch[0][4 * q + 1]);
                        ch[0][4 * q + 2] = fmaf(w[u], g.z, ch[0][4 * q + 2]);
                        ch[0][4 * q + 3] = fmaf(w[u], g.w, ch[0][4 * q + 3]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < RC; ++r) {
        if constexpr (kCh == 4) tacc[r] = (ch[0][r] + ch[1][r]) + (ch[2][r] + ch[3][r]);
        else tacc[r] = ch[0][r];
    }
}

// part[split][i][rc0 + r] = sum over the split's columns j != i of J_ij x_j(rc0 + r).
// XT = float (iterates) or int8_t (spins).
template <int RC, typename XT>
__global__ void __launch_bounds__(kPT)
proc_partial(const XT *__restrict__ x, float *__restrict__ part, int64_t n, int R, int rc0, int64_t offset,
             int tiles_per_split, int n_tiles) {
    __shared__ __align__(16) float tf[kPN * RC];
    const int64_t row0 = static_cast<int64_t>(blockIdx.x) * kPT;
    const int64_t i = row0 + threadIdx.x;
    const int t0 = static_cast<int>(blockIdx.y) * tiles_per_split;
    const int t1 = min(n_tiles, t0 + tiles_per_split);
    const uint64_t i1 = static_cast<uint64_t>(i) + 1;
    const uint64_t D = phase64(i1);
    uint64_t P[4];
    P[0] = phase64(i1 * (static_cast<uint64_t>(t0) * kPN + 1) + static_cast<uint64_t>(offset));
    P[1] = P[0] + D;
    P[2] = P[1] + D;
    P[3] = P[2] + D;
    const uint64_t D4 = 4 * D;
    float acc[RC];
#pragma unroll
    for (int r = 0; r < RC; ++r) acc[r] = 0.f;
    const int rcn = min(RC, R - rc0);
    for (int t = t0; t < t1; ++t) {
        const int64_t j0 = static_cast<int64_t>(t) * kPN;
        __syncthreads();
        for (int e = threadIdx.x; e < kPN * RC; e += kPT) {
            const int jj = e / RC, r = e - jj * RC;
            const int64_t j = j0 + jj;
            float v = 0.f;
            if (j < n && r < rcn) v = static_cast<float>(x[j * R + rc0 + r]);
            tf[e] = v;
        }
        __syncthreads();
        float tacc[RC];
        if (j0 == row0) tile_pass<RC, true>(tf, P, D4, tacc, threadIdx.x);
        else tile_pass<RC, false>(tf, P, D4, tacc, -1);
#pragma unroll
        for (int r = 0; r < RC; ++r) acc[r] += tacc[r];
    }
    if (i >= n) return;
    float *dst = part + (static_cast<int64_t>(blockIdx.y) * n + i) * R + rc0;
#pragma unroll
    for (int r = 0; r < RC; ++r)
        if (r < rcn) dst[r] = acc[r];
}

// x_out = cbrt((u + alpha x) / beta) with u = sum of the split partials (in split order)
__global__ void proc_finish_step(const float *__restrict__ part, int S, const float *__restrict__ x,
                                 float *__restrict__ xo, int64_t count, float alpha, float zs, float xsc) {
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < count;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        float u = part[e];
        for (int s = 1; s < S; ++s) u += part[static_cast<int64_t>(s) * count + e];
        xo[e] = cbrt_pow2((u + alpha * x[e]) * zs) * xsc;
    }
}

constexpr int kQT = 256;

// qpart[r][block] = sum over the block's rows of s_ir u_ir in FP64 (fixed order)
__global__ void __launch_bounds__(kQT)
proc_finish_quad(const float *__restrict__ part, int S, const int8_t *__restrict__ s, int64_t n, int R,
                 double *__restrict__ qpart) {
    const int r = blockIdx.y;
    const int64_t count = n * R;
    const int64_t rows_per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = static_cast<int64_t>(blockIdx.x) * rows_per, hi = min(n, lo + rows_per);
    double q = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kQT) {
        const int64_t e = i * R + r;
        float u = part[e];
        for (int k = 1; k < S; ++k) u += part[static_cast<int64_t>(k) * count + e];
        q += static_cast<double>(s[e]) * static_cast<double>(u);
    }
    __shared__ double red[kQT];
    red[threadIdx.x] = q;
    __syncthreads();
    for (int w = kQT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) qpart[static_cast<int64_t>(r) * gridDim.x + blockIdx.x] = red[0];
}

// the couplings of rows row0.. and columns col0.. as the product kernels generate
// them (64-bit phase at every 32nd column, 32-bit chain in between)
__global__ void proc_couplings(int64_t row0, int rows, int64_t col0, int cols, int64_t offset,
                               float *__restrict__ out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const uint64_t i1 = static_cast<uint64_t>(row0 + r) + 1;
    const uint64_t D = phase64(i1);
    const uint32_t d = top32_rounded(D);
    uint64_t P = phase64(i1 * (static_cast<uint64_t>(col0) + 1) + static_cast<uint64_t>(offset));
    uint32_t t = 0;
    for (int j = 0; j < cols; ++j) {
        if ((j & 31) == 0) {
            t = static_cast<uint32_t>(P >> 32);
            P += 32 * D;
        }
        out[static_cast<int64_t>(r) * cols + j] = row0 + r == col0 + j ? 0.f : coupling(t);
        t += d;
    }
}

// H(x) of Eq. Hamilton per replica (no field), one block per replica, FP64 in a fixed order:
// beta/4 sum x^4 - alpha/2 sum x^2 - 1/2 sum x u with u = J x
__global__ void __launch_bounds__(kQT)
proc_ham(const float *__restrict__ x, const float *__restrict__ u, int64_t n, int R, const double *__restrict__ alpha_d,
         int alpha_len, int k, const double *__restrict__ beta_d, double *__restrict__ H_out) {
    const int r = blockIdx.x;
    double s4 = 0.0, s2 = 0.0, su = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kQT) {
        const double xv = x[i * R + r];
        const double x2 = xv * xv;
        s4 += x2 * x2;
        s2 += x2;
        su += xv * static_cast<double>(u[i * R + r]);
    }
    __shared__ double red[3][kQT];
    red[0][threadIdx.x] = s4;
    red[1][threadIdx.x] = s2;
    red[2][threadIdx.x] = su;
    __syncthreads();
    for (int w = kQT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int t = 0; t < 3; ++t) red[t][threadIdx.x] += red[t][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double a = alpha_d[k < alpha_len ? k : alpha_len - 1], b = beta_d[0];
        H_out[r] = b / 4.0 * red[0][0] - a / 2.0 * red[1][0] - 0.5 * red[2][0];
    }
}

struct SplitPlan {
    int row_blocks, n_tiles, tiles_per_split, S;
};

SplitPlan plan_splits(const ising_context *c) {
    SplitPlan p;
    p.row_blocks = static_cast<int>((c->n + kPT - 1) / kPT);
    p.n_tiles = static_cast<int>((c->n + kPN - 1) / kPN);
    // at least 16 CTAs per SM over the whole launch (so the last wave is a small share)
    const int64_t want = 16LL * c->num_sms;
    int S = static_cast<int>(std::min<int64_t>((want + p.row_blocks - 1) / p.row_blocks, p.n_tiles));
    S = std::max(1, std::min(S, 65535));
    p.tiles_per_split = (p.n_tiles + S - 1) / S;
    p.S = (p.n_tiles + p.tiles_per_split - 1) / p.tiles_per_split;
    return p;
}

// the partial products of every replica chunk into part [S][n][R]
template <typename XT>
ising_status_t proc_products(const ising_context *c, const XT *x, float *part, int R, const SplitPlan &pl,
                             cudaStream_t st) {
    const dim3 grid(static_cast<unsigned>(pl.row_blocks), static_cast<unsigned>(pl.S));
    for (int rc0 = 0; rc0 < R; rc0 += 16) {
        const int left = R - rc0;
#define DOCH_PROC_LAUNCH(RCV)                                                                                 \
    proc_partial<RCV, XT><<<grid, kPT, 0, st>>>(x, part, c->n, R, rc0, c->proc_offset, pl.tiles_per_split, \
                                                pl.n_tiles)
        if (left == 1) DOCH_PROC_LAUNCH(1);
        else if (left == 2) DOCH_PROC_LAUNCH(2);
        else if (left <= 4) DOCH_PROC_LAUNCH(4);
        else if (left <= 8) DOCH_PROC_LAUNCH(8);
        else DOCH_PROC_LAUNCH(16);
#undef DOCH_PROC_LAUNCH
        DOCH_CUDA(cudaGetLastError());
    }
    return ISING_OK;
}

int stream_blocks(const ising_context *c, int64_t count) {
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((count + 255) / 256, 8LL * c->num_sms)));
}


// ---- one replica: each generated coupling serves both J_ij x_j and J_ji x_i ----
//
// Row tiles of kSR kPT = 1024 rows (kSR rows per thread, rows r0 + t + 256 k).
// A tile's own 1024 x 1024 diagonal block runs as rows only (j != i tested);
// every column j beyond the tile is taken once, in column tiles of 256: the
// thread adds J_ij x_j to its rows' sums and J_ij x_i to per-lane column sums,
// which a 32-lane butterfly (each step halves the columns a lane holds) and a
// fixed-order sum over the 8 warps reduce to one value per column. Rows and
// columns receive their contributions from many CTAs, so they accumulate as
// int64 fixed-point numbers (scale 2^k with n max|x| 2^k < 2^61): integer
// additions commute, so the atomics give the same sums in any order. Each
// added value is an FP32 sum over at most 256 terms (columns) or 1024 terms
// (rows of a column), rounded once to the fixed point (relative 2^-61 n).

constexpr int kSR = 4;             // rows per thread
constexpr int kSTR = kSR * kPT;    // rows per row tile
constexpr int kSTC = 256;          // columns per column tile
constexpr int kSUnit = 64;         // column tiles per work unit

// lane l returns the sum over the warp's lanes of v[l] (v[b]: column b of a 32-column chunk)
__device__ __forceinline__ float reduce_scatter32(float (&v)[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        const bool up = lane & m;
#pragma unroll
        for (int b = 0; b < m; ++b) {
            const float send = up ? v[b] : v[b + m];
            const float keep = up ? v[b + m] : v[b];
            v[b] = keep + __shfl_xor_sync(0xffffffffu, send, m);
        }
    }
    return v[0];
}

// exponent k of the fixed-point scale 2^k with n m 2^k < 2^60 for m = max |x| (1 for spins)
__host__ __device__ __forceinline__ int fixed_exp(float m, int64_t n) {
    if (!(m > 0.f)) return 0;
    int e;
    frexpf(m * static_cast<float>(n), &e);  // m n < 2^e up to the rounding of the product
    const int k = 59 - e;
    return k < -120 ? -120 : (k > 120 ? 120 : k);
}

__global__ void proc_maxabs(const float *__restrict__ x, int64_t n, unsigned *__restrict__ out) {
    float m = 0.f;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        m = fmaxf(m, fabsf(x[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));  // non-negative floats order as integers
}

// ABS: row and column sums of |J_ij| (x taken as all ones, not read)
template <typename XT, bool DIAG, bool ABS>
__device__ __forceinline__ void sym_unit(const XT *__restrict__ x, unsigned long long *__restrict__ acc, float scale,
                                         int4 un, int64_t n, int64_t offset) {
    __shared__ __align__(16) float xs[kSTC];
    __shared__ float red[kPT / 32][kSTC];
    const int64_t r0 = static_cast<int64_t>(un.x) * kSTR;
    const int64_t c_begin = DIAG ? r0 : static_cast<int64_t>(un.y) * kSTC;
    const int ntile = DIAG ? static_cast<int>((min(n, r0 + kSTR) - r0 + kSTC - 1) / kSTC) : un.z;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float xr[kSR];
    uint64_t P[kSR], D32[kSR];  // phase at the next 32-column chunk, its advance per chunk
    uint32_t d[kSR];            // rounded top 32 bits of the per-column increment
    long long racc[kSR];
#pragma unroll
    for (int k = 0; k < kSR; ++k) {
        const int64_t i = r0 + threadIdx.x + kPT * k;
        xr[k] = i < n ? (ABS ? 1.f : static_cast<float>(x[i])) : 0.f;
        const uint64_t i1 = static_cast<uint64_t>(i) + 1;
        const uint64_t D = phase64(i1);
        D32[k] = 32 * D;
        d[k] = top32_rounded(D);
        P[k] = phase64(i1 * (static_cast<uint64_t>(c_begin) + 1) + static_cast<uint64_t>(offset));
        racc[k] = 0;
    }
    for (int tile = 0; tile < ntile; ++tile) {
        const int64_t c0 = c_begin + static_cast<int64_t>(tile) * kSTC;
        __syncthreads();
        xs[threadIdx.x] = c0 + threadIdx.x < n ? (ABS ? 1.f : static_cast<float>(x[c0 + threadIdx.x])) : 0.f;
        __syncthreads();
        float trs[kSR];
#pragma unroll
        for (int k = 0; k < kSR; ++k) trs[k] = 0.f;
        for (int chunk = 0; chunk < kSTC / 32; ++chunk) {
            float col[32], crs[kSR];
            uint32_t tk[kSR];
#pragma unroll
            for (int k = 0; k < kSR; ++k) {
                crs[k] = 0.f;
                tk[k] = static_cast<uint32_t>(P[k] >> 32);
                P[k] += D32[k];
            }
#pragma unroll
            for (int b4 = 0; b4 < 32; b4 += 4) {
                const float4 xq = *reinterpret_cast<const float4 *>(xs + chunk * 32 + b4);
                const float xv[4] = {xq.x, xq.y, xq.z, xq.w};
#pragma unroll
                for (int bb = 0; bb < 4; ++bb) {
                    const int b = b4 + bb;
#pragma unroll
                    for (int k = 0; k < kSR; ++k) {
                        float w = coupling(tk[k]);
                        if (ABS) w = fabsf(w);
                        tk[k] += d[k];
                        if (DIAG && c0 + chunk * 32 + b == r0 + threadIdx.x + kPT * k) w = 0.f;
                        crs[k] = fmaf(w, xv[bb], crs[k]);
                        if (!DIAG) col[b] = k == 0 ? w * xr[0] : fmaf(w, xr[k], col[b]);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < kSR; ++k) trs[k] += crs[k];
            if (!DIAG) red[warp][chunk * 32 + lane] = reduce_scatter32(col);
        }
#pragma unroll
        for (int k = 0; k < kSR; ++k) racc[k] += __float2ll_rn(trs[k] * scale);
        if (!DIAG) {
            __syncthreads();
            float cs = 0.f;
#pragma unroll
            for (int w = 0; w < kPT / 32; ++w) cs += red[w][threadIdx.x];
            if (c0 + threadIdx.x < n)
                atomicAdd(acc + c0 + threadIdx.x, static_cast<unsigned long long>(__float2ll_rn(cs * scale)));
        }
    }
#pragma unroll
    for (int k = 0; k < kSR; ++k) {
        const int64_t i = r0 + threadIdx.x + kPT * k;
        if (i < n) atomicAdd(acc + i, static_cast<unsigned long long>(racc[k]));
    }
}

// unit: (row tile, first column tile, column tiles, 1 = diagonal block); m > 0: fixed max |x|
template <typename XT, bool ABS = false>
__global__ void __launch_bounds__(kPT, 2)
proc_sym(const XT *__restrict__ x, unsigned long long *__restrict__ acc, const unsigned *__restrict__ maxbits,
         float m, const int4 *__restrict__ units, int64_t n, int64_t offset) {
    const int4 un = units[blockIdx.x];
    const float scale = ldexpf(1.f, fixed_exp(m > 0.f ? m : __uint_as_float(*maxbits), n));
    if (un.w) sym_unit<XT, true, ABS>(x, acc, scale, un, n, offset);
    else sym_unit<XT, false, ABS>(x, acc, scale, un, n, offset);
}

// u = the fixed-point sums as floats (clears them)
__global__ void proc_sym_to_float(unsigned long long *__restrict__ acc, const unsigned *__restrict__ maxbits,
                                  float *__restrict__ u, int64_t n) {
    const double inv = ldexp(1.0, -fixed_exp(__uint_as_float(*maxbits), n));
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        u[i] = static_cast<float>(static_cast<double>(static_cast<long long>(acc[i])) * inv);
        acc[i] = 0ull;
    }
}

// per block: max over rows of the fixed-point sums (FP64); clears them
__global__ void __launch_bounds__(kQT)
proc_sym_rowmax(unsigned long long *__restrict__ acc, int64_t n, double inv, double *__restrict__ bmax) {
    double m = 0.0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kQT + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kQT) {
        m = fmax(m, static_cast<double>(static_cast<long long>(acc[i])) * inv);
        acc[i] = 0ull;
    }
    __shared__ double red[kQT];
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = kQT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) bmax[blockIdx.x] = red[0];
}

// u = sum of the split partials in split order
__global__ void proc_sum_splits(const float *__restrict__ part, int S, float *__restrict__ u, int64_t count) {
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < count;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        float v = part[e];
        for (int s = 1; s < S; ++s) v += part[static_cast<int64_t>(s) * count + e];
        u[e] = v;
    }
}

// x_out = cbrt((u + alpha x) / beta) with u the fixed-point sums; clears them
__global__ void proc_sym_finish(unsigned long long *__restrict__ acc, const unsigned *__restrict__ maxbits,
                                const float *__restrict__ x, float *__restrict__ xo, int64_t n, float alpha,
                                float zs, float xsc) {
    const double inv = ldexp(1.0, -fixed_exp(__uint_as_float(*maxbits), n));
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float u = static_cast<float>(static_cast<double>(static_cast<long long>(acc[i])) * inv);
        acc[i] = 0ull;
        xo[i] = cbrt_pow2((u + alpha * x[i]) * zs) * xsc;
    }
}

// qpart[block] = sum over the block's rows of s_i u_i (FP64, fixed order); clears the sums
__global__ void __launch_bounds__(kQT)
proc_sym_quad(unsigned long long *__restrict__ acc, const int8_t *__restrict__ s, int64_t n, double inv,
              double *__restrict__ qpart) {
    const int64_t rows_per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = static_cast<int64_t>(blockIdx.x) * rows_per, hi = min(n, lo + rows_per);
    double q = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kQT) {
        q += static_cast<double>(s[i]) * (static_cast<double>(static_cast<long long>(acc[i])) * inv);
        acc[i] = 0ull;
    }
    __shared__ double red[kQT];
    red[threadIdx.x] = q;
    __syncthreads();
    for (int w = kQT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) qpart[blockIdx.x] = red[0];
}

// work units of the symmetric product (diagonal blocks first), and the
// accumulators [n] int64 + the max |x| word, zeroed once
ising_status_t sym_setup(ising_context *c) {
    if (c->proc_units_count > 0) return ISING_OK;
    const int64_t n = c->n;
    const int64_t rt = (n + kSTR - 1) / kSTR, ct = (n + kSTC - 1) / kSTC;
    int64_t total = rt;  // counted before anything is allocated
    for (int64_t I = 0; I < rt; ++I) {
        const int64_t first = (I + 1) * (kSTR / kSTC);
        if (first < ct) total += (ct - first + kSUnit - 1) / kSUnit;
    }
    if (total > 0x7FFFFFFF) return fail(ISING_ERR_UNSUPPORTED, "procedural product: too many work units");
    std::vector<int4> u;
    u.reserve(static_cast<size_t>(total));
    for (int64_t I = 0; I < rt; ++I) u.push_back(make_int4(static_cast<int>(I), 0, 0, 1));
    for (int64_t I = 0; I < rt; ++I) {
        const int64_t first = (I + 1) * (kSTR / kSTC);
        for (int64_t t = first; t < ct; t += kSUnit)
            u.push_back(make_int4(static_cast<int>(I), static_cast<int>(t),
                                  static_cast<int>(std::min<int64_t>(kSUnit, ct - t)), 0));
    }
    DOCH_CHECK(c->proc_units.ensure(sizeof(int4) * u.size()));
    DOCH_CUDA(cudaMemcpy(c->proc_units.ptr, u.data(), sizeof(int4) * u.size(), cudaMemcpyHostToDevice));
    DOCH_CHECK(c->proc_acc.ensure(sizeof(unsigned long long) * n + 256));
    DOCH_CUDA(cudaMemset(c->proc_acc.ptr, 0, sizeof(unsigned long long) * n + 256));
    c->proc_units_count = static_cast<int>(u.size());
    return ISING_OK;
}

unsigned *sym_maxword(ising_context *c) {
    return reinterpret_cast<unsigned *>(c->proc_acc.as<unsigned long long>() + c->n);
}

// m/2 radians for an integer m < 2^64, reduced to [-pi, pi): the turn
// fraction m / (4 pi) from floor(2^96 / (4 pi)) in integers
double half_angle(uint64_t m) {
    const uint64_t top = mulmod96_top(m, 0x145F306Du, 0xC9C882A5u, 0x3F84EAFAu);
    return static_cast<double>(static_cast<int64_t>(top)) * (6.283185307179586476925 / 18446744073709551616.0);
}

struct Neumaier {
    double s = 0.0, c = 0.0;
    void add(double v) {
        const double t = s + v;
        c += std::fabs(s) >= std::fabs(v) ? (s - t) + v : (v - t) + s;
        s = t;
    }
    double value() const { return s + c; }
};

}  // namespace

// sum_{i != j} J_ij and sum_{i != j} J_ij^2 by the geometric series
//   sum_{j=1..n} sin(c + j i) = sin(c + (n+1) i / 2) sin(n i / 2) / sin(i / 2),
//   sum_{j=1..n} cos(2c + 2 j i) = cos(2c + (n+1) i) sin(n i) / sin(i),
// with J_ij^2 = (1 - cos(2 i j + 2 c)) / 2, less the diagonal terms.
void proc_closed_sums(int64_t n, int64_t c, double *s1, double *s2) {
    Neumaier a, b;
    const uint64_t un = static_cast<uint64_t>(n), uc = static_cast<uint64_t>(c);
    for (uint64_t i = 1; i <= un; ++i) {
        const uint64_t m_sum = 2 * uc + (un + 1) * i;  // c + (n+1) i / 2 in half radians
        const double rs = std::sin(half_angle(m_sum)) * std::sin(half_angle(un * i)) / std::sin(half_angle(i));
        const double rc = std::cos(half_angle(2 * m_sum)) * std::sin(half_angle(2 * un * i)) /
                          std::sin(half_angle(2 * i));
        const uint64_t m_d = 2 * (i * i + uc);
        a.add(rs - std::sin(half_angle(m_d)));
        b.add(rc - std::cos(half_angle(2 * m_d)));
    }
    *s1 = a.value();
    *s2 = 0.5 * (static_cast<double>(n) * (static_cast<double>(n) - 1.0) - b.value());
}

ising_status_t proc_step(ising_context *c, const float *x_in, float *x_out, int R, double alpha, double inv_beta,
                         cudaStream_t st) {
    const int k = cbrt_prescale_exp(inv_beta);
    const float zs = static_cast<float>(std::ldexp(inv_beta, 3 * k));
    const float xsc = std::ldexp(1.0f, -k);
    if (R == 1) {
        DOCH_CHECK(sym_setup(c));
        unsigned *mw = sym_maxword(c);
        DOCH_CUDA(cudaMemsetAsync(mw, 0, sizeof(unsigned), st));
        proc_maxabs<<<stream_blocks(c, c->n), 256, 0, st>>>(x_in, c->n, mw);
        proc_sym<float><<<c->proc_units_count, kPT, 0, st>>>(x_in, c->proc_acc.as<unsigned long long>(), mw, 0.f,
                                                           c->proc_units.as<int4>(), c->n, c->proc_offset);
        proc_sym_finish<<<stream_blocks(c, c->n), 256, 0, st>>>(c->proc_acc.as<unsigned long long>(), mw, x_in,
                                                              x_out, c->n, static_cast<float>(alpha), zs, xsc);
        DOCH_CUDA(cudaGetLastError());
        return ISING_OK;
    }
    const SplitPlan pl = plan_splits(c);
    const int64_t count = c->n * R;
    DOCH_CHECK(c->partials.ensure(sizeof(float) * count * pl.S));
    float *part = c->partials.as<float>();
    DOCH_CHECK(proc_products<float>(c, x_in, part, R, pl, st));
    proc_finish_step<<<stream_blocks(c, count), 256, 0, st>>>(part, pl.S, x_in, x_out, count,
                                                             static_cast<float>(alpha), zs, xsc);
    DOCH_CUDA(cudaGetLastError());
    return ISING_OK;
}

// E = -1/2 s^T J s and cut = -1/2 (sum_{i != j} J_ij - s^T J s) per replica, into
// E_d and cut_d (device, R each)
ising_status_t proc_energy(ising_context *c, const void *x, int xtype, int R, double *E_d, double *cut_d,
                           cudaStream_t st) {
    const SplitPlan pl = plan_splits(c);
    const int64_t count = c->n * R;
    const int qb = static_cast<int>(std::min<int64_t>((c->n + kQT - 1) / kQT, 64));
    const size_t part_b = (sizeof(float) * count * pl.S + 255) & ~size_t(255);
    const size_t spin_b = (static_cast<size_t>(count) + 255) & ~size_t(255);
    DOCH_CHECK(c->partials.ensure(part_b + spin_b + sizeof(double) * R * qb));
    float *part = c->partials.as<float>();
    int8_t *s = reinterpret_cast<int8_t *>(c->partials.as<unsigned char>() + part_b);
    double *qp = reinterpret_cast<double *>(c->partials.as<unsigned char>() + part_b + spin_b);
    DOCH_CHECK(write_spins(c, x, xtype, R, s, st));
    if (R == 1) {
        DOCH_CHECK(sym_setup(c));
        proc_sym<int8_t><<<c->proc_units_count, kPT, 0, st>>>(s, c->proc_acc.as<unsigned long long>(), nullptr, 1.f,
                                                            c->proc_units.as<int4>(), c->n, c->proc_offset);
        const double inv = std::ldexp(1.0, -fixed_exp(1.f, c->n));
        proc_sym_quad<<<qb, kQT, 0, st>>>(c->proc_acc.as<unsigned long long>(), s, c->n, inv, qp);
    } else {
        DOCH_CHECK(proc_products<int8_t>(c, s, part, R, pl, st));
        proc_finish_quad<<<dim3(qb, R), kQT, 0, st>>>(part, pl.S, s, c->n, R, qp);
    }
    DOCH_CUDA(cudaGetLastError());
    std::vector<double> qh(static_cast<size_t>(R) * qb);
    DOCH_CUDA(cudaMemcpyAsync(qh.data(), qp, sizeof(double) * qh.size(), cudaMemcpyDeviceToHost, st));
    DOCH_CUDA(cudaStreamSynchronize(st));
    std::vector<double> E(R), cut(R);
    for (int r = 0; r < R; ++r) {
        double q = 0.0;
        for (int b = 0; b < qb; ++b) q += qh[static_cast<size_t>(r) * qb + b];
        E[r] = -0.5 * q;
        cut[r] = -0.5 * (c->proc_s1 - q);
    }
    DOCH_CUDA(cudaMemcpyAsync(E_d, E.data(), sizeof(double) * R, cudaMemcpyHostToDevice, st));
    DOCH_CUDA(cudaMemcpyAsync(cut_d, cut.data(), sizeof(double) * R, cudaMemcpyHostToDevice, st));
    DOCH_CUDA(cudaStreamSynchronize(st));
    return ISING_OK;
}

// u = J x (FP32, [n][R]), for the ADOCH passes
ising_status_t proc_product(ising_context *c, const float *x, float *u, int R, cudaStream_t st) {
    if (R == 1) {
        DOCH_CHECK(sym_setup(c));
        unsigned *mw = sym_maxword(c);
        DOCH_CUDA(cudaMemsetAsync(mw, 0, sizeof(unsigned), st));
        proc_maxabs<<<stream_blocks(c, c->n), 256, 0, st>>>(x, c->n, mw);
        proc_sym<float><<<c->proc_units_count, kPT, 0, st>>>(x, c->proc_acc.as<unsigned long long>(), mw, 0.f,
                                                           c->proc_units.as<int4>(), c->n, c->proc_offset);
        proc_sym_to_float<<<stream_blocks(c, c->n), 256, 0, st>>>(c->proc_acc.as<unsigned long long>(), mw, u, c->n);
        DOCH_CUDA(cudaGetLastError());
        return ISING_OK;
    }
    const SplitPlan pl = plan_splits(c);
    const int64_t count = c->n * R;
    DOCH_CHECK(c->partials.ensure(sizeof(float) * count * pl.S));
    float *part = c->partials.as<float>();
    DOCH_CHECK(proc_products<float>(c, x, part, R, pl, st));
    proc_sum_splits<<<stream_blocks(c, count), 256, 0, st>>>(part, pl.S, u, count);
    DOCH_CUDA(cudaGetLastError());
    return ISING_OK;
}

// H(x^k) of Eq. Hamilton per replica into H_out [R] (device): one product and an FP64 reduction
ising_status_t proc_hamiltonian(ising_context *c, const float *x, int R, const ParamTabs &p, int k, double *H_out,
                                cudaStream_t st) {
    DOCH_CHECK(c->proc_u.ensure(sizeof(float) * c->n * R));
    float *u = c->proc_u.as<float>();
    DOCH_CHECK(proc_product(c, x, u, R, st));
    proc_ham<<<R, kQT, 0, st>>>(x, u, c->n, R, p.alpha_d, p.alpha_len, k, p.beta_d, H_out);
    DOCH_CUDA(cudaGetLastError());
    return ISING_OK;
}

// Eq. alphabeta with the Wigner estimate of Eq. estimate_eig_J; the row sums
// of |J_ij| by the symmetric product with |J| and all-ones x
ising_status_t proc_params(ising_context *c, double eta, double *alpha, double *beta) {
    DOCH_CHECK(sym_setup(c));
    constexpr int kMB = 64;
    DevBuf b;
    DOCH_CHECK(b.ensure(sizeof(double) * kMB));
    proc_sym<float, true><<<c->proc_units_count, kPT>>>(nullptr, c->proc_acc.as<unsigned long long>(), nullptr, 1.f,
                                                       c->proc_units.as<int4>(), c->n, c->proc_offset);
    proc_sym_rowmax<<<kMB, kQT>>>(c->proc_acc.as<unsigned long long>(), c->n, std::ldexp(1.0, -fixed_exp(1.f, c->n)),
                                  b.as<double>());
    cudaError_t e = cudaGetLastError();
    std::vector<double> h(kMB);
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), b.ptr, sizeof(double) * kMB, cudaMemcpyDeviceToHost);
    b.release();
    if (e != cudaSuccess) return cuda_fail(e, "procedural row sums");
    const double rowmax = *std::max_element(h.begin(), h.end());
    const double n = static_cast<double>(c->n);
    const double cnt = n * (n - 1.0);
    const double mean = c->proc_s1 / cnt;
    const double var = std::max(0.0, c->proc_s2 / cnt - mean * mean);
    *alpha = eta * 2.0 * std::sqrt(var) * std::sqrt(n);
    *beta = std::pow(n, 1.5) * (*alpha + rowmax);
    return ISING_OK;
}

}  // namespace doch

extern "C" ising_status_t ising_selftest_procedural(int64_t row0, int32_t rows, int64_t col0, int32_t cols,
                                                    int64_t c, float *J_out, void *stream) {
    return doch::guarded([&]() -> ising_status_t {
        using namespace doch;
        if (!J_out || row0 < 0 || col0 < 0 || rows < 0 || cols < 0 || c < 0 || c > (int64_t(1) << 40) ||
            row0 + rows > (int64_t(1) << 30) || col0 + cols > (int64_t(1) << 30))
            return fail(ISING_ERR_INVALID_ARG, "selftest_procedural: bad argument");
        if (rows == 0 || cols == 0) return ISING_OK;
        const cudaStream_t st = static_cast<cudaStream_t>(stream);
        proc_couplings<<<(rows + 127) / 128, 128, 0, st>>>(row0, rows, col0, cols, c, J_out);
        DOCH_CUDA(cudaGetLastError());
        DOCH_CUDA(cudaStreamSynchronize(st));
        return ISING_OK;
    });
}
