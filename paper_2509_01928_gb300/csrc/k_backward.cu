// Adjoint of N DOCH steps (derived from Eq. FPE; the paper has no gradients).
//
// Precision: the forward iterates (checkpoints and recomputed segments) are
// FP32 or FP64 as the caller's x0; the adjoint recursion (g, w) runs in FP32.
// The FP64 forward exists because d x^(k+1) / d x^k contains
// 1 / (3 (x^(k+1))^2): components that pass near zero in the transient make
// the gradient sensitive to the trajectory, and an FP32 trajectory shifts
// those factors enough to move some gradients by 1e-3..1e-1 relative on
// random regular graphs. Along an FP64 trajectory the FP32 adjoint is
// accurate to ~1e-6.
//
// Loss: L = (1/R) sum_r ( -1/2 x_r^T J x_r - h^T x_r ) at x^N.
//   g^N = dL/dx^N = -(1/R) (J x^N + h)
//   for k = N-1 .. 0 (x^(k+1) = cbrt(z^k), dx^(k+1)/dz^k = 1 / (3 (x^(k+1))^2)):
//     w^k = g^(k+1) / (3 (x^(k+1))^2)            (0 where x^(k+1) = 0, counted)
//     dL/dalpha_k = sum_{i,r} w^k_ir x^k_ir / beta
//     g^k = (J w^k + alpha_k w^k) / beta           (J = J^T)
//   dL/dx^0 = g^0.
//
// Memory: x is kept only every C steps (checkpoints); each segment is
// recomputed from its checkpoint with the forward kernel (deterministic, so
// the recomputed iterates equal the forward ones) before its adjoint steps
// run. The adjoint kernel of step k gathers w^k at the neighbours and forms, for
// its own rows, g^k and the next step's w^(k-1) = g^k / (3 (x^k)^2): one
// gather per neighbour; the loss kernel forms w^(N-1) from g^N. dL/dalpha_k and the loss
// are summed per thread (for FP32 iterates a compensated FP32 sum: of the row's
// FP32 dot product in the adjoint step, of exact product splits in the loss;
// FP64 arithmetic runs at a small fraction of the FP32 rate on this part; FP64
// for FP64 iterates), then in FP64 across threads, blocks and launches in a
// fixed order (run-to-run identical). The weights 1 / (3 x^2) use the fast
// division (within 2 ulp) where the denominator is a normal number.
//
// Thread layout as in the forward CSR kernel: one thread per (row, chunk of
// V = 4/2/1 replicas), grid-stride over a grid of one resident wave. The adjoint
// step pipelines its loads across the rows of a thread (row i, i + S, i + 2S, ...):
// while row i's neighbours are gathered, the first batch of column / value
// entries of row i + S and the row_ptr pair of row i + 2S are in flight, so a
// row waits for one round of memory latency instead of three (row_ptr -> col ->
// gather). Entries past a row's first batch follow one at a time, in entry order.
#include "csr_pipe.cuh"
#include "hamsum.cuh"
#include "internal.cuh"

namespace doch {
namespace {

constexpr int kBThreads = 256;
constexpr int kBatchB = 4;  // entries whose loads are issued together

template <int V> struct F4;
template <> struct F4<1> { using type = float; };
template <> struct F4<2> { using type = float2; };
template <> struct F4<4> { using type = float4; };

template <int V>
__device__ __forceinline__ void ld(const float *p, float (&v)[V]) {
    using T = typename F4<V>::type;
    const T w = __ldg(reinterpret_cast<const T *>(p));
    const float *q = reinterpret_cast<const float *>(&w);
#pragma unroll
    for (int k = 0; k < V; ++k) v[k] = q[k];
}

// FP64 iterates: loaded as doubles (two 16-byte loads for V = 4)
template <int V>
__device__ __forceinline__ void ld(const double *p, double (&v)[V]) {
    if constexpr (V == 4) {
        const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
        const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    } else if constexpr (V == 2) {
        const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
        v[0] = a.x; v[1] = a.y;
    } else {
        v[0] = __ldg(p);
    }
}

template <int V>
__device__ __forceinline__ void st(float *p, const float (&v)[V]) {
    using T = typename F4<V>::type;
    T w;
    float *q = reinterpret_cast<float *>(&w);
#pragma unroll
    for (int k = 0; k < V; ++k) q[k] = v[k];
    *reinterpret_cast<T *>(p) = w;
}

// w = g / (3 x^2), 0 where x = 0: the fast division (within 2 ulp) for a normal
// denominator below 2^126, the IEEE division for the rest
__device__ __forceinline__ float dcbrt_weight(float g, float x) {
    const float d = 3.0f * x * x;
    if (d >= 0x1p-126f && d < 0x1p126f) return __fdividef(g, d);
    return x == 0.0f ? 0.0f : g / d;
}

__device__ __forceinline__ double block_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __shared__ double red[kBThreads / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kBThreads / 32; ++w) t += red[w];
    __syncthreads();
    return t;
}

// g^N = -(J x^N + h) / R and per-block partial sums of -1/2 x u - h x (per thread
// a compensated FP32 sum of the products for FP32 iterates, FP64 for FP64 ones;
// FP64 across the block); the kernel stores w^(N-1) = g^N / (3 (x^N)^2) (0 where x^N = 0, counted), the
// quantity the first adjoint step gathers. The product u is formed in the
// iterate type XT.
template <typename XT, typename VT, int V>
__global__ void __launch_bounds__(kBThreads)
loss_w_kernel(const XT *__restrict__ x, float *__restrict__ w, const int64_t *__restrict__ row_ptr,
              const int32_t *__restrict__ col, const VT *__restrict__ val, const XT *__restrict__ h,
              int64_t n, int R, double *__restrict__ part, unsigned long long *__restrict__ zeros) {
    const int C = R / V;
    const XT invR = XT(1) / static_cast<XT>(R);
    double acc = 0.0;
    DotSum32 acc32;
    unsigned nz = 0;
    const int rows_per_block = kBThreads / C;
    const int ch = threadIdx.x % C;
    const int rl = threadIdx.x / C;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * rows_per_block + rl; rl < rows_per_block && i < n;
         i += static_cast<int64_t>(gridDim.x) * rows_per_block) {
        XT u[V];
#pragma unroll
        for (int q = 0; q < V; ++q) u[q] = XT(0);
        const int64_t e1 = __ldg(row_ptr + i + 1);
        for (int64_t e = __ldg(row_ptr + i); e < e1; e += kBatchB) {
            const int cnt = e1 - e < kBatchB ? static_cast<int>(e1 - e) : kBatchB;
            int64_t js[kBatchB];
            XT ws[kBatchB];
#pragma unroll
            for (int t = 0; t < kBatchB; ++t) {
                js[t] = t < cnt ? __ldg(col + e + t) : 0;
                ws[t] = t < cnt ? static_cast<XT>(__ldg(val + e + t)) : XT(0);
            }
            XT xv[kBatchB][V];
#pragma unroll
            for (int t = 0; t < kBatchB; ++t)
                if (t < cnt) ld<V>(x + js[t] * R + ch * V, xv[t]);
#pragma unroll
            for (int t = 0; t < kBatchB; ++t)
                if (t < cnt) {
#pragma unroll
                    for (int q = 0; q < V; ++q) u[q] += ws[t] * xv[t][q];
                }
        }
        XT xi[V];
        float wi[V];
        ld<V>(x + i * R + ch * V, xi);
        const XT hi = h ? h[i] : XT(0);
#pragma unroll
        for (int q = 0; q < V; ++q) {
            if constexpr (sizeof(XT) == 4) {
                acc32.add(xi[q], -0.5f * u[q]);
                if (h) acc32.add(xi[q], -hi);
            } else {
                acc += -0.5 * xi[q] * u[q] - hi * xi[q];
            }
            const float gi = static_cast<float>(-(u[q] + hi) * invR);
            nz += xi[q] == XT(0);
            wi[q] = dcbrt_weight(gi, static_cast<float>(xi[q]));
        }
        st<V>(w + i * R + ch * V, wi);
    }
    if constexpr (sizeof(XT) == 4) acc = acc32.value();
    const double b = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = b;
    unsigned tot = nz;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd(zeros, static_cast<unsigned long long>(tot));
}

// One adjoint step k: from w^k (gathered at the neighbours) and x^k (the row's own),
//   dL/dalpha_k partial += w^k_i x^k_i,  g^k_i = (sum_j J_ij w^k_j + alpha_k w^k_i) / beta,
// then the next step's w^(k-1)_i = g^k_i / (3 (x^k_i)^2) (0 where x^k_i = 0, counted),
// or g^0 itself when k = 0 (final). One gather per neighbour: w^k was formed once per
// row by the step before. Iterates of type XT are rounded to FP32 for this arithmetic.
template <typename XT, typename VT, int V, typename IT>
__global__ void __launch_bounds__(kBThreads, kAdjointBlocksPerSm)
adjoint_step_kernel(const float *__restrict__ w_in, const XT *__restrict__ x_cur, float *__restrict__ w_out,
                    const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                    const VT *__restrict__ val, IT n, int R, float alpha_k, float inv_beta, int final_step,
                    double *__restrict__ part, unsigned long long *__restrict__ zeros) {
    const int C = R / V;
    // sum of w x: compensated FP32 for FP32 iterates, FP64 for FP64 iterates
    double ga = 0.0;
    DotSum32 ga32;
    unsigned nz = 0;
    const int rows_per_block = kBThreads / C;
    const int ch = threadIdx.x % C;
    const int rl = threadIdx.x / C;
    const IT S = static_cast<IT>(gridDim.x) * rows_per_block;
    // threads past the block's last full row take no rows
    IT i = rl < rows_per_block ? static_cast<IT>(blockIdx.x) * rows_per_block + rl : n;
    IT e0, e1, f0, f1;  // entry ranges of rows i and i + S
    int32_t js[kBatchB];
    float ws[kBatchB];
    pipe_row_range(row_ptr, i, n, e0, e1);
    pipe_row_range(row_ptr, i + S, n, f0, f1);
    pipe_first_batch<kBatchB>(col, val, e0, e1, js, ws);
    for (; i < n; i += S) {
        const int cnt = e1 - e0 < kBatchB ? static_cast<int>(e1 - e0) : kBatchB;
        float wj[kBatchB][V];
#pragma unroll
        for (int t = 0; t < kBatchB; ++t)
            if (t < cnt) ld<V>(w_in + static_cast<int64_t>(js[t]) * R + ch * V, wj[t]);
        float wi[V];
        XT xc[V];
        ld<V>(w_in + static_cast<int64_t>(i) * R + ch * V, wi);
        ld<V>(x_cur + static_cast<int64_t>(i) * R + ch * V, xc);
        // the next row's first batch and the range of the row after it
        int32_t js2[kBatchB];
        float ws2[kBatchB];
        pipe_first_batch<kBatchB>(col, val, f0, f1, js2, ws2);
        IT g0, g1;
        pipe_row_range(row_ptr, i + 2 * S, n, g0, g1);
        float acc[V];
#pragma unroll
        for (int q = 0; q < V; ++q) acc[q] = 0.f;
#pragma unroll
        for (int t = 0; t < kBatchB; ++t)
            if (t < cnt) {
#pragma unroll
                for (int q = 0; q < V; ++q) acc[q] += ws[t] * wj[t][q];
            }
        // entries past the first batch, in entry order
#pragma unroll 4
        for (IT e = e0 + kBatchB; e < e1; ++e) {
            const int64_t j = __ldg(col + e);
            const float wv = static_cast<float>(__ldg(val + e));
            float wr[V];
            ld<V>(w_in + j * R + ch * V, wr);
#pragma unroll
            for (int q = 0; q < V; ++q) acc[q] += wv * wr[q];
        }
        float out[V];
        if constexpr (sizeof(XT) == 4) {  // the row's V products in FP32, then the compensated sum
            float dot = wi[0] * xc[0];
#pragma unroll
            for (int q = 1; q < V; ++q) dot = fmaf(wi[q], xc[q], dot);
            ga32.add(dot);
        }
#pragma unroll
        for (int q = 0; q < V; ++q) {
            if constexpr (sizeof(XT) == 8) ga += static_cast<double>(wi[q]) * xc[q];
            const float g = (acc[q] + alpha_k * wi[q]) * inv_beta;
            if (final_step) {
                out[q] = g;
            } else {
                nz += xc[q] == XT(0);
                out[q] = dcbrt_weight(g, static_cast<float>(xc[q]));
            }
        }
        st<V>(w_out + static_cast<int64_t>(i) * R + ch * V, out);
        e0 = f0;
        e1 = f1;
        f0 = g0;
        f1 = g1;
#pragma unroll
        for (int t = 0; t < kBatchB; ++t) {
            js[t] = js2[t];
            ws[t] = ws2[t];
        }
    }
    if constexpr (sizeof(XT) == 4) ga = ga32.value();
    const double b = block_sum(ga);
    if (threadIdx.x == 0) part[blockIdx.x] = b;
    unsigned tot = nz;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd(zeros, static_cast<unsigned long long>(tot));
}

// grad_alpha[k] = sum_b part[k][b] / beta; loss = sum_b lpart[b] / R. One warp per
// output (warp k < iters: grad_alpha[k]; warp iters: the loss): lane l sums the
// blocks b = l, l + 32, ... in order, then a fixed shuffle tree (run-to-run identical).
__global__ void adjoint_finish(const double *__restrict__ part, int iters, int blocks, double beta,
                               const double *__restrict__ lpart, int lblocks, int R,
                               double *__restrict__ grad_alpha, double *__restrict__ loss) {
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k > iters) return;  // whole warps only: blockDim.x is a multiple of 32
    const double *src = k < iters ? part + static_cast<int64_t>(k) * blocks : lpart;
    const int m = k < iters ? blocks : lblocks;
    double s = 0.0;
    for (int b = lane; b < m; b += 32) s += src[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        if (k < iters) grad_alpha[k] = s / beta;
        else *loss = s / R;
    }
}

__global__ void widen_kernel(const float *__restrict__ a, double *__restrict__ b, int64_t count) {
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < count;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x)
        b[t] = a[t];
}

template <typename XT, typename VT, int V>
void launch_loss(const ising_context *c, const XT *x, float *w, int R, int grid, double *part,
                 unsigned long long *zeros, cudaStream_t st) {
    const XT *h = nullptr;
    if constexpr (sizeof(XT) == 8) h = c->h_f64; else h = c->h_f32;
    loss_w_kernel<XT, VT, V><<<grid, kBThreads, 0, st>>>(x, w, c->row_ptr, c->col, static_cast<const VT *>(c->val),
                                                         h, c->n, R, part, zeros);
}

template <typename XT, typename VT, int V>
void launch_adj(const ising_context *c, const float *wi, const XT *xc, float *wo, int R, float a, float ib,
                int final_step, int grid, double *part, unsigned long long *zeros, cudaStream_t st) {
    if (c->n < (int64_t(1) << 30) && c->nnz < (int64_t(1) << 30))  // 32-bit rows and entry offsets
        adjoint_step_kernel<XT, VT, V, int><<<grid, kBThreads, 0, st>>>(
            wi, xc, wo, c->row_ptr, c->col, static_cast<const VT *>(c->val), static_cast<int>(c->n), R, a, ib,
            final_step, part, zeros);
    else
        adjoint_step_kernel<XT, VT, V, int64_t><<<grid, kBThreads, 0, st>>>(
            wi, xc, wo, c->row_ptr, c->col, static_cast<const VT *>(c->val), c->n, R, a, ib, final_step, part,
            zeros);
}

template <typename XT, typename VT>
ising_status_t loss_v(const ising_context *c, const XT *x, float *w, int R, int V, int grid, double *part,
                      unsigned long long *zeros, cudaStream_t st) {
    if (V == 4) launch_loss<XT, VT, 4>(c, x, w, R, grid, part, zeros, st);
    else if (V == 2) launch_loss<XT, VT, 2>(c, x, w, R, grid, part, zeros, st);
    else launch_loss<XT, VT, 1>(c, x, w, R, grid, part, zeros, st);
    DOCH_CUDA(cudaGetLastError());
    return ISING_OK;
}

template <typename XT, typename VT>
ising_status_t adj_v(const ising_context *c, const float *wi, const XT *xc, float *wo, int R, int V, float a,
                     float ib, int final_step, int grid, double *part, unsigned long long *zeros, cudaStream_t st) {
    if (V == 4) launch_adj<XT, VT, 4>(c, wi, xc, wo, R, a, ib, final_step, grid, part, zeros, st);
    else if (V == 2) launch_adj<XT, VT, 2>(c, wi, xc, wo, R, a, ib, final_step, grid, part, zeros, st);
    else launch_adj<XT, VT, 1>(c, wi, xc, wo, R, a, ib, final_step, grid, part, zeros, st);
    DOCH_CUDA(cudaGetLastError());
    return ISING_OK;
}

template <typename XT>
ising_status_t loss_t(const ising_context *c, const XT *x, float *w, int R, int V, int grid, double *part,
                      unsigned long long *zeros, cudaStream_t st) {
    switch (c->jtype) {
        case ISING_I8: return loss_v<XT, int8_t>(c, x, w, R, V, grid, part, zeros, st);
        case ISING_I32: return loss_v<XT, int32_t>(c, x, w, R, V, grid, part, zeros, st);
        case ISING_F32: return loss_v<XT, float>(c, x, w, R, V, grid, part, zeros, st);
        case ISING_F64: return loss_v<XT, double>(c, x, w, R, V, grid, part, zeros, st);
        default: return fail(ISING_ERR_UNSUPPORTED, "backward: coupling type");
    }
}

template <typename XT>
ising_status_t adj_t(const ising_context *c, const float *wi, const XT *xc, float *wo, int R, int V,
                     float alpha_k, float inv_beta, int final_step, int grid, double *part,
                     unsigned long long *zeros, cudaStream_t st) {
    switch (c->jtype) {
        case ISING_I8: return adj_v<XT, int8_t>(c, wi, xc, wo, R, V, alpha_k, inv_beta, final_step, grid, part, zeros, st);
        case ISING_I32: return adj_v<XT, int32_t>(c, wi, xc, wo, R, V, alpha_k, inv_beta, final_step, grid, part, zeros, st);
        case ISING_F32: return adj_v<XT, float>(c, wi, xc, wo, R, V, alpha_k, inv_beta, final_step, grid, part, zeros, st);
        case ISING_F64: return adj_v<XT, double>(c, wi, xc, wo, R, V, alpha_k, inv_beta, final_step, grid, part, zeros, st);
        default: return fail(ISING_ERR_UNSUPPORTED, "backward: coupling type");
    }
}

}  // namespace

ising_status_t csr_loss_w(const ising_context *c, const void *x, int xtype, float *w, int R, int V, int grid,
                          double *part, unsigned long long *zeros, cudaStream_t st) {
    if (xtype == ISING_F64) return loss_t<double>(c, static_cast<const double *>(x), w, R, V, grid, part, zeros, st);
    return loss_t<float>(c, static_cast<const float *>(x), w, R, V, grid, part, zeros, st);
}

ising_status_t csr_adjoint_step(const ising_context *c, const float *w_in, const void *x_cur, int xtype,
                                float *w_out, int R, int V, float alpha_k, float inv_beta, bool final_step,
                                int grid, double *part, unsigned long long *zeros, cudaStream_t st) {
    if (xtype == ISING_F64)
        return adj_t<double>(c, w_in, static_cast<const double *>(x_cur), w_out, R, V, alpha_k, inv_beta,
                             final_step ? 1 : 0, grid, part, zeros, st);
    return adj_t<float>(c, w_in, static_cast<const float *>(x_cur), w_out, R, V, alpha_k, inv_beta,
                        final_step ? 1 : 0, grid, part, zeros, st);
}

ising_status_t widen_f32_to_f64(const float *a, double *b, int64_t count, int num_sms, cudaStream_t st) {
    int64_t blocks = (count + 255) / 256;
    if (blocks > 8LL * num_sms) blocks = 8LL * num_sms;
    if (blocks < 1) blocks = 1;
    widen_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(a, b, count);
    DOCH_CUDA(cudaGetLastError());
    return ISING_OK;
}

ising_status_t adjoint_finish_launch(const double *part, int iters, int blocks, double beta,
                                     const double *lpart, int lblocks, int R, double *grad_alpha,
                                     double *loss, cudaStream_t st) {
    const int threads = 128;                                  // 4 warps per block
    const int warps = iters + 1;                              // one per gradient entry, one for the loss
    adjoint_finish<<<(warps + 3) / 4, threads, 0, st>>>(part, iters, blocks, beta, lpart, lblocks, R,
                                                       grad_alpha, loss);
    DOCH_CUDA(cudaGetLastError());
    return ISING_OK;
}

}  // namespace doch
