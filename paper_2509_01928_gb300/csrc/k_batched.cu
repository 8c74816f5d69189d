// Many independent CSR instances of uneven size in one persistent launch.
//
// Each instance b owns rows [off[b], off[b+1]) of a concatenated CSR matrix
// and runs `iters` DOCH steps (Eq. FPE with the field in g) on its R
// replicas with its own alpha_b (or schedule) and beta_b. A CTA takes a whole
// instance from an atomic work queue -- instances are queued longest first
// (work ~ rows x (entries per row + 1)), which bounds the makespan by about
// max(total / CTAs, largest instance) -- and runs all of its steps, separated
// by __syncthreads(): no CTA ever waits for another. Threads own (row, chunk
// of V replicas) items, so each CSR entry is read once per V replicas and
// each neighbour gather is a V-wide vector. The iterate lives in two global
// buffers (L2-resident per instance); loads of x use coherent global loads
// because the same launch writes it.
#include "internal.cuh"

namespace doch {
namespace {

constexpr int kBatch = 8;  // neighbours whose loads are issued together

template <int V> struct FV;
template <> struct FV<1> { using type = float; };
template <> struct FV<2> { using type = float2; };
template <> struct FV<4> { using type = float4; };

template <int V>
__device__ __forceinline__ void ldx(const float *p, float (&v)[V]) {
    using T = typename FV<V>::type;
    const T w = *reinterpret_cast<const T *>(p);  // coherent: x is written in this launch
    const float *q = reinterpret_cast<const float *>(&w);
#pragma unroll
    for (int k = 0; k < V; ++k) v[k] = q[k];
}

template <int V>
__device__ __forceinline__ void stx(float *p, const float (&v)[V]) {
    using T = typename FV<V>::type;
    T w;
    float *q = reinterpret_cast<float *>(&w);
#pragma unroll
    for (int k = 0; k < V; ++k) q[k] = v[k];
    *reinterpret_cast<T *>(p) = w;
}

template <typename VT, int V>
__global__ void batched_persistent(float *xa, float *xb,
                                   const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                   const VT *__restrict__ val, const float *__restrict__ h,
                                   const int64_t *__restrict__ off, const int32_t *__restrict__ order,
                                   int n_inst, int R, const float *__restrict__ alpha_tab, int alpha_len,
                                   const float *__restrict__ inv_beta_tab, int iters, int *__restrict__ queue) {
    __shared__ int next;
    const int C = R / V;
    // each thread keeps one replica chunk and strides over rows: no division in the loop
    const int rows_step = blockDim.x / C;
    const int ch = threadIdx.x % C;
    const int row0 = threadIdx.x / C;
    const bool active = row0 < rows_step;
    while (true) {
        if (threadIdx.x == 0) next = atomicAdd(queue, 1);
        __syncthreads();
        const int w = next;
        __syncthreads();
        if (w >= n_inst) break;
        const int b = __ldg(order + w);
        const int64_t lo = __ldg(off + b), hi = __ldg(off + b + 1);
        const float ib = __ldg(inv_beta_tab + b);
        for (int k = 0; k < iters; ++k) {
            const float *xi = (k & 1) ? xb : xa;
            float *xo = (k & 1) ? xa : xb;
            const float a = __ldg(alpha_tab + static_cast<int64_t>(b) * alpha_len + (alpha_len == 1 ? 0 : k));
            for (int64_t i = lo + row0; i < hi && active; i += rows_step) {
                float acc[V];
#pragma unroll
                for (int q = 0; q < V; ++q) acc[q] = 0.f;
                const int64_t e1 = __ldg(row_ptr + i + 1);
                // neighbours in batches of kBatch: all index/weight loads first, then all
                // gathers, then the sums, so one batch costs two memory latencies
                for (int64_t e0 = __ldg(row_ptr + i); e0 < e1; e0 += kBatch) {
                    const int cnt = static_cast<int>(e1 - e0 < kBatch ? e1 - e0 : kBatch);
                    int js[kBatch];
                    float ws[kBatch];
#pragma unroll
                    for (int q = 0; q < kBatch; ++q) {
                        js[q] = q < cnt ? __ldg(col + e0 + q) : 0;
                        ws[q] = q < cnt ? static_cast<float>(__ldg(val + e0 + q)) : 0.f;
                    }
                    float xv[kBatch][V];
#pragma unroll
                    for (int q = 0; q < kBatch; ++q)
                        if (q < cnt) ldx<V>(xi + static_cast<int64_t>(js[q]) * R + ch * V, xv[q]);
#pragma unroll
                    for (int q = 0; q < kBatch; ++q)
                        if (q < cnt) {
#pragma unroll
                            for (int r = 0; r < V; ++r) acc[r] += ws[q] * xv[q][r];
                        }
                }
                float xs[V], out[V];
                ldx<V>(xi + i * R + ch * V, xs);
                const float hi_ = h ? __ldg(h + i) : 0.f;
#pragma unroll
                for (int q = 0; q < V; ++q) out[q] = cbrtf((acc[q] + a * xs[q] + hi_) * ib);
                stx<V>(xo + i * R + ch * V, out);
            }
            __syncthreads();
        }
    }
}

template <typename VT, int V>
ising_status_t launch_b(const ising_context *c, const BatchedConfig &cfg, float *xa, float *xb, int R,
                        const ParamTabs &p, int iters, cudaStream_t st) {
    if (R / V > cfg.threads) return ISING_ERR_UNSUPPORTED;  // a CTA must hold one row's chunks
    auto kern = batched_persistent<VT, V>;
    cudaFuncAttributes attr;
    DOCH_CUDA(cudaFuncGetAttributes(&attr, kern));
    if (cfg.threads > attr.maxThreadsPerBlock) return ISING_ERR_UNSUPPORTED;  // shape not launchable
    int occ = 0;
    DOCH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, cfg.threads, 0));
    if (occ < 1) occ = 1;
    if (occ > cfg.ctas_per_sm) occ = cfg.ctas_per_sm;
    int grid = c->num_sms * occ;
    if (grid > c->n_inst) grid = c->n_inst;
    DOCH_CUDA(cudaMemsetAsync(c->batch_queue, 0, sizeof(int), st));
    kern<<<grid, cfg.threads, 0, st>>>(xa, xb, c->row_ptr, c->col, static_cast<const VT *>(c->val), c->h_f32,
                                       c->inst_off, c->batch_order, c->n_inst, R, p.alpha_f, p.alpha_len,
                                       p.inv_beta_f, iters, c->batch_queue);
    DOCH_CUDA(cudaGetLastError());
    return ISING_OK;
}

template <int V>
ising_status_t dispatch_b(const ising_context *c, const BatchedConfig &cfg, float *xa, float *xb, int R,
                          const ParamTabs &p, int iters, cudaStream_t st) {
    switch (c->jtype) {
        case ISING_I8: return launch_b<int8_t, V>(c, cfg, xa, xb, R, p, iters, st);
        case ISING_I32: return launch_b<int32_t, V>(c, cfg, xa, xb, R, p, iters, st);
        case ISING_F32: return launch_b<float, V>(c, cfg, xa, xb, R, p, iters, st);
        case ISING_F64: return launch_b<double, V>(c, cfg, xa, xb, R, p, iters, st);
        default: return fail(ISING_ERR_UNSUPPORTED, "batched: coupling type");
    }
}

}  // namespace

ising_status_t batched_launch(const ising_context *c, const BatchedConfig &cfg, float *xa, float *xb, int R,
                              const ParamTabs &p, int iters, cudaStream_t st) {
    if (cfg.vec == 4 && R % 4 == 0) return dispatch_b<4>(c, cfg, xa, xb, R, p, iters, st);
    if (cfg.vec >= 2 && R % 2 == 0) return dispatch_b<2>(c, cfg, xa, xb, R, p, iters, st);
    return dispatch_b<1>(c, cfg, xa, xb, R, p, iters, st);
}

}  // namespace doch
