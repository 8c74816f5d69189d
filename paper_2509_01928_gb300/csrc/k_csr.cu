// DOCH step for couplings in CSR form, Eq. FPE with the field inside g:
//   x_out[i][r] = cbrt( ( sum_e val[e] x_in[col[e]][r] + alpha_b x_in[i][r] + h_i ) / beta_b )
// for the instance b that owns row i (batched instances are concatenated).
//
// csr_step: one launch per step. A thread owns one row and a vector chunk of
// V replicas (V = 4/2/1 floats or 2/1 doubles), so the threads of a row read
// consecutive replicas of each neighbour x[j][*] (coalesced) and share the
// row's col/val entries. FP32 steps take the cube root as the prescaled
// power-of-two form of cbrt.cuh (the lattice, batched and dense kernels use the
// same form), FP64 steps cbrt.
//
// csr_step_pipe: the same step for short rows (at most kPipeAvgDeg entries per
// row on average, one instance, no monitor). The grid is one resident wave and a
// thread's loads are pipelined across its rows (csr_pipe.cuh); the sums are the
// ones csr_step forms, in the same order.
//
// csr_fused: the whole iteration in one launch for instances that fit in
// shared memory. One CTA per (instance, replica) keeps that replica's
// iterate in two shared-memory buffers and separates the steps with
// __syncthreads(); the CSR arrays stream through L1/L2.
#include <algorithm>

#include "cbrt.cuh"
#include "csr_pipe.cuh"
#include "hamsum.cuh"
#include "internal.cuh"

namespace doch {
namespace {

template <typename T>
__device__ __forceinline__ T dcbrt(T z) {
    if constexpr (sizeof(T) == 4) return cbrtf(z);
    else return cbrt(z);
}

// The update of the step kernels, x = cbrt(z / beta) for z = (J x + alpha x + h)_i:
// FP32 through the prescaled power-of-two cube root (cbrt.cuh; zs = 2^(3k) / beta,
// xsc = 2^-k per instance), FP64 through cbrt(z / beta).
template <typename T>
__device__ __forceinline__ T step_update(T z, T beta, float zs, float xsc) {
    if constexpr (sizeof(T) == 4) return cbrt_pow2(z * zs) * xsc;
    else return cbrt(z / beta);
}

__device__ __forceinline__ int find_inst(const int64_t *__restrict__ off, int n_inst, int64_t i) {
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename T, int V> struct VecOf;
template <> struct VecOf<float, 1> { using type = float; };
template <> struct VecOf<float, 2> { using type = float2; };
template <> struct VecOf<float, 4> { using type = float4; };
template <> struct VecOf<double, 1> { using type = double; };
template <> struct VecOf<double, 2> { using type = double2; };

template <typename T, int V>
__device__ __forceinline__ void ldv(const T *p, T (&v)[V]) {
    using VT = typename VecOf<T, V>::type;
    const VT w = __ldg(reinterpret_cast<const VT *>(p));
    const T *q = reinterpret_cast<const T *>(&w);
#pragma unroll
    for (int k = 0; k < V; ++k) v[k] = q[k];
}

template <typename T, int V>
__device__ __forceinline__ void stv(T *p, const T (&v)[V]) {
    using VT = typename VecOf<T, V>::type;
    VT w;
    T *q = reinterpret_cast<T *>(&w);
#pragma unroll
    for (int k = 0; k < V; ++k) q[k] = v[k];
    *reinterpret_cast<VT *>(p) = w;
}

constexpr int kCsrBatch = 8;  // entries whose loads are issued together

// H monitor fused into the step (TRACE, one instance): the step already holds
// u = J x^(k) and x^(k), so it also sums the terms of H(x^(k)) (Eq. Hamilton,
// -h^T x for a field): x^4, x^2, x u, h x per replica. FP64 iterates sum in
// FP64; FP32 iterates form the terms in FP32 and sum them per thread with a
// compensated (Kahan) FP32 sum. Each block writes FP64 partials
// hpart[block][R][4], summed over threads in a fixed order.
template <typename XT, typename VT, int V, bool TRACE>
__global__ void __launch_bounds__(256)
csr_step_kernel(const XT *__restrict__ xi, XT *__restrict__ xo, const int64_t *__restrict__ row_ptr,
                const int32_t *__restrict__ col, const VT *__restrict__ val, const XT *__restrict__ h,
                const int64_t *__restrict__ inst_off, int n_inst, int64_t n, int R,
                const XT *__restrict__ alpha_tab, int alpha_len, int k,
                const XT *__restrict__ beta_tab, const float *__restrict__ zs_tab,
                const float *__restrict__ xs_tab, double *__restrict__ hpart) {
    const int C = R / V;
    const int ak = alpha_len == 1 ? 0 : k;
    // each thread keeps one replica chunk and strides over rows: no division in the loop
    const int rows_per_block = blockDim.x / C;
    const int ch = threadIdx.x % C;
    const int rl = threadIdx.x / C;
    HamSum<XT> hs[TRACE ? V : 1][4];
    // the cube root's prescale (FP32): one instance's values are loaded once per thread -- two
    // loads per row cost the S5 workload 2.5 % -- batched instances look theirs up per row
    float zs0 = 1.f, xsc0 = 1.f;
    if constexpr (sizeof(XT) == 4) {
        zs0 = __ldg(zs_tab);
        xsc0 = __ldg(xs_tab);
    }
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * rows_per_block + rl; rl < rows_per_block && i < n;
         i += static_cast<int64_t>(gridDim.x) * rows_per_block) {
        const int b = n_inst > 1 ? find_inst(inst_off, n_inst, i) : 0;
        const XT a = alpha_tab[static_cast<int64_t>(b) * alpha_len + ak];
        const XT bb = beta_tab[b];
        float zs = zs0, xsc = xsc0;
        if (sizeof(XT) == 4 && n_inst > 1) {
            zs = __ldg(zs_tab + b);
            xsc = __ldg(xs_tab + b);
        }
        XT acc[V];
#pragma unroll
        for (int q = 0; q < V; ++q) acc[q] = XT(0);
        const int64_t e1 = __ldg(row_ptr + i + 1);
        int64_t e = __ldg(row_ptr + i);
        // entries in batches of kCsrBatch: the index/value loads first, then the gathers, then
        // the products in entry order (the same sums as one entry at a time)
        for (; e + kCsrBatch <= e1; e += kCsrBatch) {
            int32_t js[kCsrBatch];
            XT ws[kCsrBatch];
#pragma unroll
            for (int t = 0; t < kCsrBatch; ++t) {
                js[t] = __ldg(col + e + t);
                ws[t] = static_cast<XT>(__ldg(val + e + t));
            }
            XT xv[kCsrBatch][V];
#pragma unroll
            for (int t = 0; t < kCsrBatch; ++t) ldv<XT, V>(xi + static_cast<int64_t>(js[t]) * R + ch * V, xv[t]);
#pragma unroll
            for (int t = 0; t < kCsrBatch; ++t)
#pragma unroll
                for (int q = 0; q < V; ++q) acc[q] += ws[t] * xv[t][q];
        }
        for (; e < e1; ++e) {
            const int64_t j = __ldg(col + e);
            const XT w = static_cast<XT>(__ldg(val + e));
            XT xv[V];
            ldv<XT, V>(xi + j * R + ch * V, xv);
#pragma unroll
            for (int q = 0; q < V; ++q) acc[q] += w * xv[q];
        }
        XT xs[V], out[V];
        ldv<XT, V>(xi + i * R + ch * V, xs);
        const XT hi = h ? h[i] : XT(0);
#pragma unroll
        for (int q = 0; q < V; ++q) out[q] = step_update(acc[q] + a * xs[q] + hi, bb, zs, xsc);
        stv<XT, V>(xo + i * R + ch * V, out);
        if constexpr (TRACE) {
#pragma unroll
            for (int q = 0; q < V; ++q) {
                const XT x2 = xs[q] * xs[q];
                hs[q][0].add(x2 * x2);
                hs[q][1].add(x2);
                hs[q][2].add(xs[q] * acc[q]);
                hs[q][3].add(hi * xs[q]);
            }
        }
    }
    if constexpr (TRACE) {
        // per replica: threads of the same chunk ch (rows rl = 0 .. rows_per_block-1) in row order
        __shared__ double red[256][4];
#pragma unroll
        for (int q = 0; q < V; ++q) {
#pragma unroll
            for (int m = 0; m < 4; ++m) red[threadIdx.x][m] = hs[q][m].value();
            __syncthreads();
            if (rl == 0) {
                double t[4] = {0.0, 0.0, 0.0, 0.0};
                for (int r2 = 0; r2 < rows_per_block; ++r2)
#pragma unroll
                    for (int m = 0; m < 4; ++m) t[m] += red[r2 * C + ch][m];
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    hpart[(static_cast<int64_t>(blockIdx.x) * R + ch * V + q) * 4 + m] = t[m];
            }
            __syncthreads();
        }
    }
}

constexpr int kPipeB = 4;  // entries of a row's first batch, loaded one row ahead

// Rows and entry offsets are 32-bit here (n, nnz < 2^30, checked by use_pipe).
template <typename XT>
constexpr int pipe_blocks_per_sm() { return sizeof(XT) == 4 ? kCsrPipeBlocksPerSm : kCsrPipeBlocksPerSm - 1; }

template <typename XT, typename VT, int V>
__global__ void __launch_bounds__(256, pipe_blocks_per_sm<XT>())
csr_step_pipe_kernel(const XT *__restrict__ xi, XT *__restrict__ xo, const int64_t *__restrict__ row_ptr,
                     const int32_t *__restrict__ col, const VT *__restrict__ val, const XT *__restrict__ h,
                     int n, int R, const XT *__restrict__ alpha_tab, int alpha_len, int k,
                     const XT *__restrict__ beta_tab, const float *__restrict__ zs_tab,
                     const float *__restrict__ xs_tab) {
    const int C = R / V;
    const XT a = alpha_tab[alpha_len == 1 ? 0 : k];
    const XT bb = beta_tab[0];
    float zs = 1.f, xsc = 1.f;
    if constexpr (sizeof(XT) == 4) {
        zs = zs_tab[0];
        xsc = xs_tab[0];
    }
    const int rows_per_block = blockDim.x / C;
    const int ch = threadIdx.x % C;
    const int rl = threadIdx.x / C;
    const int S = static_cast<int>(gridDim.x) * rows_per_block;
    int i = rl < rows_per_block ? static_cast<int>(blockIdx.x) * rows_per_block + rl : n;
    int e0, e1, f0, f1;  // entry ranges of rows i and i + S
    int32_t js[kPipeB];
    XT ws[kPipeB];
    pipe_row_range(row_ptr, i, n, e0, e1);
    pipe_row_range(row_ptr, i + S, n, f0, f1);
    pipe_first_batch<kPipeB>(col, val, e0, e1, js, ws);
    for (; i < n; i += S) {
        const int cnt = e1 - e0 < kPipeB ? static_cast<int>(e1 - e0) : kPipeB;
        XT xv[kPipeB][V];
#pragma unroll
        for (int t = 0; t < kPipeB; ++t)
            if (t < cnt) ldv<XT, V>(xi + static_cast<int64_t>(js[t]) * R + ch * V, xv[t]);
        XT xs[V];
        ldv<XT, V>(xi + static_cast<int64_t>(i) * R + ch * V, xs);
        const XT hi = h ? h[i] : XT(0);
        // the next row's first batch and the range of the row after it
        int32_t js2[kPipeB];
        XT ws2[kPipeB];
        pipe_first_batch<kPipeB>(col, val, f0, f1, js2, ws2);
        int g0, g1;
        pipe_row_range(row_ptr, i + 2 * S, n, g0, g1);
        XT acc[V];
#pragma unroll
        for (int q = 0; q < V; ++q) acc[q] = XT(0);
#pragma unroll
        for (int t = 0; t < kPipeB; ++t)
            if (t < cnt) {
#pragma unroll
                for (int q = 0; q < V; ++q) acc[q] += ws[t] * xv[t][q];
            }
        // entries past the first batch, in entry order
#pragma unroll 4
        for (int e = e0 + kPipeB; e < e1; ++e) {
            const int64_t j = __ldg(col + e);
            const XT w = static_cast<XT>(__ldg(val + e));
            XT xr[V];
            ldv<XT, V>(xi + j * R + ch * V, xr);
#pragma unroll
            for (int q = 0; q < V; ++q) acc[q] += w * xr[q];
        }
        XT out[V];
#pragma unroll
        for (int q = 0; q < V; ++q) out[q] = step_update(acc[q] + a * xs[q] + hi, bb, zs, xsc);
        stv<XT, V>(xo + static_cast<int64_t>(i) * R + ch * V, out);
        e0 = f0;
        e1 = f1;
        f0 = g0;
        f1 = g1;
#pragma unroll
        for (int t = 0; t < kPipeB; ++t) {
            js[t] = js2[t];
            ws[t] = ws2[t];
        }
    }
}

// One CTA per (instance b = blockIdx.y, replica r = blockIdx.x); shared
// memory holds two copies of that instance's iterate for replica r.
template <typename XT, typename VT>
__global__ void __launch_bounds__(1024)
csr_fused_kernel(XT *__restrict__ x, const int64_t *__restrict__ row_ptr,
                 const int32_t *__restrict__ col, const VT *__restrict__ val,
                 const XT *__restrict__ h, const int64_t *__restrict__ inst_off, int64_t n, int R,
                 const double *__restrict__ alpha_tab, int alpha_len,
                 const double *__restrict__ beta_tab, int iters) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    XT *buf = reinterpret_cast<XT *>(smem_raw);
    const int b = blockIdx.y, r = blockIdx.x;
    const int64_t lo = inst_off ? inst_off[b] : 0;
    const int64_t hi = inst_off ? inst_off[b + 1] : n;
    const int nb = static_cast<int>(hi - lo);
    XT *cur = buf, *nxt = buf + nb;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) cur[i] = x[(lo + i) * R + r];
    const XT bb = static_cast<XT>(beta_tab[b]);
    __syncthreads();
    for (int k = 0; k < iters; ++k) {
        const XT a = static_cast<XT>(alpha_tab[static_cast<int64_t>(b) * alpha_len +
                                               (alpha_len == 1 ? 0 : k)]);
        for (int i = threadIdx.x; i < nb; i += blockDim.x) {
            const int64_t row = lo + i;
            XT acc = XT(0);
            const int64_t e1 = __ldg(row_ptr + row + 1);
            for (int64_t e = __ldg(row_ptr + row); e < e1; ++e)
                acc += static_cast<XT>(__ldg(val + e)) * cur[__ldg(col + e) - lo];
            const XT hv = h ? h[row] : XT(0);
            nxt[i] = dcbrt((acc + a * cur[i] + hv) / bb);
        }
        __syncthreads();
        XT *t = cur; cur = nxt; nxt = t;
    }
    for (int i = threadIdx.x; i < nb; i += blockDim.x) x[(lo + i) * R + r] = cur[i];
}

// Small instances over a cluster of K CTAs per (instance b = blockIdx.y, replica r = blockIdx.x / K):
// every CTA keeps both copies of the pair's whole iterate, computes the rows of its share
// [q c, (q+1) c) (c = ceil(n_b / K), q its rank in the cluster) with the arithmetic of
// csr_fused_kernel, and stores each new value into the next copy of all K CTAs (distributed
// shared memory); a cluster barrier ends each step. The same iterates as one CTA per pair, with
// the FP64 arithmetic of a pair spread over K SMs.
__device__ __forceinline__ uint32_t cl_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cl_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cl_map(const void *p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                 : "=r"(r)
                 : "r"(static_cast<uint32_t>(__cvta_generic_to_shared(p))), "r"(rank));
    return r;
}
__device__ __forceinline__ void cl_store(uint32_t a, double v) {
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}
__device__ __forceinline__ void cl_store(uint32_t a, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}

template <typename XT, typename VT>
__global__ void __launch_bounds__(1024)
csr_fused_cluster(XT *__restrict__ x, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                  const VT *__restrict__ val, const XT *__restrict__ h, const int64_t *__restrict__ inst_off,
                  int64_t n, int R, const double *__restrict__ alpha_tab, int alpha_len,
                  const double *__restrict__ beta_tab, int iters, int K) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    XT *buf = reinterpret_cast<XT *>(smem_raw);
    const uint32_t q = cl_rank();
    const int b = blockIdx.y, r = blockIdx.x / K;
    const int64_t lo = inst_off ? inst_off[b] : 0;
    const int64_t hi = inst_off ? inst_off[b + 1] : n;
    const int nb = static_cast<int>(hi - lo);
    const int chunk = (nb + K - 1) / K;
    const int i0 = min(nb, static_cast<int>(q) * chunk), i1 = min(nb, i0 + chunk);
    XT *cur = buf, *nxt = buf + nb;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) cur[i] = x[(lo + i) * R + r];
    const XT bb = static_cast<XT>(beta_tab[b]);
    cl_sync();  // every CTA of the cluster runs, and has loaded, before the first remote store
    for (int k = 0; k < iters; ++k) {
        const XT a = static_cast<XT>(alpha_tab[static_cast<int64_t>(b) * alpha_len + (alpha_len == 1 ? 0 : k)]);
        for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            const int64_t row = lo + i;
            XT acc = XT(0);
            const int64_t e1 = __ldg(row_ptr + row + 1);
            for (int64_t e = __ldg(row_ptr + row); e < e1; ++e)
                acc += static_cast<XT>(__ldg(val + e)) * cur[__ldg(col + e) - lo];
            const XT hv = h ? h[row] : XT(0);
            const XT v = dcbrt((acc + a * cur[i] + hv) / bb);
            nxt[i] = v;
            for (int t = 0; t < K; ++t)
                if (t != static_cast<int>(q)) cl_store(cl_map(nxt + i, static_cast<uint32_t>(t)), v);
        }
        cl_sync();  // the new values of every share are in every CTA; the old copy is free
        XT *t = cur;
        cur = nxt;
        nxt = t;
    }
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) x[(lo + i) * R + r] = cur[i];
}

int step_blocks(const ising_context *c, int C) {
    const int rows_per_block = C <= 256 ? 256 / C : 1;
    int64_t blocks = (c->n + rows_per_block - 1) / rows_per_block;
    const int64_t cap = static_cast<int64_t>(c->num_sms) * 32;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return static_cast<int>(blocks);
}

// short rows: the pipelined kernel (one resident wave, 32-bit row and entry offsets) serves one
// instance without the monitor
bool use_pipe(const ising_context *c, int C, bool traced) {
    return !traced && c->n_inst == 1 && C <= 256 && c->nnz <= static_cast<int64_t>(kPipeAvgDeg) * c->n &&
           c->n < (int64_t(1) << 30) && c->nnz < (int64_t(1) << 30);
}

template <typename XT>
int pipe_blocks(const ising_context *c, int C) {
    const int rows_per_block = 256 / C;
    int64_t blocks = (c->n + rows_per_block - 1) / rows_per_block;
    const int64_t cap = static_cast<int64_t>(c->num_sms) * pipe_blocks_per_sm<XT>();
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return static_cast<int>(blocks);
}

// the update tables of a step: beta (FP64) or the cube root's prescale (FP32, per instance)
template <typename XT>
struct StepTabs {
    const XT *alpha;
    int alpha_len;
    const XT *beta;
    const float *zs;
    const float *xsc;
};

template <typename XT, typename VT, int V>
void launch_step(const ising_context *c, const XT *xi, XT *xo, int R, const XT *h, const StepTabs<XT> &t, int k,
                 double *hpart, cudaStream_t st) {
    const int C = R / V;
    if (use_pipe(c, C, hpart != nullptr)) {
        csr_step_pipe_kernel<XT, VT, V><<<static_cast<unsigned>(pipe_blocks<XT>(c, C)), 256, 0, st>>>(
            xi, xo, c->row_ptr, c->col, static_cast<const VT *>(c->val), h, static_cast<int>(c->n), R, t.alpha,
            t.alpha_len, k, t.beta, t.zs, t.xsc);
        return;
    }
    const int blocks = step_blocks(c, C);
    const int threads = C <= 256 ? 256 : ((C + 31) / 32) * 32;
    if (hpart)
        csr_step_kernel<XT, VT, V, true><<<static_cast<unsigned>(blocks), threads, 0, st>>>(
            xi, xo, c->row_ptr, c->col, static_cast<const VT *>(c->val), h, c->inst_off, c->n_inst,
            c->n, R, t.alpha, t.alpha_len, k, t.beta, t.zs, t.xsc, hpart);
    else
        csr_step_kernel<XT, VT, V, false><<<static_cast<unsigned>(blocks), threads, 0, st>>>(
            xi, xo, c->row_ptr, c->col, static_cast<const VT *>(c->val), h, c->inst_off, c->n_inst,
            c->n, R, t.alpha, t.alpha_len, k, t.beta, t.zs, t.xsc, nullptr);
}

template <typename XT, int V>
ising_status_t dispatch_val(const ising_context *c, const XT *xi, XT *xo, int R, const XT *h, const StepTabs<XT> &t,
                            int k, double *hpart, cudaStream_t st) {
    if (R / V > 1024) return fail(ISING_ERR_UNSUPPORTED, "CSR step: R / vector width must be <= 1024");
    if (hpart && R / V > 256) return ISING_ERR_UNSUPPORTED;  // the fused monitor needs one row per 256 threads
    switch (c->jtype) {
        case ISING_I8: launch_step<XT, int8_t, V>(c, xi, xo, R, h, t, k, hpart, st); break;
        case ISING_I32: launch_step<XT, int32_t, V>(c, xi, xo, R, h, t, k, hpart, st); break;
        case ISING_F32: launch_step<XT, float, V>(c, xi, xo, R, h, t, k, hpart, st); break;
        case ISING_F64: launch_step<XT, double, V>(c, xi, xo, R, h, t, k, hpart, st); break;
        default: return fail(ISING_ERR_UNSUPPORTED, "CSR value type not supported on the device");
    }
    DOCH_CUDA(cudaGetLastError());
    return ISING_OK;
}

// the cluster size for the fused kernel: the largest K in {16, 8, 4, 2} (16 is a non-portable size)
// that leaves each CTA at least 32 rows and keeps all pairs' clusters within the SMs; 1 when none does
int fused_cluster_k(const ising_context *c, int R, int kmax) {
    for (int K = kmax; K >= 2; K >>= 1)
        if (static_cast<int64_t>(c->n_inst) * R * K <= c->num_sms && c->max_inst_n >= 32LL * K) return K;
    return 1;
}

template <typename XT, typename VT>
ising_status_t launch_fused_cluster(const ising_context *c, XT *x, int R, const XT *h, const ParamTabs &p,
                                    int iters, int K, cudaStream_t st) {
    const size_t smem = 2 * static_cast<size_t>(c->max_inst_n) * sizeof(XT);
    auto kern = csr_fused_cluster<XT, VT>;
    DOCH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    if (K > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return ISING_ERR_UNSUPPORTED;
    }
    const int64_t chunk = (c->max_inst_n + K - 1) / K;
    int threads = static_cast<int>(std::min<int64_t>(1024, (chunk + 31) / 32 * 32));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = static_cast<unsigned>(K);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(static_cast<unsigned>(R * K), static_cast<unsigned>(c->n_inst));
    cfg.blockDim = dim3(static_cast<unsigned>(threads));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess || nclusters < 1) {
        cudaGetLastError();
        return ISING_ERR_UNSUPPORTED;
    }
    DOCH_CUDA(cudaLaunchKernelEx(&cfg, kern, x, static_cast<const int64_t *>(c->row_ptr),
                                 static_cast<const int32_t *>(c->col), static_cast<const VT *>(c->val), h,
                                 static_cast<const int64_t *>(c->n_inst > 1 ? c->inst_off : nullptr), c->n, R,
                                 p.alpha_d, p.alpha_len, p.beta_d, iters, K));
    return ISING_OK;
}

template <typename XT, typename VT>
ising_status_t launch_fused(const ising_context *c, XT *x, int R, const XT *h,
                            const ParamTabs &p, int iters, cudaStream_t st) {
    for (int kmax = 16; kmax >= 2; kmax >>= 1) {
        const int K = fused_cluster_k(c, R, kmax);
        if (K < 2) break;
        const ising_status_t s = launch_fused_cluster<XT, VT>(c, x, R, h, p, iters, K, st);
        if (s != ISING_ERR_UNSUPPORTED) return s;
        kmax = K;  // this size is not available: try the next smaller one
    }
    const size_t smem = 2 * static_cast<size_t>(c->max_inst_n) * sizeof(XT);
    auto kern = csr_fused_kernel<XT, VT>;
    DOCH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(smem)));
    int threads = 1024;
    if (c->max_inst_n < 1024) threads = static_cast<int>(((c->max_inst_n + 31) / 32) * 32);
    if (threads < 32) threads = 32;
    dim3 grid(static_cast<unsigned>(R), static_cast<unsigned>(c->n_inst));
    kern<<<grid, threads, smem, st>>>(x, c->row_ptr, c->col, static_cast<const VT *>(c->val), h,
                                      c->n_inst > 1 ? c->inst_off : nullptr, c->n, R, p.alpha_d,
                                      p.alpha_len, p.beta_d, iters);
    DOCH_CUDA(cudaGetLastError());
    return ISING_OK;
}

template <typename XT>
ising_status_t fused_dispatch(const ising_context *c, XT *x, int R, const XT *h,
                              const ParamTabs &p, int iters, cudaStream_t st) {
    switch (c->jtype) {
        case ISING_I8: return launch_fused<XT, int8_t>(c, x, R, h, p, iters, st);
        case ISING_I32: return launch_fused<XT, int32_t>(c, x, R, h, p, iters, st);
        case ISING_F32: return launch_fused<XT, float>(c, x, R, h, p, iters, st);
        case ISING_F64: return launch_fused<XT, double>(c, x, R, h, p, iters, st);
        default: return fail(ISING_ERR_UNSUPPORTED, "CSR value type not supported on the device");
    }
}

}  // namespace

size_t csr_fused_max_spins(int xtype) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return 0;
    return static_cast<size_t>(optin) / (2 * (xtype == ISING_F64 ? 8 : 4));
}

static ising_status_t csr_step_impl(const ising_context *c, const void *xi, void *xo, int xtype, int R,
                                    const ParamTabs &p, int k, double *hpart, int *blocks, cudaStream_t st) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(xi) | reinterpret_cast<uintptr_t>(xo);
    if (xtype == ISING_F32) {
        const float *x_in = static_cast<const float *>(xi);
        float *x_out = static_cast<float *>(xo);
        const StepTabs<float> t{p.alpha_f, p.alpha_len, p.inv_beta_f, p.zscale_f, p.xscale_f};
        if (R % 4 == 0 && a % 16 == 0) {
            *blocks = step_blocks(c, R / 4);
            return dispatch_val<float, 4>(c, x_in, x_out, R, c->h_f32, t, k, hpart, st);
        }
        if (R % 2 == 0 && a % 8 == 0) {
            *blocks = step_blocks(c, R / 2);
            return dispatch_val<float, 2>(c, x_in, x_out, R, c->h_f32, t, k, hpart, st);
        }
        *blocks = step_blocks(c, R);
        return dispatch_val<float, 1>(c, x_in, x_out, R, c->h_f32, t, k, hpart, st);
    }
    if (xtype == ISING_F64) {
        const double *x_in = static_cast<const double *>(xi);
        double *x_out = static_cast<double *>(xo);
        const StepTabs<double> t{p.alpha_d, p.alpha_len, p.beta_d, nullptr, nullptr};
        if (R % 2 == 0 && a % 16 == 0) {
            *blocks = step_blocks(c, R / 2);
            return dispatch_val<double, 2>(c, x_in, x_out, R, c->h_f64, t, k, hpart, st);
        }
        *blocks = step_blocks(c, R);
        return dispatch_val<double, 1>(c, x_in, x_out, R, c->h_f64, t, k, hpart, st);
    }
    return fail(ISING_ERR_UNSUPPORTED, "CSR iterate type must be F32 or F64");
}

ising_status_t csr_step(const ising_context *c, const void *xi, void *xo, int xtype, int R,
                        const ParamTabs &p, int k, cudaStream_t st) {
    int blocks = 0;
    return csr_step_impl(c, xi, xo, xtype, R, p, k, nullptr, &blocks, st);
}

ising_status_t csr_step_traced(ising_context *c, const void *xi, void *xo, int xtype, int R, const ParamTabs &p,
                               int k, double alpha_k, double beta, double *H_out, cudaStream_t st) {
    if (c->n_inst != 1) return ISING_ERR_UNSUPPORTED;
    const size_t max_blocks = static_cast<size_t>(c->num_sms) * 32;  // the cap of step_blocks
    DOCH_CHECK(c->partials.ensure(sizeof(double) * 4 * static_cast<size_t>(R) * max_blocks));
    int blocks = 0;
    const ising_status_t s = csr_step_impl(c, xi, xo, xtype, R, p, k, c->partials.as<double>(), &blocks, st);
    if (s != ISING_OK) return s;
    return ham_fused_finish_launch(c->partials.as<double>(), blocks, R, alpha_k, beta, H_out, st);
}

ising_status_t csr_fused(const ising_context *c, void *x, int xtype, int R, const ParamTabs &p,
                         int iters, cudaStream_t st) {
    if (static_cast<size_t>(c->max_inst_n) > csr_fused_max_spins(xtype))
        return ISING_ERR_UNSUPPORTED;
    if (xtype == ISING_F64)
        return fused_dispatch<double>(c, static_cast<double *>(x), R, c->h_f64, p, iters, st);
    if (xtype == ISING_F32)
        return fused_dispatch<float>(c, static_cast<float *>(x), R, c->h_f32, p, iters, st);
    return ISING_ERR_UNSUPPORTED;
}

}  // namespace doch
