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
// because the same launch writes it. Gather indices are 32-bit element
// indices into the iterate viewed as [n][R/V] V-vectors (n R / V < 2^31 is
// checked on the host). The cube root is the prescaled base-2 form
// cbrt(z zscale_b) xscale_b with the instance's power-of-two prescale.
#include <algorithm>
#include <vector>

#include "cbrt.cuh"
#include "internal.cuh"

namespace doch {
namespace {

constexpr int kBatch = 8;  // neighbours whose loads are issued together
constexpr int kPairBatch = 4;  // ELL slot pairs whose loads are issued together (resident kernel)

template <int V> struct FV;
template <> struct FV<1> { using type = float; };
template <> struct FV<2> { using type = float2; };
template <> struct FV<4> { using type = float4; };

template <int V>
__device__ __forceinline__ void ldx(const typename FV<V>::type *p, float (&v)[V]) {
    const typename FV<V>::type w = *p;  // coherent: x is written in this launch
    const float *q = reinterpret_cast<const float *>(&w);
#pragma unroll
    for (int k = 0; k < V; ++k) v[k] = q[k];
}

template <int V>
__device__ __forceinline__ void stx(typename FV<V>::type *p, const float (&v)[V]) {
    typename FV<V>::type w;
    float *q = reinterpret_cast<float *>(&w);
#pragma unroll
    for (int k = 0; k < V; ++k) q[k] = v[k];
    *p = w;
}

template <typename VT, int V>
__global__ void batched_persistent(float *xa, float *xb,
                                   const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                   const VT *__restrict__ val, const float *__restrict__ h,
                                   const int64_t *__restrict__ off, const int32_t *__restrict__ order,
                                   int n_inst, int R, const float *__restrict__ alpha_tab, int alpha_len,
                                   const float *__restrict__ zscale_tab, const float *__restrict__ xscale_tab,
                                   int iters, int *__restrict__ queue) {
    using T = typename FV<V>::type;
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
        const float zs = __ldg(zscale_tab + b), xsc = __ldg(xscale_tab + b);
        for (int k = 0; k < iters; ++k) {
            const T *xi = reinterpret_cast<const T *>((k & 1) ? xb : xa) + ch;
            T *xo = reinterpret_cast<T *>((k & 1) ? xa : xb) + ch;
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
                        if (q < cnt) ldx<V>(xi + js[q] * C, xv[q]);
#pragma unroll
                    for (int q = 0; q < kBatch; ++q)
                        if (q < cnt) {
#pragma unroll
                            for (int r = 0; r < V; ++r) acc[r] += ws[q] * xv[q][r];
                        }
                }
                float xs[V], out[V];
                const int ic = static_cast<int>(i) * C;
                ldx<V>(xi + ic, xs);
                const float hi_ = h ? __ldg(h + i) : 0.f;
#pragma unroll
                for (int q = 0; q < V; ++q) out[q] = cbrt_pow2((acc[q] + a * xs[q] + hi_) * zs) * xsc;
                stx<V>(xo + ic, out);
            }
            __syncthreads();
        }
    }
}

template <typename VT, int V>
ising_status_t launch_b(const ising_context *c, const BatchedConfig &cfg, float *xa, float *xb, int R,
                        const ParamTabs &p, int iters, cudaStream_t st) {
    if (R / V > cfg.threads) return ISING_ERR_UNSUPPORTED;  // a CTA must hold one row's chunks
    if (c->n * (R / V) >= (int64_t(1) << 31))
        return fail(ISING_ERR_UNSUPPORTED, "batched: n R / V must be below 2^31 (32-bit gather indices)");
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
                                       p.zscale_f, p.xscale_f, iters, c->batch_queue);
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

// ---------------------------------------------------------------------------
// Shared-memory resident variant. A work item is (instance b, replicas g0 ..
// g0+G-1); one CTA runs all steps of an item with both Jacobi copies of that
// slice of the iterate in shared memory ([n_b][G] floats each), so every
// neighbour gather is a G-wide shared-memory load and only the couplings are
// re-read (from L2) each step, from the transposed ELL copy in slot pairs:
// pair p of rows i .. i+31 is 32 consecutive (column, column) and (weight,
// weight) pairs, one coalesced 4-byte and one 8-byte load per warp for two
// slots (the width D is even). G is chosen per instance, the largest power of
// two dividing R with 2 n_b G floats fitting the CTA's shared memory. Items
// are queued longest first; the iterate is updated in place in global memory
// at the end of the item (items own disjoint slices).

template <int G>
__device__ __forceinline__ void ldg_vec(const float *p, float (&v)[G]) {
    if constexpr (G >= 4) {
#pragma unroll
        for (int c = 0; c < G / 4; ++c) {
            const float4 t = reinterpret_cast<const float4 *>(p)[c];
            v[4 * c] = t.x; v[4 * c + 1] = t.y; v[4 * c + 2] = t.z; v[4 * c + 3] = t.w;
        }
    } else if constexpr (G == 2) {
        const float2 t = *reinterpret_cast<const float2 *>(p);
        v[0] = t.x; v[1] = t.y;
    } else {
        v[0] = *p;
    }
}

template <int G>
__device__ __forceinline__ void st_vec(float *p, const float (&v)[G]) {
    if constexpr (G >= 4) {
#pragma unroll
        for (int c = 0; c < G / 4; ++c)
            reinterpret_cast<float4 *>(p)[c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
    } else if constexpr (G == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    } else {
        *p = v[0];
    }
}

// Row j of an iterate slice in shared memory ([n_b][G] floats). For G >= 8 the
// 16-byte chunks of a row are permuted by an XOR of bits of j, so that the chunk c
// of random rows spreads over all eight 16-byte bank groups of a 128-byte line
// (without it, rows of 32 or 64 bytes put chunk c in only 4 or 2 of them, and the
// random neighbour gathers of a warp conflict 2-4 times as often).
template <int G>
__device__ __forceinline__ int swz(int j, int c) {
    if constexpr (G == 16) return c ^ ((j >> 1) & 3);
    else if constexpr (G == 8) return c ^ ((j >> 2) & 1);
    else return c;
}

template <int G>
__device__ __forceinline__ void lds_row(const float *base, int j, float (&v)[G]) {
    if constexpr (G >= 8) {
        const float4 *r = reinterpret_cast<const float4 *>(base + j * G);
#pragma unroll
        for (int c = 0; c < G / 4; ++c) {
            const float4 t = r[swz<G>(j, c)];
            v[4 * c] = t.x; v[4 * c + 1] = t.y; v[4 * c + 2] = t.z; v[4 * c + 3] = t.w;
        }
    } else {
        ldg_vec<G>(base + j * G, v);
    }
}

template <int G>
__device__ __forceinline__ void sts_row(float *base, int j, const float (&v)[G]) {
    if constexpr (G >= 8) {
        float4 *r = reinterpret_cast<float4 *>(base + j * G);
#pragma unroll
        for (int c = 0; c < G / 4; ++c)
            r[swz<G>(j, c)] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
    } else {
        st_vec<G>(base + j * G, v);
    }
}

// Stopping rule of Remark S2 inside the resident kernel (eps > 0): block-wide
// sums of (x^(k+1) - x^(k))^2 and (x^(k))^2 per replica of the item (FP32 per
// thread and warp, FP64 across warps); a replica with r^(k) < eps is frozen
// (its later updates keep x) and its step count written; the item ends when
// all of its replicas are frozen.
struct ResidentStop {
    float eps;        // 0: no stopping rule
    int32_t *steps;   // [pair] steps taken, or NULL
    float (*red)[32]; // [warps][2 G] per-warp sums
    int *frozen;      // [G]
    int *all_frozen;
};

// ONECOPY: only x^(k) is held in shared memory ([n_b][G] floats, so G can be
// twice as large as with two copies); each step writes x^(k+1) to the item's
// own contiguous region `gx` of a global scratch array ([n_b][G] floats, L2
// resident) and, after a barrier, reads it back into shared memory.
template <int G, bool STOP, bool ONECOPY>
__device__ __forceinline__ void resident_item(float *__restrict__ x, int R, int64_t lo, int nb, int g0, int D,
                                              const uint16_t *__restrict__ ecol, const float *__restrict__ eval,
                                              const float *__restrict__ h, const float *__restrict__ alpha_row,
                                              int alpha_len, float zs, float xsc, int iters, float *s0, float *s1,
                                              float *gx, int pair0, const ResidentStop &stop) {
    const int T = blockDim.x;
    constexpr bool stopping = STOP;
    // the slot pairs: (column 2p | column 2p + 1 << 16) and (weight 2p, weight 2p + 1);
    // ecol and eval start at an even slot (the widths are even), so these are aligned
    const uint32_t *__restrict__ ecol2 = reinterpret_cast<const uint32_t *>(ecol);
    const float2 *__restrict__ eval2 = reinterpret_cast<const float2 *>(eval);
    for (int i = threadIdx.x; i < nb; i += T) {
        float v[G];
        ldg_vec<G>(x + (lo + i) * R + g0, v);
        sts_row<G>(s0, i, v);
    }
    if (STOP && threadIdx.x < G) {
        stop.frozen[threadIdx.x] = 0;
        if (stop.steps) stop.steps[pair0 + threadIdx.x] = iters;
    }
    if (STOP && threadIdx.x == 0) *stop.all_frozen = 0;
    __syncthreads();
    float *cur = s0, *nxt = s1;
    for (int k = 0; k < iters; ++k) {
        const float a = __ldg(alpha_row + (alpha_len == 1 ? 0 : k));
        bool frz[STOP ? G : 1];
        float dsum[STOP ? G : 1], ssum[STOP ? G : 1];
        if constexpr (STOP) {
#pragma unroll
            for (int q = 0; q < G; ++q) {
                frz[q] = stop.frozen[q];
                dsum[q] = ssum[q] = 0.f;
            }
        }
        for (int i = threadIdx.x; i < nb; i += T) {
            float acc[G];
#pragma unroll
            for (int q = 0; q < G; ++q) acc[q] = 0.f;
            // slot pairs in batches of kPairBatch: the (coalesced) index/weight loads of a
            // batch first, then the shared-memory gathers and products in CSR order
            const int D2 = D >> 1;
            for (int p0 = 0; p0 < D2; p0 += kPairBatch) {
                const int cnt = D2 - p0 < kPairBatch ? D2 - p0 : kPairBatch;
                uint32_t jj[kPairBatch];
                float2 ww[kPairBatch];
#pragma unroll
                for (int q = 0; q < kPairBatch; ++q) {
                    const int at = (p0 + q) * nb + i;  // < D n_b / 2 < 2^31 (checked on the host)
                    jj[q] = q < cnt ? __ldg(ecol2 + at) : 0u;
                    ww[q] = q < cnt ? __ldg(eval2 + at) : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int q = 0; q < kPairBatch; ++q)
                    if (q < cnt) {
                        float xv[G];
                        lds_row<G>(cur, static_cast<int>(jj[q] & 0xffffu), xv);
#pragma unroll
                        for (int r = 0; r < G; ++r) acc[r] += ww[q].x * xv[r];
                        lds_row<G>(cur, static_cast<int>(jj[q] >> 16), xv);
#pragma unroll
                        for (int r = 0; r < G; ++r) acc[r] += ww[q].y * xv[r];
                    }
            }
            float xs[G], out[G];
            lds_row<G>(cur, i, xs);
            const float hv = h ? __ldg(h + lo + i) : 0.f;
#pragma unroll
            for (int q = 0; q < G; ++q) out[q] = cbrt_pow2((acc[q] + a * xs[q] + hv) * zs) * xsc;
            if constexpr (STOP) {
#pragma unroll
                for (int q = 0; q < G; ++q) {
                    if (frz[q]) out[q] = xs[q];
                    const float e = out[q] - xs[q];
                    dsum[q] += e * e;
                    ssum[q] += xs[q] * xs[q];
                }
            }
            if constexpr (ONECOPY) st_vec<G>(gx + static_cast<int64_t>(i) * G, out);
            else sts_row<G>(nxt, i, out);
        }
        if constexpr (STOP) {
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
            for (int q = 0; q < G; ++q) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    dsum[q] += __shfl_xor_sync(0xffffffffu, dsum[q], o);
                    ssum[q] += __shfl_xor_sync(0xffffffffu, ssum[q], o);
                }
                if (lane == 0) {
                    stop.red[warp][q] = dsum[q];
                    stop.red[warp][G + q] = ssum[q];
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                int all = 1;
                for (int q = 0; q < G; ++q) {
                    if (!stop.frozen[q]) {
                        double dd = 0.0, ss = 0.0;
                        for (int w = 0; w < T / 32; ++w) {
                            dd += static_cast<double>(stop.red[w][q]);
                            ss += static_cast<double>(stop.red[w][G + q]);
                        }
                        if (sqrt(dd) / sqrt(ss) < static_cast<double>(stop.eps)) {
                            stop.frozen[q] = 1;
                            if (stop.steps) stop.steps[pair0 + q] = k + 1;
                        }
                    }
                    all &= stop.frozen[q];
                }
                *stop.all_frozen = all;
            }
        }
        __syncthreads();
        if constexpr (ONECOPY) {
            // x^(k+1) back into shared memory (the global writes of this block are visible
            // after the barrier; plain loads, as the data was written in this launch)
            if (k + 1 < iters && !(STOP && *stop.all_frozen)) {
                for (int i = threadIdx.x; i < nb; i += T) {
                    float v[G];
                    ldg_vec<G>(gx + static_cast<int64_t>(i) * G, v);
                    sts_row<G>(cur, i, v);
                }
                __syncthreads();
            }
        } else {
            float *t = cur; cur = nxt; nxt = t;
        }
        if (STOP && *stop.all_frozen) break;  // uniform: read after the barrier
    }
    for (int i = threadIdx.x; i < nb; i += T) {
        float v[G];
        if constexpr (ONECOPY) {
            if (iters > 0) ldg_vec<G>(gx + static_cast<int64_t>(i) * G, v);
            else lds_row<G>(cur, i, v);
        } else {
            lds_row<G>(cur, i, v);
        }
        st_vec<G>(x + (lo + i) * R + g0, v);
    }
}

template <bool STOP, bool ONECOPY, int THREADS>
__global__ void __launch_bounds__(THREADS, 1)
batched_resident(float *__restrict__ x, const uint16_t *__restrict__ ell_col, const float *__restrict__ ell_val,
                 const int64_t *__restrict__ ell_off, const float *__restrict__ h, const int64_t *__restrict__ off,
                 const int4 *__restrict__ items, int n_items, int R, const float *__restrict__ alpha_tab,
                 int alpha_len, const float *__restrict__ zscale_tab, const float *__restrict__ xscale_tab,
                 int iters, float eps, int32_t *__restrict__ steps, int *__restrict__ queue, float *scratch) {
    extern __shared__ float4 res_smem4[];
    __shared__ int next;
    __shared__ float stop_red[STOP ? 32 : 1][32];
    __shared__ int stop_frozen[16];
    __shared__ int stop_all;
    const ResidentStop stop{eps, steps, stop_red, stop_frozen, &stop_all};
    while (true) {
        if (threadIdx.x == 0) next = atomicAdd(queue, 1);
        __syncthreads();  // also: every thread is done with the previous item's shared memory
        const int w = next;
        __syncthreads();
        if (w >= n_items) break;
        const int4 it = __ldg(items + w);  // (instance, first replica, G, ELL slots)
        const int b = it.x;
        const int64_t lo = __ldg(off + b);
        const int nb = static_cast<int>(__ldg(off + b + 1) - lo);
        float *s0 = reinterpret_cast<float *>(res_smem4);
        float *s1 = ONECOPY ? s0 : s0 + static_cast<size_t>(nb) * it.z;
        // the item's region of the one-copy scratch: [instance][replica group][n_b][G]
        float *gx = ONECOPY ? scratch + lo * R + static_cast<int64_t>(it.y) * nb : nullptr;
        const float *arow = alpha_tab + static_cast<int64_t>(b) * alpha_len;
        const float zs = __ldg(zscale_tab + b), xsc = __ldg(xscale_tab + b);
        const int64_t eo = __ldg(ell_off + b);
        const uint16_t *ec = ell_col + eo;
        const float *ev = ell_val + eo;
        switch (it.z) {
            case 16: resident_item<16, STOP, ONECOPY>(x, R, lo, nb, it.y, it.w, ec, ev, h, arow, alpha_len, zs, xsc, iters, s0, s1, gx, b * R + it.y, stop); break;
            case 8: resident_item<8, STOP, ONECOPY>(x, R, lo, nb, it.y, it.w, ec, ev, h, arow, alpha_len, zs, xsc, iters, s0, s1, gx, b * R + it.y, stop); break;
            case 4: resident_item<4, STOP, ONECOPY>(x, R, lo, nb, it.y, it.w, ec, ev, h, arow, alpha_len, zs, xsc, iters, s0, s1, gx, b * R + it.y, stop); break;
            case 2: resident_item<2, STOP, ONECOPY>(x, R, lo, nb, it.y, it.w, ec, ev, h, arow, alpha_len, zs, xsc, iters, s0, s1, gx, b * R + it.y, stop); break;
            default: resident_item<1, STOP, ONECOPY>(x, R, lo, nb, it.y, it.w, ec, ev, h, arow, alpha_len, zs, xsc, iters, s0, s1, gx, b * R + it.y, stop); break;
        }
    }
}

template <bool STOP, bool ONECOPY, int THREADS>
ising_status_t launch_resident_t(ising_context *c, const ResidentItems &its, float *x, int R, const ParamTabs &p,
                                 int iters, float eps, int32_t *steps, float *scratch, cudaStream_t st) {
    auto kern = batched_resident<STOP, ONECOPY, THREADS>;
    const int smem = static_cast<int>(its.smem);
    DOCH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int occ = 0;
    DOCH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, THREADS, smem));
    if (occ < 1) return ISING_ERR_UNSUPPORTED;
    int grid = c->num_sms * occ;
    if (grid > its.count) grid = its.count;
    DOCH_CUDA(cudaMemsetAsync(c->batch_queue, 0, sizeof(int), st));
    kern<<<grid, THREADS, smem, st>>>(x, c->ell_col, c->ell_val, c->ell_off, c->h_f32, c->inst_off,
                                      its.buf.as<int4>(), its.count, R, p.alpha_f, p.alpha_len, p.zscale_f,
                                      p.xscale_f, iters, eps, steps, c->batch_queue, scratch);
    DOCH_CUDA(cudaGetLastError());
    return ISING_OK;
}

ising_status_t launch_resident(ising_context *c, const ResidentConfig &cfg, float *x, int R, const ParamTabs &p,
                               int iters, float eps, int32_t *steps, float *scratch, cudaStream_t st) {
    const ResidentItems &its = c->res_items[cfg.one_copy ? 1 : 0];
    const bool stop = eps > 0.f;
#define DOCH_RES_LAUNCH(S, O, T) return launch_resident_t<S, O, T>(c, its, x, R, p, iters, eps, steps, scratch, st)
    if (cfg.threads == 512) {
        if (stop) { if (cfg.one_copy) DOCH_RES_LAUNCH(true, true, 512); DOCH_RES_LAUNCH(true, false, 512); }
        if (cfg.one_copy) DOCH_RES_LAUNCH(false, true, 512);
        DOCH_RES_LAUNCH(false, false, 512);
    }
    if (stop) { if (cfg.one_copy) DOCH_RES_LAUNCH(true, true, 1024); DOCH_RES_LAUNCH(true, false, 1024); }
    if (cfg.one_copy) DOCH_RES_LAUNCH(false, true, 1024);
    DOCH_RES_LAUNCH(false, false, 1024);
#undef DOCH_RES_LAUNCH
}

}  // namespace

// Work items of the resident kernel for R replicas (cached per handle, variant and R);
// ISING_ERR_UNSUPPORTED when an instance does not fit shared memory even with G = 1.
// copies = 2 (both Jacobi copies in shared memory) or 1 (one copy, the new iterate
// through the global scratch).
ising_status_t resident_items(ising_context *c, int R, bool one_copy) {
    ResidentItems &its = c->res_items[one_copy ? 1 : 0];
    if (its.R == R) return its.count > 0 ? ISING_OK : ISING_ERR_UNSUPPORTED;
    ++its.gen;
    int dev = 0, optin = 0;
    DOCH_CUDA(cudaGetDevice(&dev));
    DOCH_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int64_t cap = optin - 5120;  // the kernel's static shared memory (queue slot, stopping-rule sums)
    const int64_t copies = one_copy ? 1 : 2;
    struct Item { int64_t work; int b, g0, G; };
    std::vector<Item> items;
    size_t smem = 0;
    its.R = R;
    its.count = 0;
    for (int b = 0; b < c->n_inst; ++b) {
        const int64_t nb = c->inst_off_h[b + 1] - c->inst_off_h[b];
        int G = 16;
        while (G > 1 && (R % G != 0 || copies * nb * G * 4 > cap)) G >>= 1;
        if (copies * nb * G * 4 > cap) return ISING_ERR_UNSUPPORTED;
        if (static_cast<int64_t>(c->ell_deg_h[b]) * nb >= (int64_t(1) << 31)) return ISING_ERR_UNSUPPORTED;
        smem = std::max(smem, static_cast<size_t>(copies * nb * G * 4));
        for (int g0 = 0; g0 < R; g0 += G) items.push_back({(nb + c->inst_nnz_h[b]) * G, b, g0, G});
    }
    std::stable_sort(items.begin(), items.end(), [](const Item &u, const Item &v) { return u.work > v.work; });
    std::vector<int4> host(items.size());
    for (size_t i = 0; i < items.size(); ++i)
        host[i] = make_int4(items[i].b, items[i].g0, items[i].G, c->ell_deg_h[items[i].b]);
    DOCH_CHECK(its.buf.ensure(sizeof(int4) * host.size()));
    DOCH_CUDA(cudaMemcpy(its.buf.ptr, host.data(), sizeof(int4) * host.size(), cudaMemcpyHostToDevice));
    its.count = static_cast<int>(host.size());
    its.smem = std::max<size_t>(smem, 16);
    return ISING_OK;
}

bool batched_resident_ok(ising_context *c, float *x, int R) {
    if (!c->batch_queue || !c->ell_col || c->inst_nnz_h.size() != static_cast<size_t>(c->n_inst)) return false;
    if (reinterpret_cast<uintptr_t>(x) % 16 != 0) return false;
    return resident_items(c, R, false) == ISING_OK;
}

ising_status_t batched_resident_launch(ising_context *c, const ResidentConfig &cfg, float *x, int R,
                                       const ParamTabs &p, int iters, cudaStream_t st, float eps, int32_t *steps) {
    if (!c->batch_queue || !c->ell_col || c->inst_nnz_h.size() != static_cast<size_t>(c->n_inst))
        return ISING_ERR_UNSUPPORTED;
    if (reinterpret_cast<uintptr_t>(x) % 16 != 0) return ISING_ERR_UNSUPPORTED;
    const ising_status_t s = resident_items(c, R, cfg.one_copy);
    if (s != ISING_OK) return s;
    float *scratch = nullptr;
    if (cfg.one_copy) {
        DOCH_CHECK(c->res_scratch.ensure(static_cast<size_t>(c->n) * R * sizeof(float)));
        scratch = c->res_scratch.as<float>();
    }
    return launch_resident(c, cfg, x, R, p, iters, eps, steps, scratch, st);
}

ising_status_t batched_launch(const ising_context *c, const BatchedConfig &cfg, float *xa, float *xb, int R,
                              const ParamTabs &p, int iters, cudaStream_t st) {
    if (cfg.vec == 4 && R % 4 == 0) return dispatch_b<4>(c, cfg, xa, xb, R, p, iters, st);
    if (cfg.vec >= 2 && R % 2 == 0) return dispatch_b<2>(c, cfg, xa, xb, R, p, iters, st);
    return dispatch_b<1>(c, cfg, xa, xb, R, p, iters, st);
}

}  // namespace doch
