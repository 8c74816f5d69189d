// Stopping rule of Remark S2 per (instance, replica) pair: after the step
// x^(k) -> x^(k+1), r^(k) = ||x^(k+1) - x^(k)||_2 / ||x^(k)||_2, and a pair
// stops at the first k with r^(k) < eps, keeping x^(k+1).
//  norm pass: per (instance, replica, chunk) block, partial sums of
//             (x^(k+1) - x^(k))^2 and (x^(k))^2 in a fixed order: per thread a
//             compensated FP32 sum for FP32 iterates (FP64 arithmetic runs at a
//             small fraction of the FP32 rate on this part), FP64 for FP64
//             iterates; FP64 across threads;
//  decide:    one block per pair adds the chunk partials in a fixed order,
//             evaluates r^(k) and, for a pair still running, records the step
//             count, marks it stopped and lowers the running-pair counter;
//  keep:      rows of the pairs that stopped at this step are copied to the
//             result; pairs that never stop take x^(max_iters) at the end.
#include <cmath>

#include "hamsum.cuh"
#include "internal.cuh"

namespace doch {
namespace {

constexpr int kSThreads = 256;
constexpr int kDThreads = 128;

template <typename XT>
__global__ void __launch_bounds__(kSThreads)
stop_norms(const XT *__restrict__ xc, const XT *__restrict__ xn, const int64_t *__restrict__ inst_off, int64_t n,
           int R, int chunks, double *__restrict__ partials) {
    const int ch = blockIdx.x, r = blockIdx.y, b = blockIdx.z;
    const int64_t lo = inst_off ? inst_off[b] : 0;
    const int64_t hi = inst_off ? inst_off[b + 1] : n;
    const int64_t len = hi - lo;
    const int64_t s0 = lo + len * ch / chunks, s1 = lo + len * (ch + 1) / chunks;
    double d = 0.0, s = 0.0;
    DotSum32 d32, s32;
    for (int64_t i = s0 + threadIdx.x; i < s1; i += kSThreads) {
        if constexpr (sizeof(XT) == 4) {
            const float a = xc[i * R + r];
            const float e = xn[i * R + r] - a;
            d32.add(e, e);
            s32.add(a, a);
        } else {
            const double a = xc[i * R + r];
            const double e = xn[i * R + r] - a;
            d += e * e;
            s += a * a;
        }
    }
    if constexpr (sizeof(XT) == 4) {
        d = d32.value();
        s = s32.value();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        d += __shfl_xor_sync(0xffffffffu, d, o);
        s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    __shared__ double red[kSThreads / 32][2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[warp][0] = d;
        red[warp][1] = s;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double t = 0.0;
        for (int w = 0; w < kSThreads / 32; ++w) t += red[w][threadIdx.x];
        partials[((static_cast<int64_t>(b) * R + r) * chunks + ch) * 2 + threadIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kDThreads)
stop_decide(const double *__restrict__ partials, int chunks, double eps, int k, int *__restrict__ running,
            int32_t *__restrict__ steps, int *__restrict__ stopped_now, int *__restrict__ n_running) {
    const int t = blockIdx.x;
    __shared__ double red[kDThreads][2];
    double d = 0.0, s = 0.0;
    for (int ch = threadIdx.x; ch < chunks; ch += kDThreads) {
        d += partials[(static_cast<int64_t>(t) * chunks + ch) * 2];
        s += partials[(static_cast<int64_t>(t) * chunks + ch) * 2 + 1];
    }
    red[threadIdx.x][0] = d;
    red[threadIdx.x][1] = s;
    __syncthreads();
    for (int w = kDThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            red[threadIdx.x][0] += red[threadIdx.x + w][0];
            red[threadIdx.x][1] += red[threadIdx.x + w][1];
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    int now = 0;
    if (running[t]) {
        const double rk = std::sqrt(red[0][0]) / std::sqrt(red[0][1]);
        if (rk < eps) {
            running[t] = 0;
            steps[t] = k + 1;
            now = 1;
            atomicSub(n_running, 1);
        }
    }
    stopped_now[t] = now;
}

// rows of the pairs that stopped at this step -> the result
template <typename XT>
__global__ void __launch_bounds__(kSThreads)
stop_keep(const XT *__restrict__ xn, XT *__restrict__ res, const int *__restrict__ flag,
          const int64_t *__restrict__ inst_off, int64_t n, int R, int chunks) {
    const int ch = blockIdx.x, r = blockIdx.y, b = blockIdx.z;
    if (!flag[b * R + r]) return;  // uniform over the block
    const int64_t lo = inst_off ? inst_off[b] : 0;
    const int64_t hi = inst_off ? inst_off[b + 1] : n;
    const int64_t len = hi - lo;
    const int64_t s0 = lo + len * ch / chunks, s1 = lo + len * (ch + 1) / chunks;
    for (int64_t i = s0 + threadIdx.x; i < s1; i += kSThreads) res[i * R + r] = xn[i * R + r];
}

int stop_chunks(const ising_context *c, int R) {
    const int64_t pairs = static_cast<int64_t>(c->n_inst) * R;
    int64_t ch = (4LL * c->num_sms + pairs - 1) / pairs;
    const int64_t cap = (c->max_inst_n + kSThreads - 1) / kSThreads;
    if (ch > cap) ch = cap;
    if (ch < 1) ch = 1;
    if (ch > 65535) ch = 65535;
    return static_cast<int>(ch);
}

template <typename XT>
ising_status_t stop_step_typed(ising_context *c, const XT *xc, const XT *xn, XT *res, int R, double eps, int k,
                               StopState &s, cudaStream_t st) {
    const int chunks = stop_chunks(c, R);
    const int pairs = c->n_inst * R;
    const int64_t *off = c->n_inst > 1 ? c->inst_off : nullptr;
    dim3 grid(static_cast<unsigned>(chunks), static_cast<unsigned>(R), static_cast<unsigned>(c->n_inst));
    stop_norms<XT><<<grid, kSThreads, 0, st>>>(xc, xn, off, c->n, R, chunks, s.partials);
    DOCH_CUDA(cudaGetLastError());
    stop_decide<<<pairs, kDThreads, 0, st>>>(s.partials, chunks, eps, k, s.running, s.steps, s.stopped_now,
                                             s.n_running);
    DOCH_CUDA(cudaGetLastError());
    stop_keep<XT><<<grid, kSThreads, 0, st>>>(xn, res, s.stopped_now, off, c->n, R, chunks);
    DOCH_CUDA(cudaGetLastError());
    return ISING_OK;
}

template <typename XT>
ising_status_t stop_finish_typed(ising_context *c, const XT *xc, XT *res, int R, StopState &s, cudaStream_t st) {
    const int chunks = stop_chunks(c, R);
    const int64_t *off = c->n_inst > 1 ? c->inst_off : nullptr;
    dim3 grid(static_cast<unsigned>(chunks), static_cast<unsigned>(R), static_cast<unsigned>(c->n_inst));
    stop_keep<XT><<<grid, kSThreads, 0, st>>>(xc, res, s.running, off, c->n, R, chunks);
    DOCH_CUDA(cudaGetLastError());
    return ISING_OK;
}

}  // namespace

size_t stop_partials_bytes(const ising_context *c, int R) {
    return sizeof(double) * 2 * static_cast<size_t>(c->n_inst) * R * stop_chunks(c, R);
}

ising_status_t stop_step(ising_context *c, const void *xc, const void *xn, void *res, int xtype, int R, double eps,
                         int k, StopState &s, cudaStream_t st) {
    if (xtype == ISING_F32)
        return stop_step_typed<float>(c, static_cast<const float *>(xc), static_cast<const float *>(xn),
                                      static_cast<float *>(res), R, eps, k, s, st);
    if (xtype == ISING_F64)
        return stop_step_typed<double>(c, static_cast<const double *>(xc), static_cast<const double *>(xn),
                                       static_cast<double *>(res), R, eps, k, s, st);
    return fail(ISING_ERR_INVALID_ARG, "stopping rule: iterates must be F32 or F64");
}

ising_status_t stop_finish(ising_context *c, const void *xc, void *res, int xtype, int R, StopState &s,
                           cudaStream_t st) {
    if (xtype == ISING_F32)
        return stop_finish_typed<float>(c, static_cast<const float *>(xc), static_cast<float *>(res), R, s, st);
    if (xtype == ISING_F64)
        return stop_finish_typed<double>(c, static_cast<const double *>(xc), static_cast<double *>(res), R, s, st);
    return fail(ISING_ERR_INVALID_ARG, "stopping rule: iterates must be F32 or F64");
}

}  // namespace doch
