// Device-side problem generation and parameter rule.
//
// Algorithm S5 (Supplementary Note 9): for every pair i > j draw z in
// {1, ..., N_p}, N_p = floor(102300 / p); if z < 1023 then J_ij = J_ji =
// z - 511. The draw of pair (i, j) is value t = i (i - 1) / 2 + j of a
// counter-based SplitMix64 stream (Steele, Lea and Flood, OOPSLA 2014):
// u = mix(seed + (t + 1) * 0x9E3779B97F4A7C15), z = 1 + floor(u N_p / 2^64),
// so z < 1023 exactly when u < T = ceil(1022 * 2^64 / N_p). Because any
// pair's draw can be recomputed, every row is generated independently and
// already sorted: row i draws (i, j) for j < i and (j, i) for j > i (the
// mirrored entry), one warp per row, in a counting pass and a filling pass
// around an exclusive scan of the row counts. Explicit zeros (z = 511) are
// stored, as in the algorithm.
//
// Parameter rule of Eq. alphabeta on the device: FP64 sums of J_ij and
// J_ij^2 over the off-diagonal entries and the largest row sum of |J_ij|
// (fixed-order block reductions), lambda_max(-J) by the power method on
// -J + ||J||_inf I (FP64, a counter-based start vector, the same stopping
// test as the host rule: |lambda_k - lambda_(k-1)| <= 1e-13 |lambda_k| after
// ten steps, at most 20000 steps), or the Wigner estimate 2 <J> sqrt(n).
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace doch {
namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kM1 = 0xBF58476D1CE4E5B9ull;
constexpr uint64_t kM2 = 0x94D049BB133111EBull;
constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kGThreads = 256;

// device scratch released when the scope ends (error returns included)
struct ScopedBuf {
    DevBuf b;
    ~ScopedBuf() { b.release(); }
};

__host__ __device__ __forceinline__ uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * kM1;
    z = (z ^ (z >> 27)) * kM2;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t s5_draw(uint64_t sd, int64_t i, int64_t j) {
    const uint64_t a = static_cast<uint64_t>(i > j ? i : j), b = static_cast<uint64_t>(i > j ? j : i);
    const uint64_t t = a * (a - 1) / 2 + b;
    return sm_mix(sd + (t + 1) * kGamma);
}

// one warp per row (warp-uniform loops)
__global__ void s5_count(int64_t n, uint64_t sd, uint64_t thr, int64_t *__restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t i = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        int64_t c = 0;
        for (int64_t j0 = 0; j0 < n; j0 += 32) {
            const int64_t j = j0 + lane;
            const bool keep = j < n && j != i && s5_draw(sd, i, j) < thr;
            c += __popc(__ballot_sync(kFullMask, keep));
        }
        if (lane == 0) cnt[i] = c;
    }
}

__global__ void s5_fill(int64_t n, uint64_t sd, uint64_t thr, uint64_t np, const int64_t *__restrict__ row_ptr,
                        int32_t *__restrict__ col, int32_t *__restrict__ val) {
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const int64_t warps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t i = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        int64_t base = row_ptr[i];
        for (int64_t j0 = 0; j0 < n; j0 += 32) {
            const int64_t j = j0 + lane;
            uint64_t u = 0;
            bool keep = false;
            if (j < n && j != i) {
                u = s5_draw(sd, i, j);
                keep = u < thr;
            }
            const unsigned m = __ballot_sync(kFullMask, keep);
            if (keep) {
                const int64_t at = base + __popc(m & below);
                col[at] = static_cast<int32_t>(j);
                val[at] = static_cast<int32_t>(1 + __umul64hi(u, np)) - 511;
            }
            base += __popc(m);
        }
    }
}

// exclusive scan of n int64 counts into out[0..n] (out[n] = total), in
// blocks of kScan, block totals scanned by one thread, then added back
constexpr int kScan = 1024;

__global__ void __launch_bounds__(kScan)
scan_blocks(const int64_t *__restrict__ in, int64_t n, int64_t *__restrict__ out, int64_t *__restrict__ sums) {
    __shared__ int64_t warp_tot[kScan / 32];
    const int64_t i = static_cast<int64_t>(blockIdx.x) * kScan + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t v = i < n ? in[i] : 0;
    int64_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(kFullMask, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t w = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(kFullMask, w, o);
            if (lane >= o) w += y;
        }
        warp_tot[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const int64_t before = warp ? warp_tot[warp - 1] : 0;
    if (i < n) out[i] = before + incl - v;
    if (threadIdx.x == kScan - 1) sums[blockIdx.x] = warp_tot[kScan / 32 - 1];
}

__global__ void scan_sums(int64_t *__restrict__ sums, int64_t nb, int64_t *__restrict__ total) {
    int64_t run = 0;
    for (int64_t b = 0; b < nb; ++b) {
        const int64_t v = sums[b];
        sums[b] = run;
        run += v;
    }
    *total = run;
}

__global__ void scan_add(int64_t *__restrict__ out, int64_t n, const int64_t *__restrict__ sums) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * kScan + threadIdx.x;
    if (i < n) out[i] += sums[blockIdx.x];
}

__global__ void max_count(const int64_t *__restrict__ cnt, int64_t n, unsigned long long *__restrict__ mx) {
    unsigned long long m = 0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        m = m > static_cast<unsigned long long>(cnt[i]) ? m : static_cast<unsigned long long>(cnt[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(kFullMask, m, o);
        m = m > y ? m : y;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(mx, m);
}

// ---- parameter rule --------------------------------------------------------

template <typename VT>
struct CsrRows {
    const int64_t *row_ptr;
    const int32_t *col;
    const VT *val;
    // sums of J_ij, J_ij^2, |J_ij| over row i
    __device__ void stats(int64_t i, double &s1, double &s2, double &sa) const {
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const double w = static_cast<double>(val[e]);
            s1 += w;
            s2 += w * w;
            sa += fabs(w);
        }
    }
    __device__ double product(const double *v, int64_t i) const {
        double s = 0.0;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) s += static_cast<double>(val[e]) * v[col[e]];
        return s;
    }
};

struct TorusRows {
    const int8_t *right, *down;
    int64_t Lr, Lc;
    __device__ void nb(int64_t i, int64_t &l, int64_t &r, int64_t &u, int64_t &d) const {
        const int64_t rr = i / Lc, cc = i - rr * Lc;
        l = rr * Lc + (cc == 0 ? Lc - 1 : cc - 1);
        r = rr * Lc + (cc + 1 == Lc ? 0 : cc + 1);
        u = (rr == 0 ? Lr - 1 : rr - 1) * Lc + cc;
        d = (rr + 1 == Lr ? 0 : rr + 1) * Lc + cc;
    }
    __device__ void stats(int64_t i, double &s1, double &s2, double &sa) const {
        int64_t l, r, u, d;
        nb(i, l, r, u, d);
        const double w[4] = {static_cast<double>(right[i]), static_cast<double>(right[l]),
                             static_cast<double>(down[i]), static_cast<double>(down[u])};
        for (int k = 0; k < 4; ++k) {
            s1 += w[k];
            s2 += w[k] * w[k];
            sa += fabs(w[k]);
        }
    }
    __device__ double product(const double *v, int64_t i) const {
        int64_t l, r, u, d;
        nb(i, l, r, u, d);
        return static_cast<double>(right[i]) * v[r] + static_cast<double>(right[l]) * v[l] +
               static_cast<double>(down[i]) * v[d] + static_cast<double>(down[u]) * v[u];
    }
};

template <typename Acc>
__device__ __forceinline__ Acc wsum(Acc v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
    return v;
}

__device__ __forceinline__ double wmax(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFullMask, v, o));
    return v;
}

// per block: (sum J, sum J^2, max row sum |J|) in a fixed order
template <typename Rows>
__global__ void __launch_bounds__(kGThreads) stats_blocks(Rows rows, int64_t n, double *__restrict__ part) {
    double s1 = 0.0, s2 = 0.0, mx = 0.0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kGThreads + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kGThreads) {
        double sa = 0.0;
        rows.stats(i, s1, s2, sa);
        mx = fmax(mx, sa);
    }
    __shared__ double red[kGThreads / 32][3];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    s1 = wsum(s1);
    s2 = wsum(s2);
    mx = wmax(mx);
    if (lane == 0) {
        red[warp][0] = s1;
        red[warp][1] = s2;
        red[warp][2] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0, c = 0.0;
        for (int w = 0; w < kGThreads / 32; ++w) {
            a += red[w][0];
            b += red[w][1];
            c = fmax(c, red[w][2]);
        }
        part[blockIdx.x * 3] = a;
        part[blockIdx.x * 3 + 1] = b;
        part[blockIdx.x * 3 + 2] = c;
    }
}

// power method step on M = -J + sigma I: y = M v and per-block (v . y, y . y)
template <typename Rows>
__global__ void __launch_bounds__(kGThreads)
power_step(Rows rows, int64_t n, double sigma, const double *__restrict__ v, double *__restrict__ y,
           double *__restrict__ part) {
    double rq = 0.0, yy = 0.0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kGThreads + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kGThreads) {
        const double t = -rows.product(v, i) + sigma * v[i];
        y[i] = t;
        rq += v[i] * t;
        yy += t * t;
    }
    __shared__ double red[kGThreads / 32][2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    rq = wsum(rq);
    yy = wsum(yy);
    if (lane == 0) {
        red[warp][0] = rq;
        red[warp][1] = yy;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < kGThreads / 32; ++w) {
            a += red[w][0];
            b += red[w][1];
        }
        part[blockIdx.x * 2] = a;
        part[blockIdx.x * 2 + 1] = b;
    }
}

// one block: add the partials in block order; lam[it] = v . y; scale = 1 / ||y||
__global__ void power_finish(const double *__restrict__ part, int nblocks, double *__restrict__ lam, int it,
                             double *__restrict__ inv_norm) {
    __shared__ double red[kGThreads][2];
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < nblocks; k += kGThreads) {
        a += part[k * 2];
        b += part[k * 2 + 1];
    }
    red[threadIdx.x][0] = a;
    red[threadIdx.x][1] = b;
    __syncthreads();
    for (int w = kGThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            red[threadIdx.x][0] += red[threadIdx.x + w][0];
            red[threadIdx.x][1] += red[threadIdx.x + w][1];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        lam[it] = red[0][0];
        const double ny = sqrt(red[0][1]);
        *inv_norm = ny > 0.0 ? 1.0 / ny : 0.0;
    }
}

__global__ void scale_vec(double *__restrict__ v, const double *__restrict__ y, int64_t n,
                          const double *__restrict__ inv_norm) {
    const double s = *inv_norm;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        v[i] = y[i] * s;
}

// start vector: counter-based uniform(-1/2, 1/2) draws
__global__ void start_vec(double *__restrict__ v, int64_t n) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        v[i] = static_cast<double>(sm_mix((static_cast<uint64_t>(i) + 1) * kGamma) >> 11) * (1.0 / 9007199254740992.0) -
               0.5;
}

__global__ void sumsq_blocks(const double *__restrict__ v, int64_t n, double *__restrict__ part) {
    double s = 0.0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kGThreads + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kGThreads)
        s += v[i] * v[i];
    __shared__ double red[kGThreads / 32];
    s = wsum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int w = 0; w < kGThreads / 32; ++w) a += red[w];
        part[blockIdx.x * 2] = 0.0;
        part[blockIdx.x * 2 + 1] = a;
    }
}

template <typename Rows>
ising_status_t params_rows(const ising_context *c, const Rows &rows, double eta, int method, double *alpha,
                           double *beta) {
    const int64_t n = c->n;
    int nblocks = static_cast<int>(std::min<int64_t>((n + kGThreads - 1) / kGThreads, 4LL * c->num_sms));
    if (nblocks < 1) nblocks = 1;
    constexpr int kBatchIt = 32;   // power steps between host checks
    constexpr int kMaxIt = 20000;
    ScopedBuf buf;
    const size_t vb = sizeof(double) * n;
    DOCH_CHECK(buf.b.ensure(2 * vb + sizeof(double) * (3 * nblocks + kMaxIt + 8)));
    double *v = buf.b.as<double>(), *y = v + n, *part = y + n, *lam = part + 3 * nblocks, *inv = lam + kMaxIt;
    // sums and the infinity norm
    stats_blocks<Rows><<<nblocks, kGThreads>>>(rows, n, part);
    ising_status_t s = ISING_OK;
    {
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) s = cuda_fail(e, "stats_blocks");
    }
    std::vector<double> hp(3 * nblocks);
    if (s == ISING_OK) {
        const cudaError_t e = cudaMemcpy(hp.data(), part, sizeof(double) * 3 * nblocks, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) s = cuda_fail(e, "cudaMemcpy (stats)");
    }
    if (s != ISING_OK) return s;
    double s1 = 0.0, s2 = 0.0, rowmax = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        s1 += hp[3 * b];
        s2 += hp[3 * b + 1];
        rowmax = std::max(rowmax, hp[3 * b + 2]);
    }
    int meth = method == 0 ? (n < 10000 ? 1 : 2) : method;
    double lam_neg = 0.0;
    if (meth == 2) {
        const double cnt = static_cast<double>(n) * (n - 1.0);
        const double mean = cnt > 0 ? s1 / cnt : 0.0;
        const double var = cnt > 0 ? std::max(0.0, s2 / cnt - mean * mean) : 0.0;
        lam_neg = 2.0 * std::sqrt(var) * std::sqrt(static_cast<double>(n));
    } else {
        const int gb = static_cast<int>(std::min<int64_t>((n + 255) / 256, 16LL * c->num_sms));
        start_vec<<<gb, 256>>>(v, n);
        sumsq_blocks<<<nblocks, kGThreads>>>(v, n, part);
        power_finish<<<1, kGThreads>>>(part, nblocks, lam, 0, inv);
        scale_vec<<<gb, 256>>>(v, v, n, inv);
        std::vector<double> lh(kBatchIt);
        double prev = -1.0, cur = 0.0;
        bool done = false;
        for (int it0 = 0; it0 < kMaxIt && !done && s == ISING_OK; it0 += kBatchIt) {
            const int it1 = std::min(kMaxIt, it0 + kBatchIt);
            for (int it = it0; it < it1; ++it) {
                power_step<Rows><<<nblocks, kGThreads>>>(rows, n, rowmax, v, y, part);
                power_finish<<<1, kGThreads>>>(part, nblocks, lam, it, inv);
                scale_vec<<<gb, 256>>>(v, y, n, inv);
            }
            const cudaError_t e = cudaMemcpy(lh.data(), lam + it0, sizeof(double) * (it1 - it0), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) {
                s = cuda_fail(e, "cudaMemcpy (power method)");
                break;
            }
            for (int it = it0; it < it1; ++it) {  // the host rule's test, step by step
                cur = lh[it - it0];
                if (it > 10 && std::fabs(cur - prev) <= 1e-13 * std::fabs(cur)) {
                    done = true;
                    break;
                }
                prev = cur;
            }
        }
        lam_neg = cur - rowmax;
    }
    if (s != ISING_OK) return s;
    *alpha = eta * lam_neg;
    *beta = std::pow(static_cast<double>(n), 1.5) * (*alpha + rowmax);
    return ISING_OK;
}

}  // namespace

ising_status_t s5_generate(ising_context *c, int64_t n, uint64_t sd, uint64_t thr, uint64_t np) {
    ScopedBuf cnt_buf, sums_buf;
    DevBuf &cnt = cnt_buf.b, &sums = sums_buf.b;
    const int64_t nb = (n + kScan - 1) / kScan;
    DOCH_CHECK(cnt.ensure(sizeof(int64_t) * n));
    DOCH_CHECK(sums.ensure(sizeof(int64_t) * (nb + 2)));
    void *rp = nullptr;
    DOCH_CUDA(cudaMalloc(&rp, sizeof(int64_t) * (n + 1)));
    c->row_ptr = static_cast<int64_t *>(rp);
    const int blocks = static_cast<int>(std::min<int64_t>((n + 7) / 8, 64LL * c->num_sms));
    s5_count<<<blocks, kGThreads>>>(n, sd, thr, cnt.as<int64_t>());
    DOCH_CUDA(cudaGetLastError());
    int64_t *sb = sums.as<int64_t>();
    scan_blocks<<<static_cast<unsigned>(nb), kScan>>>(cnt.as<int64_t>(), n, c->row_ptr, sb);
    scan_sums<<<1, 1>>>(sb, nb, c->row_ptr + n);
    scan_add<<<static_cast<unsigned>(nb), kScan>>>(c->row_ptr, n, sb);
    unsigned long long *mx = reinterpret_cast<unsigned long long *>(sb + nb);
    DOCH_CUDA(cudaMemset(mx, 0, sizeof(unsigned long long)));
    max_count<<<static_cast<int>(std::min<int64_t>((n + 255) / 256, 8LL * c->num_sms)), 256>>>(cnt.as<int64_t>(), n,
                                                                                               mx);
    DOCH_CUDA(cudaGetLastError());
    int64_t nnz = 0;
    unsigned long long rmax = 0;
    DOCH_CUDA(cudaMemcpy(&nnz, c->row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost));
    DOCH_CUDA(cudaMemcpy(&rmax, mx, sizeof(rmax), cudaMemcpyDeviceToHost));
    void *cp = nullptr, *vp = nullptr;
    DOCH_CUDA(cudaMalloc(&cp, sizeof(int32_t) * (nnz > 0 ? nnz : 1)));
    c->col = static_cast<int32_t *>(cp);
    DOCH_CUDA(cudaMalloc(&vp, sizeof(int32_t) * (nnz > 0 ? nnz : 1)));
    c->val = vp;
    s5_fill<<<blocks, kGThreads>>>(n, sd, thr, np, c->row_ptr, c->col, static_cast<int32_t *>(c->val));
    DOCH_CUDA(cudaGetLastError());
    DOCH_CUDA(cudaDeviceSynchronize());
    c->nnz = nnz;
    c->max_row_nnz = static_cast<int64_t>(rmax);
    return ISING_OK;
}

uint64_t s5_stream_seed(uint64_t seed, uint64_t tag) { return sm_mix(seed * kGamma + tag * kM2); }

ising_status_t params_device(const ising_context *c, double eta, int method, double *alpha, double *beta) {
    if (c->format == ISING_FMT_TORUS2D)
        return params_rows(c, TorusRows{c->right, c->down, c->l_rows, c->l_cols}, eta, method, alpha, beta);
    if (c->format != ISING_FMT_CSR) return fail(ISING_ERR_UNSUPPORTED, "device parameters: CSR or TORUS2D");
    switch (c->jtype) {
        case ISING_I8:
            return params_rows(c, CsrRows<int8_t>{c->row_ptr, c->col, static_cast<const int8_t *>(c->val)}, eta,
                               method, alpha, beta);
        case ISING_I32:
            return params_rows(c, CsrRows<int32_t>{c->row_ptr, c->col, static_cast<const int32_t *>(c->val)}, eta,
                               method, alpha, beta);
        case ISING_F32:
            return params_rows(c, CsrRows<float>{c->row_ptr, c->col, static_cast<const float *>(c->val)}, eta,
                               method, alpha, beta);
        case ISING_F64:
            return params_rows(c, CsrRows<double>{c->row_ptr, c->col, static_cast<const double *>(c->val)}, eta,
                               method, alpha, beta);
        default: return fail(ISING_ERR_UNSUPPORTED, "device parameters: coupling type");
    }
}

}  // namespace doch
