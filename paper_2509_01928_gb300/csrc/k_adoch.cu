// ADOCH (Algorithm 2): the DOCH map with a Nesterov-type extrapolation that
// is kept only when it passes a non-monotone test on the DC Hamiltonian H of
// Eq. Hamilton, H(x) = beta/4 sum x^4 - alpha/2 sum x^2 - 1/2 x^T J x - h^T x:
//   t_0 = 1, t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2, c_k = (t_k - 1) / t_{k+1},
//   y^k = x^k + c_k (x^k - x^{k-1})   (y^0 = x^0),
//   v^k = y^k if H(y^k) <= max(H(x^{max(0,k-q)}), ..., H(x^k)), else x^k,
//   x^{k+1} = T(v^k) = cbrt((J v^k + alpha v^k + h) / beta).
// One coupling product per step, by linearity: u^k = J x^k is formed once,
// J y^k = (1 + c_k) u^k - c_k u^{k-1}, and J v^k is u^k or J y^k. Each step is
//  (1) pass: u^k and, per (instance, replica, chunk) block, FP64 partial sums
//      of the terms of H(x^k) and H(y^k) in a fixed order;
//  (2) decide: one block per (instance, replica) adds the chunk partials in a
//      fixed order, forms H(x^k) and H(y^k), keeps the last q+1 values of H(x)
//      and sets the acceptance flag;
//  (3) update: x^{k+1} = T(v^k) element-wise.
// The coupling product and the update run in the iterate's precision (as the
// DOCH step kernels); H is reduced in FP64 across threads and blocks. With
// FP32 iterates each thread first sums its sites' terms in FP32 with Kahan
// compensation (FP64 arithmetic is a small fraction of the FP32 rate here),
// with FP64 iterates in FP64.
#include <cmath>
#include <utility>

#include "internal.cuh"

namespace doch {
namespace {

constexpr int kAThreads = 256;
constexpr int kTerms = 8;  // x^4, x^2, x u, h x, y^4, y^2, y Jy, h y

template <typename T>
__device__ __forceinline__ T acbrt(T z) {
    if constexpr (sizeof(T) == 4) return cbrtf(z);
    else return cbrt(z);
}

// scale by 1/beta: float tables hold 1/beta (multiply), double tables hold beta (divide)
template <typename T>
__device__ __forceinline__ T ascale(T v, T b) {
    if constexpr (sizeof(T) == 4) return v * b;
    else return v / b;
}

// u_i = (J x)_i for replica r, in the iterate's precision and the step kernels' order
template <typename XT, typename VT>
struct CsrProduct {
    const int64_t *row_ptr;
    const int32_t *col;
    const VT *val;
    static constexpr bool kGrid = false;
    __device__ XT operator()(const XT *x, int64_t i, int64_t, int64_t, int r, int R) const {
        XT acc = XT(0);
        const int64_t e1 = row_ptr[i + 1];
        for (int64_t e = row_ptr[i]; e < e1; ++e)
            acc += static_cast<XT>(val[e]) * x[static_cast<int64_t>(col[e]) * R + r];
        return acc;
    }
};

template <typename XT>
struct TorusProduct {
    const int8_t *right, *down;
    int64_t Lr, Lc;
    static constexpr bool kGrid = true;  // wants the (row, column) of site i
    __device__ XT operator()(const XT *x, int64_t i, int64_t rr, int64_t cc, int r, int R) const {
        const int64_t s_l = rr * Lc + (cc == 0 ? Lc - 1 : cc - 1);
        const int64_t s_r = rr * Lc + (cc + 1 == Lc ? 0 : cc + 1);
        const int64_t s_u = (rr == 0 ? Lr - 1 : rr - 1) * Lc + cc;
        const int64_t s_d = (rr + 1 == Lr ? 0 : rr + 1) * Lc + cc;
        return static_cast<XT>(right[i]) * x[s_r * R + r] + static_cast<XT>(right[s_l]) * x[s_l * R + r] +
               static_cast<XT>(down[i]) * x[s_d * R + r] + static_cast<XT>(down[s_u]) * x[s_u * R + r];
    }
};

template <typename Acc>
__device__ __forceinline__ Acc warp_sum(Acc v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// (1) grid (chunks, R, n_inst): rows of instance b in chunk ch, replica r
template <typename XT, typename Fn>
__global__ void __launch_bounds__(kAThreads)
adoch_pass(Fn fn, const XT *__restrict__ x1, const XT *__restrict__ x0, const XT *__restrict__ u0,
           XT *__restrict__ u1, const double *__restrict__ h, const int64_t *__restrict__ inst_off, int64_t n,
           int R, int chunks, XT c, double *__restrict__ partials) {
    const int ch = blockIdx.x, r = blockIdx.y, b = blockIdx.z;
    const int64_t lo = inst_off ? inst_off[b] : 0;
    const int64_t hi = inst_off ? inst_off[b + 1] : n;
    const int64_t len = hi - lo;
    const int64_t s0 = lo + len * ch / chunks, s1 = lo + len * (ch + 1) / chunks;
    // per-thread sums: FP32 with Kahan compensation for FP32 iterates, FP64 otherwise
    using Acc = XT;
    Acc acc[kTerms], cmp[kTerms];
#pragma unroll
    for (int k = 0; k < kTerms; ++k) acc[k] = cmp[k] = Acc(0);
    auto add = [&](int k, Acc v) {
        if constexpr (sizeof(XT) == 4) {
            const Acc y = v - cmp[k];
            const Acc t = acc[k] + y;
            cmp[k] = (t - acc[k]) - y;
            acc[k] = t;
        } else {
            acc[k] += v;
        }
    };
    // (row, column) of the site, advanced without division (lattice only)
    int64_t rr = 0, cc = 0, Lc = 1;
    if constexpr (Fn::kGrid) {
        Lc = fn.Lc;
        rr = (s0 + threadIdx.x) / Lc;
        cc = (s0 + threadIdx.x) - rr * Lc;
    }
    for (int64_t i = s0 + threadIdx.x; i < s1; i += kAThreads) {
        const int64_t at = i * R + r;
        const XT u = fn(x1, i, rr, cc, r, R);
        u1[at] = u;
        const XT xv = x1[at];
        const XT y = xv + c * (xv - x0[at]);
        const XT jy = (XT(1) + c) * u - c * u0[at];
        const XT hv = h ? static_cast<XT>(h[i]) : XT(0);
        const XT x2 = xv * xv, y2 = y * y;
        add(0, x2 * x2);
        add(1, x2);
        add(2, xv * u);
        add(3, hv * xv);
        add(4, y2 * y2);
        add(5, y2);
        add(6, y * jy);
        add(7, hv * y);
        if constexpr (Fn::kGrid) {
            cc += kAThreads;
            while (cc >= Lc) {
                cc -= Lc;
                ++rr;
            }
        }
    }
    __shared__ double red[kAThreads / 32][kTerms];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < kTerms; ++k) {
        const double v = warp_sum(static_cast<double>(acc[k]) - static_cast<double>(cmp[k]));
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < kTerms) {
        double t = 0.0;
        for (int w = 0; w < kAThreads / 32; ++w) t += red[w][threadIdx.x];
        partials[((static_cast<int64_t>(b) * R + r) * chunks + ch) * kTerms + threadIdx.x] = t;
    }
}

// (2) one block per (instance, replica) pair t = b R + r: the chunk partials
// are added by the block's threads in a fixed strided order and a fixed tree
constexpr int kDThreads = 128;
__global__ void __launch_bounds__(kDThreads)
adoch_decide(const double *__restrict__ partials, int n_inst, int R, int chunks,
             const double *__restrict__ alpha_tab, const double *__restrict__ beta_tab, int k, int q,
             double *__restrict__ hist, int *__restrict__ dec, int8_t *__restrict__ acc_out,
             double *__restrict__ H_out) {
    const int t = blockIdx.x;
    const int b = t / R;
    __shared__ double red[kDThreads][kTerms];
    double s[kTerms];
#pragma unroll
    for (int j = 0; j < kTerms; ++j) s[j] = 0.0;
    for (int ch = threadIdx.x; ch < chunks; ch += kDThreads)
#pragma unroll
        for (int j = 0; j < kTerms; ++j) s[j] += partials[(static_cast<int64_t>(t) * chunks + ch) * kTerms + j];
#pragma unroll
    for (int j = 0; j < kTerms; ++j) red[threadIdx.x][j] = s[j];
    __syncthreads();
    for (int w = kDThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int j = 0; j < kTerms; ++j) red[threadIdx.x][j] += red[threadIdx.x + w][j];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double a = alpha_tab[b], be = beta_tab[b];
    const double Hx = be / 4.0 * red[0][0] - a / 2.0 * red[0][1] - 0.5 * red[0][2] - red[0][3];
    const double Hy = be / 4.0 * red[0][4] - a / 2.0 * red[0][5] - 0.5 * red[0][6] - red[0][7];
    double *ht = hist + static_cast<int64_t>(t) * (q + 1);
    ht[k % (q + 1)] = Hx;
    double m = Hx;
    for (int j = (k > q ? k - q : 0); j <= k; ++j) m = fmax(m, ht[j % (q + 1)]);
    const int accept = Hy <= m ? 1 : 0;
    dec[t] = accept;
    if (acc_out) acc_out[static_cast<int64_t>(k) * n_inst * R + t] = static_cast<int8_t>(accept);
    if (H_out) H_out[static_cast<int64_t>(k) * n_inst * R + t] = Hx;
}

// (3) grid (chunks, R, n_inst): x^{k+1} = T(v^k)
template <typename XT>
__global__ void __launch_bounds__(kAThreads)
adoch_update(const XT *__restrict__ x1, const XT *__restrict__ x0, const XT *__restrict__ u1,
             const XT *__restrict__ u0, XT *__restrict__ x2, const XT *__restrict__ h,
             const int64_t *__restrict__ inst_off, int64_t n, int R, int chunks, XT c,
             const XT *__restrict__ alpha_tab, const XT *__restrict__ beta_tab, const int *__restrict__ dec) {
    const int ch = blockIdx.x, r = blockIdx.y, b = blockIdx.z;
    const int64_t lo = inst_off ? inst_off[b] : 0;
    const int64_t hi = inst_off ? inst_off[b + 1] : n;
    const int64_t len = hi - lo;
    const int64_t s0 = lo + len * ch / chunks, s1 = lo + len * (ch + 1) / chunks;
    const bool use_y = dec[b * R + r] != 0;
    const XT a = alpha_tab[b], bb = beta_tab[b];
    for (int64_t i = s0 + threadIdx.x; i < s1; i += kAThreads) {
        const int64_t at = i * R + r;
        const XT xv = x1[at], u = u1[at];
        XT v = xv, jv = u;
        if (use_y) {
            v = xv + c * (xv - x0[at]);
            jv = (XT(1) + c) * u - c * u0[at];
        }
        const XT hv = h ? h[i] : XT(0);
        x2[at] = acbrt(ascale(jv + a * v + hv, bb));
    }
}

int adoch_chunks(const ising_context *c, int R) {
    const int64_t pairs = static_cast<int64_t>(c->n_inst) * R;
    int64_t ch = (4LL * c->num_sms + pairs - 1) / pairs;
    const int64_t cap = (c->max_inst_n + kAThreads - 1) / kAThreads;
    if (ch > cap) ch = cap;
    if (ch < 1) ch = 1;
    if (ch > 65535) ch = 65535;
    return static_cast<int>(ch);
}

template <typename XT, typename Fn>
ising_status_t adoch_run(ising_context *c, const Fn &fn, XT *x, int R, const ParamTabs &p, const XT *h_x,
                         int iters, int q, int8_t *acc_dev, double *H_dev, cudaStream_t st) {
    const int64_t count = c->n * R;
    const int pairs = c->n_inst * R;
    const int chunks = adoch_chunks(c, R);
    auto al = [](size_t v) { return (v + 255) & ~static_cast<size_t>(255); };
    const size_t xb = al(sizeof(XT) * count);
    const size_t pb = al(sizeof(double) * static_cast<size_t>(pairs) * chunks * kTerms);
    const size_t hb = al(sizeof(double) * static_cast<size_t>(pairs) * (q + 1));
    const size_t db = al(sizeof(int) * static_cast<size_t>(pairs));
    DOCH_CHECK(c->ckpt.ensure(4 * xb + pb + hb + db));
    unsigned char *base = c->ckpt.as<unsigned char>();
    XT *bx[3] = {x, reinterpret_cast<XT *>(base), reinterpret_cast<XT *>(base + xb)};  // x^k, x^{k-1}, x^{k+1}
    XT *bu[2] = {reinterpret_cast<XT *>(base + 2 * xb), reinterpret_cast<XT *>(base + 3 * xb)};  // u^{k-1}, u^k
    double *part = reinterpret_cast<double *>(base + 4 * xb);
    double *hist = reinterpret_cast<double *>(base + 4 * xb + pb);
    int *dec = reinterpret_cast<int *>(base + 4 * xb + pb + hb);
    XT *x1 = bx[0], *x0 = bx[1], *x2 = bx[2], *u0 = bu[0], *u1 = bu[1];
    DOCH_CUDA(cudaMemcpyAsync(x0, x1, sizeof(XT) * count, cudaMemcpyDeviceToDevice, st));  // x^{-1} := x^0
    DOCH_CUDA(cudaMemsetAsync(u0, 0, sizeof(XT) * count, st));
    const XT *alpha = nullptr, *beta = nullptr;
    if constexpr (sizeof(XT) == 4) {
        alpha = p.alpha_f;
        beta = p.inv_beta_f;
    } else {
        alpha = p.alpha_d;
        beta = p.beta_d;
    }
    const int64_t *off = c->n_inst > 1 ? c->inst_off : nullptr;
    const double *h_d = c->has_h ? c->h_f64 : nullptr;
    dim3 grid(static_cast<unsigned>(chunks), static_cast<unsigned>(R), static_cast<unsigned>(c->n_inst));
    double t = 1.0;
    for (int k = 0; k < iters; ++k) {
        const double t_next = (1.0 + std::sqrt(1.0 + 4.0 * t * t)) / 2.0;
        const XT ck = static_cast<XT>(k >= 1 ? (t - 1.0) / t_next : 0.0);
        adoch_pass<XT, Fn><<<grid, kAThreads, 0, st>>>(fn, x1, x0, u0, u1, h_d, off, c->n, R, chunks, ck, part);
        DOCH_CUDA(cudaGetLastError());
        adoch_decide<<<pairs, kDThreads, 0, st>>>(part, c->n_inst, R, chunks, p.alpha_d, p.beta_d, k, q, hist,
                                                  dec, acc_dev, H_dev);
        DOCH_CUDA(cudaGetLastError());
        adoch_update<XT><<<grid, kAThreads, 0, st>>>(x1, x0, u1, u0, x2, h_x, off, c->n, R, chunks, ck, alpha,
                                                     beta, dec);
        DOCH_CUDA(cudaGetLastError());
        // rotate: x^{k-1} <- x^k <- x^{k+1}, u^{k-1} <- u^k
        XT *tx = x0;
        x0 = x1;
        x1 = x2;
        x2 = tx;
        std::swap(u0, u1);
        t = t_next;
    }
    if (x1 != x) DOCH_CUDA(cudaMemcpyAsync(x, x1, sizeof(XT) * count, cudaMemcpyDeviceToDevice, st));
    return ISING_OK;
}

template <typename XT>
ising_status_t adoch_dispatch(ising_context *c, XT *x, int R, const ParamTabs &p, const XT *h_x, int iters,
                              int q, int8_t *acc_dev, double *H_dev, cudaStream_t st) {
    if (c->format == ISING_FMT_TORUS2D)
        return adoch_run<XT>(c, TorusProduct<XT>{c->right, c->down, c->l_rows, c->l_cols}, x, R, p, h_x, iters,
                             q, acc_dev, H_dev, st);
    if (c->format != ISING_FMT_CSR) return fail(ISING_ERR_UNSUPPORTED, "ADOCH runs on CSR or TORUS2D couplings");
    switch (c->jtype) {
        case ISING_I8:
            return adoch_run<XT>(c, CsrProduct<XT, int8_t>{c->row_ptr, c->col, static_cast<const int8_t *>(c->val)},
                                 x, R, p, h_x, iters, q, acc_dev, H_dev, st);
        case ISING_I32:
            return adoch_run<XT>(c, CsrProduct<XT, int32_t>{c->row_ptr, c->col, static_cast<const int32_t *>(c->val)},
                                 x, R, p, h_x, iters, q, acc_dev, H_dev, st);
        case ISING_F32:
            return adoch_run<XT>(c, CsrProduct<XT, float>{c->row_ptr, c->col, static_cast<const float *>(c->val)},
                                 x, R, p, h_x, iters, q, acc_dev, H_dev, st);
        case ISING_F64:
            return adoch_run<XT>(c, CsrProduct<XT, double>{c->row_ptr, c->col, static_cast<const double *>(c->val)},
                                 x, R, p, h_x, iters, q, acc_dev, H_dev, st);
        default: return fail(ISING_ERR_UNSUPPORTED, "CSR value type not supported on the device");
    }
}

}  // namespace

ising_status_t adoch_iterate(ising_context *c, void *x, int xtype, int R, const ParamTabs &p, int iters, int q,
                             int8_t *acc_dev, double *H_dev, cudaStream_t st) {
    if (xtype == ISING_F32)
        return adoch_dispatch<float>(c, static_cast<float *>(x), R, p, c->has_h ? c->h_f32 : nullptr, iters, q,
                                     acc_dev, H_dev, st);
    if (xtype == ISING_F64)
        return adoch_dispatch<double>(c, static_cast<double *>(x), R, p, c->has_h ? c->h_f64 : nullptr, iters, q,
                                      acc_dev, H_dev, st);
    return fail(ISING_ERR_INVALID_ARG, "ADOCH iterates must be F32 or F64");
}

}  // namespace doch
