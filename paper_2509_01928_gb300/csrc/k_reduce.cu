// Readout reductions: sign rounding (Algorithm 1, return step; sign(0) = +1),
// the Ising energy E = -1/2 s^T J s - h^T s (Eq. IsingModel), the cut value
// cut = 1/4 sum_ij (1 - s_i s_j) W_ij with W = -2J (Supplementary Note 5),
// the Hamiltonian H(x) of Eq. Hamilton (plus -h^T x), and argmin_r E_r.
//
// Every reduction runs over (instance b, replica r, chunk c) blocks: a block
// sums its rows in a fixed thread/warp order and writes one partial per
// (b, r, c); a second kernel adds the chunk partials of each (b, r) in
// chunk order. Integer couplings accumulate in int64 (exact); real couplings
// in FP64 with that fixed order, so results are identical run to run.
//
// Per-row contributions (acc[0] = sum_j J_ij s_i s_j, acc[1] = sum_j J_ij
// (1 - s_i s_j), acc[2] = h_i s_i) give E = -acc0/2 - acc2 and
// cut = -acc1/2 after the sums over all rows.
#include <cuda_bf16.h>

#include <type_traits>

#include "internal.cuh"

namespace doch {
namespace {

constexpr int kRThreads = 256;

template <typename XT>
__device__ __forceinline__ int spin_of(XT v) {
    if constexpr (sizeof(XT) == 2) return __bfloat162float(v) >= 0.f ? 1 : -1;
    else return v >= XT(0) ? 1 : -1;
}

template <typename XT>
__device__ __forceinline__ double as_double(XT v) {
    if constexpr (sizeof(XT) == 2) return static_cast<double>(__bfloat162float(v));
    else return static_cast<double>(v);
}

template <typename Acc>
__device__ __forceinline__ Acc warp_sum(Acc v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int K, typename Acc, typename Fn>
__global__ void __launch_bounds__(kRThreads)
row_reduce(Fn fn, const int64_t *__restrict__ inst_off, int64_t n, int R, int chunks,
           Acc *__restrict__ partials) {
    const int ch = blockIdx.x, r = blockIdx.y, b = blockIdx.z;
    const int64_t lo = inst_off ? inst_off[b] : 0;
    const int64_t hi = inst_off ? inst_off[b + 1] : n;
    const int64_t len = hi - lo;
    const int64_t s0 = lo + len * ch / chunks, s1 = lo + len * (ch + 1) / chunks;
    Acc acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = Acc(0);
    for (int64_t i = s0 + threadIdx.x; i < s1; i += kRThreads) fn(i, r, acc);
    __shared__ Acc red[kRThreads / 32][K];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const Acc v = warp_sum(acc[k]);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        Acc t = Acc(0);
        for (int w = 0; w < kRThreads / 32; ++w) t += red[w][threadIdx.x];
        partials[((static_cast<int64_t>(b) * R + r) * chunks + ch) * K + threadIdx.x] = t;
    }
}

// ---- energy functors -------------------------------------------------------

template <typename XT, typename VT, typename Acc>
struct CsrEnergy {
    const XT *x;
    const int64_t *row_ptr;
    const int32_t *col;
    const VT *val;
    const Acc *h;
    int R;
    __device__ void operator()(int64_t i, int r, Acc *acc) const {
        const int si = spin_of(x[i * R + r]);
        Acc q = Acc(0), cw = Acc(0);
        const int64_t e1 = row_ptr[i + 1];
        for (int64_t e = row_ptr[i]; e < e1; ++e) {
            const int sj = spin_of(x[static_cast<int64_t>(col[e]) * R + r]);
            const Acc w = static_cast<Acc>(val[e]);
            q += w * static_cast<Acc>(sj);
            cw += w * static_cast<Acc>(1 - si * sj);
        }
        acc[0] += static_cast<Acc>(si) * q;
        acc[1] += cw;
        if (h) acc[2] += h[i] * static_cast<Acc>(si);
    }
};

template <typename XT, typename Acc>
struct TorusEnergy {
    const XT *x;
    const int8_t *right, *down;
    int64_t Lr, Lc;
    int R;
    __device__ void operator()(int64_t i, int r, Acc *acc) const {
        const int64_t rr = i / Lc, cc = i - rr * Lc;
        const int64_t jr = rr * Lc + (cc + 1 == Lc ? 0 : cc + 1);
        const int64_t jd = (rr + 1 == Lr ? 0 : rr + 1) * Lc + cc;
        const int s = spin_of(x[i * R + r]);
        const int sr = spin_of(x[jr * R + r]);
        const int sd = spin_of(x[jd * R + r]);
        const Acc wr = static_cast<Acc>(right[i]), wd = static_cast<Acc>(down[i]);
        // each lattice edge enters sum_{i,j} twice (J_ab and J_ba)
        acc[0] += Acc(2) * (wr * static_cast<Acc>(s * sr) + wd * static_cast<Acc>(s * sd));
        acc[1] += Acc(2) * (wr * static_cast<Acc>(1 - s * sr) + wd * static_cast<Acc>(1 - s * sd));
    }
};

// ---- Hamiltonian functors (acc: sum x^4, sum x^2, sum x u, sum h x) --------

template <typename XT, typename VT>
struct CsrHam {
    const XT *x;
    const int64_t *row_ptr;
    const int32_t *col;
    const VT *val;
    const double *h;
    int R;
    __device__ void operator()(int64_t i, int r, double *acc) const {
        double u = 0.0;
        const int64_t e1 = row_ptr[i + 1];
        for (int64_t e = row_ptr[i]; e < e1; ++e)
            u += static_cast<double>(val[e]) * as_double(x[static_cast<int64_t>(col[e]) * R + r]);
        const double xi = as_double(x[i * R + r]);
        const double x2 = xi * xi;
        acc[0] += x2 * x2;
        acc[1] += x2;
        acc[2] += xi * u;
        if (h) acc[3] += h[i] * xi;
    }
};

template <typename XT>
struct TorusHam {
    const XT *x;
    const int8_t *right, *down;
    int64_t Lr, Lc;
    int R;
    __device__ void operator()(int64_t i, int r, double *acc) const {
        const int64_t rr = i / Lc, cc = i - rr * Lc;
        const int64_t jl = rr * Lc + (cc == 0 ? Lc - 1 : cc - 1);
        const int64_t jr = rr * Lc + (cc + 1 == Lc ? 0 : cc + 1);
        const int64_t ju = (rr == 0 ? Lr - 1 : rr - 1) * Lc + cc;
        const int64_t jd = (rr + 1 == Lr ? 0 : rr + 1) * Lc + cc;
        const double u = right[i] * as_double(x[jr * R + r]) + right[jl] * as_double(x[jl * R + r]) +
                         down[i] * as_double(x[jd * R + r]) + down[ju] * as_double(x[ju * R + r]);
        const double xi = as_double(x[i * R + r]);
        const double x2 = xi * xi;
        acc[0] += x2 * x2;
        acc[1] += x2;
        acc[2] += xi * u;
    }
};

// ---- finalisers ------------------------------------------------------------

template <typename Acc>
__global__ void energy_finish(const Acc *__restrict__ partials, int pairs, int chunks,
                              int64_t *E_i, int64_t *cut_i, double *E_d, double *cut_d) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= pairs) return;
    Acc s[3] = {Acc(0), Acc(0), Acc(0)};
    for (int c = 0; c < chunks; ++c)
        for (int k = 0; k < 3; ++k) s[k] += partials[(static_cast<int64_t>(t) * chunks + c) * 3 + k];
    if constexpr (std::is_integral<Acc>::value) {  // int64: exact
        const int64_t E = -(s[0] / 2) - s[2];
        const int64_t cut = -(s[1] / 2);
        if (E_i) E_i[t] = E;
        if (cut_i) cut_i[t] = cut;
        if (E_d) E_d[t] = static_cast<double>(E);
        if (cut_d) cut_d[t] = static_cast<double>(cut);
    } else {
        if (E_d) E_d[t] = -0.5 * s[0] - s[2];
        if (cut_d) cut_d[t] = -0.5 * s[1];
    }
}

// H(x^(k)) per replica from the fused monitor's partials [block][R][4], blocks in order
__global__ void ham_fused_finish(const double *__restrict__ hpart, int blocks, int R, double alpha, double beta,
                                 double *__restrict__ H) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = 0; b < blocks; ++b)
#pragma unroll
        for (int m = 0; m < 4; ++m) t[m] += hpart[(static_cast<int64_t>(b) * R + r) * 4 + m];
    H[r] = beta / 4.0 * t[0] - alpha / 2.0 * t[1] - 0.5 * t[2] - t[3];
}

__global__ void ham_finish(const double *__restrict__ partials, int n_inst, int R, int chunks,
                           const double *__restrict__ alpha_tab, int alpha_len, int k,
                           const double *__restrict__ beta_tab, double *__restrict__ H) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_inst * R) return;
    const int b = t / R;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int c = 0; c < chunks; ++c)
        for (int q = 0; q < 4; ++q) s[q] += partials[(static_cast<int64_t>(t) * chunks + c) * 4 + q];
    const double a = alpha_tab[static_cast<int64_t>(b) * alpha_len + (k < alpha_len ? k : alpha_len - 1)];
    const double be = beta_tab[b];
    H[t] = be / 4.0 * s[0] - a / 2.0 * s[1] - 0.5 * s[2] - s[3];
}

__global__ void best_kernel(const int64_t *__restrict__ E_i, const double *__restrict__ E_d,
                            int n_inst, int R, int32_t *__restrict__ best) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_inst) return;
    int arg = 0;
    if (E_i) {
        int64_t m = E_i[static_cast<int64_t>(b) * R];
        for (int r = 1; r < R; ++r)
            if (E_i[static_cast<int64_t>(b) * R + r] < m) { m = E_i[static_cast<int64_t>(b) * R + r]; arg = r; }
    } else {
        double m = E_d[static_cast<int64_t>(b) * R];
        for (int r = 1; r < R; ++r)
            if (E_d[static_cast<int64_t>(b) * R + r] < m) { m = E_d[static_cast<int64_t>(b) * R + r]; arg = r; }
    }
    best[b] = arg;
}

template <typename XT>
__global__ void spins_kernel(const XT *__restrict__ x, int64_t count, int8_t *__restrict__ s) {
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < count;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x)
        s[t] = static_cast<int8_t>(spin_of(x[t]));
}

int pick_chunks(const ising_context *c, int R) {
    const int64_t pairs = static_cast<int64_t>(c->n_inst) * R;
    const int64_t want = 4LL * c->num_sms;
    int64_t ch = (want + pairs - 1) / pairs;
    const int64_t cap = (c->max_inst_n + kRThreads - 1) / kRThreads;
    if (ch > cap) ch = cap;
    if (ch < 1) ch = 1;
    if (ch > 65535) ch = 65535;
    return static_cast<int>(ch);
}

template <int K, typename Acc, typename Fn>
ising_status_t run_reduce(ising_context *c, const Fn &fn, int R, int chunks, cudaStream_t st) {
    const size_t bytes = static_cast<size_t>(c->n_inst) * R * chunks * K * sizeof(Acc);
    DOCH_CHECK(c->partials.ensure(bytes));
    dim3 grid(static_cast<unsigned>(chunks), static_cast<unsigned>(R), static_cast<unsigned>(c->n_inst));
    row_reduce<K, Acc, Fn><<<grid, kRThreads, 0, st>>>(fn, c->n_inst > 1 ? c->inst_off : nullptr,
                                                        c->n, R, chunks, c->partials.as<Acc>());
    DOCH_CUDA(cudaGetLastError());
    return ISING_OK;
}

template <typename XT, typename Acc>
ising_status_t energy_typed(ising_context *c, const XT *x, int R, int chunks, cudaStream_t st) {
    if (c->format == ISING_FMT_TORUS2D) {
        TorusEnergy<XT, Acc> fn{x, c->right, c->down, c->l_rows, c->l_cols, R};
        return run_reduce<3, Acc>(c, fn, R, chunks, st);
    }
    if (c->format == ISING_FMT_CSR) {
        const Acc *h = nullptr;
        if constexpr (std::is_integral<Acc>::value) h = reinterpret_cast<const Acc *>(c->h_i64);
        else h = reinterpret_cast<const Acc *>(c->h_f64);
        switch (c->jtype) {
            case ISING_I8: return run_reduce<3, Acc>(c, CsrEnergy<XT, int8_t, Acc>{x, c->row_ptr, c->col, static_cast<const int8_t *>(c->val), h, R}, R, chunks, st);
            case ISING_I32: return run_reduce<3, Acc>(c, CsrEnergy<XT, int32_t, Acc>{x, c->row_ptr, c->col, static_cast<const int32_t *>(c->val), h, R}, R, chunks, st);
            case ISING_F32: return run_reduce<3, Acc>(c, CsrEnergy<XT, float, Acc>{x, c->row_ptr, c->col, static_cast<const float *>(c->val), h, R}, R, chunks, st);
            case ISING_F64: return run_reduce<3, Acc>(c, CsrEnergy<XT, double, Acc>{x, c->row_ptr, c->col, static_cast<const double *>(c->val), h, R}, R, chunks, st);
            default: break;
        }
    }
    return fail(ISING_ERR_UNSUPPORTED, "energy: storage form not supported by this reduction");
}

template <typename XT>
ising_status_t ham_typed(ising_context *c, const XT *x, int R, int chunks, cudaStream_t st) {
    if (c->format == ISING_FMT_TORUS2D)
        return run_reduce<4, double>(c, TorusHam<XT>{x, c->right, c->down, c->l_rows, c->l_cols, R}, R, chunks, st);
    if (c->format == ISING_FMT_CSR) {
        const double *h = c->has_h ? c->h_f64 : nullptr;
        switch (c->jtype) {
            case ISING_I8: return run_reduce<4, double>(c, CsrHam<XT, int8_t>{x, c->row_ptr, c->col, static_cast<const int8_t *>(c->val), h, R}, R, chunks, st);
            case ISING_I32: return run_reduce<4, double>(c, CsrHam<XT, int32_t>{x, c->row_ptr, c->col, static_cast<const int32_t *>(c->val), h, R}, R, chunks, st);
            case ISING_F32: return run_reduce<4, double>(c, CsrHam<XT, float>{x, c->row_ptr, c->col, static_cast<const float *>(c->val), h, R}, R, chunks, st);
            case ISING_F64: return run_reduce<4, double>(c, CsrHam<XT, double>{x, c->row_ptr, c->col, static_cast<const double *>(c->val), h, R}, R, chunks, st);
            default: break;
        }
    }
    return fail(ISING_ERR_UNSUPPORTED, "H monitor: storage form not supported");
}

}  // namespace

ising_status_t energy_reduce(ising_context *c, const void *x, int xtype, int R, int64_t *E_i,
                             int64_t *cut_i, double *E_d, double *cut_d, cudaStream_t st) {
    const int chunks = pick_chunks(c, R);
    const int pairs = c->n_inst * R;
    if (c->integer) {
        ising_status_t s;
        switch (xtype) {
            case ISING_F32: s = energy_typed<float, int64_t>(c, static_cast<const float *>(x), R, chunks, st); break;
            case ISING_F64: s = energy_typed<double, int64_t>(c, static_cast<const double *>(x), R, chunks, st); break;
            case ISING_BF16: s = energy_typed<__nv_bfloat16, int64_t>(c, static_cast<const __nv_bfloat16 *>(x), R, chunks, st); break;
            case ISING_I8: s = energy_typed<int8_t, int64_t>(c, static_cast<const int8_t *>(x), R, chunks, st); break;
            default: return fail(ISING_ERR_INVALID_ARG, "energy: unsupported x type");
        }
        DOCH_CHECK(s);
        energy_finish<int64_t><<<(pairs + 127) / 128, 128, 0, st>>>(c->partials.as<int64_t>(), pairs,
                                                                    chunks, E_i, cut_i, E_d, cut_d);
    } else {
        ising_status_t s;
        switch (xtype) {
            case ISING_F32: s = energy_typed<float, double>(c, static_cast<const float *>(x), R, chunks, st); break;
            case ISING_F64: s = energy_typed<double, double>(c, static_cast<const double *>(x), R, chunks, st); break;
            case ISING_BF16: s = energy_typed<__nv_bfloat16, double>(c, static_cast<const __nv_bfloat16 *>(x), R, chunks, st); break;
            case ISING_I8: s = energy_typed<int8_t, double>(c, static_cast<const int8_t *>(x), R, chunks, st); break;
            default: return fail(ISING_ERR_INVALID_ARG, "energy: unsupported x type");
        }
        DOCH_CHECK(s);
        energy_finish<double><<<(pairs + 127) / 128, 128, 0, st>>>(c->partials.as<double>(), pairs,
                                                                   chunks, nullptr, nullptr, E_d, cut_d);
    }
    DOCH_CUDA(cudaGetLastError());
    return ISING_OK;
}

ising_status_t hamiltonian_reduce(ising_context *c, const void *x, int xtype, int R,
                                  const ParamTabs &p, int k, double *H_out, cudaStream_t st) {
    if (c->format == ISING_FMT_PROCEDURAL) {
        if (xtype != ISING_F32) return fail(ISING_ERR_INVALID_ARG, "PROCEDURAL iterates are F32");
        return proc_hamiltonian(c, static_cast<const float *>(x), R, p, k, H_out, st);
    }
    const int chunks = pick_chunks(c, R);
    ising_status_t s;
    switch (xtype) {
        case ISING_F32: s = ham_typed<float>(c, static_cast<const float *>(x), R, chunks, st); break;
        case ISING_F64: s = ham_typed<double>(c, static_cast<const double *>(x), R, chunks, st); break;
        case ISING_BF16: s = ham_typed<__nv_bfloat16>(c, static_cast<const __nv_bfloat16 *>(x), R, chunks, st); break;
        default: return fail(ISING_ERR_INVALID_ARG, "H monitor: unsupported x type");
    }
    DOCH_CHECK(s);
    const int pairs = c->n_inst * R;
    ham_finish<<<(pairs + 127) / 128, 128, 0, st>>>(c->partials.as<double>(), c->n_inst, R, chunks,
                                                    p.alpha_d, p.alpha_len, k, p.beta_d, H_out);
    DOCH_CUDA(cudaGetLastError());
    return ISING_OK;
}

ising_status_t ham_fused_finish_launch(const double *hpart, int blocks, int R, double alpha, double beta, double *H,
                                       cudaStream_t st) {
    ham_fused_finish<<<(R + 127) / 128, 128, 0, st>>>(hpart, blocks, R, alpha, beta, H);
    DOCH_CUDA(cudaGetLastError());
    return ISING_OK;
}

ising_status_t best_replica(const ising_context *c, const int64_t *E_i, const double *E_d, int R,
                            int32_t *best, cudaStream_t st) {
    best_kernel<<<(c->n_inst + 127) / 128, 128, 0, st>>>(E_i, E_d, c->n_inst, R, best);
    DOCH_CUDA(cudaGetLastError());
    return ISING_OK;
}

ising_status_t write_spins(const ising_context *c, const void *x, int xtype, int R, int8_t *s,
                           cudaStream_t st) {
    const int64_t count = c->n * R;
    int64_t blocks = (count + 255) / 256;
    if (blocks > 16LL * c->num_sms) blocks = 16LL * c->num_sms;
    if (blocks < 1) blocks = 1;
    switch (xtype) {
        case ISING_F32: spins_kernel<<<blocks, 256, 0, st>>>(static_cast<const float *>(x), count, s); break;
        case ISING_F64: spins_kernel<<<blocks, 256, 0, st>>>(static_cast<const double *>(x), count, s); break;
        case ISING_BF16: spins_kernel<<<blocks, 256, 0, st>>>(static_cast<const __nv_bfloat16 *>(x), count, s); break;
        case ISING_I8: spins_kernel<<<blocks, 256, 0, st>>>(static_cast<const int8_t *>(x), count, s); break;
        default: return fail(ISING_ERR_INVALID_ARG, "spins: unsupported x type");
    }
    DOCH_CUDA(cudaGetLastError());
    return ISING_OK;
}

}  // namespace doch
