// C ABI of libising_doch.so: handle lifetime, validation of J and h,
// host/device staging, the parameter rule, and dispatch of the DOCH
// iteration (Algorithm 1) and readout kernels. See include/ising.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "cbrt.cuh"
#include "internal.cuh"

namespace doch {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

ising_status_t fail(ising_status_t s, const std::string &msg) {
    g_err = msg;
    return s;
}

ising_status_t cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? ISING_ERR_OOM : ISING_ERR_CUDA;
}

ising_status_t DevBuf::ensure(size_t want) {
    if (want <= bytes) return ISING_OK;
    release();
    if (want == 0) return ISING_OK;
    cudaError_t e = cudaMalloc(&ptr, want);
    if (e != cudaSuccess) {
        ptr = nullptr;
        bytes = 0;
        cudaGetLastError();
        return cuda_fail(e, "cudaMalloc(scratch)");
    }
    bytes = want;
    return ISING_OK;
}

void DevBuf::release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

namespace {

size_t dtype_size(int t) {
    switch (t) {
        case ISING_I8: case ISING_FP8E4M3: return 1;
        case ISING_I16: case ISING_BF16: return 2;
        case ISING_I32: case ISING_F32: return 4;
        case ISING_F64: return 8;
        default: return 0;
    }
}

bool dtype_integer(int t) { return t == ISING_I8 || t == ISING_I16 || t == ISING_I32; }

// true when the pointer is device (or managed) memory; pinned and pageable
// host memory count as host
bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// copy `bytes` from a host or device pointer into a host vector
ising_status_t to_host(const void *src, size_t bytes, std::vector<unsigned char> &dst) {
    dst.resize(bytes);
    if (bytes == 0) return ISING_OK;
    if (is_device_ptr(src)) {
        DOCH_CUDA(cudaMemcpy(dst.data(), src, bytes, cudaMemcpyDeviceToHost));
    } else {
        std::memcpy(dst.data(), src, bytes);
    }
    return ISING_OK;
}

// FP8 E4M3 (OCP "fn" variant: bias 7, no infinities, S.1111.111 is NaN)
double fp8e4m3_value(uint8_t b) {
    const int e = (b >> 3) & 15, m = b & 7;
    double v;
    if (e == 15 && m == 7) v = NAN;
    else if (e == 0) v = std::ldexp(static_cast<double>(m), -9);
    else v = std::ldexp(1.0 + m / 8.0, e - 7);
    return (b & 0x80) ? -v : v;
}

double value_at(const unsigned char *base, int t, int64_t i) {
    switch (t) {
        case ISING_I8: return reinterpret_cast<const int8_t *>(base)[i];
        case ISING_I16: return reinterpret_cast<const int16_t *>(base)[i];
        case ISING_I32: return reinterpret_cast<const int32_t *>(base)[i];
        case ISING_F32: return reinterpret_cast<const float *>(base)[i];
        case ISING_F64: return reinterpret_cast<const double *>(base)[i];
        case ISING_FP8E4M3: return fp8e4m3_value(base[i]);
        case ISING_BF16: {
            const uint32_t u = static_cast<uint32_t>(reinterpret_cast<const uint16_t *>(base)[i]) << 16;
            float f;
            std::memcpy(&f, &u, 4);
            return f;
        }
        default: return NAN;
    }
}

template <typename T>
ising_status_t upload(T **dst, const void *src, size_t bytes) {
    void *p = nullptr;
    DOCH_CUDA(cudaMalloc(&p, bytes ? bytes : 1));
    *dst = static_cast<T *>(p);
    if (bytes) DOCH_CUDA(cudaMemcpy(p, src, bytes, cudaMemcpyDefault));
    return ISING_OK;
}

// Host view of a problem: J as sorted CSR rows in FP64 (or torus/dense arrays)
struct HostProblem {
    int64_t n = 0;
    int format = 0;
    int jtype = 0;
    int n_inst = 1;
    std::vector<int64_t> off;            // [n_inst + 1]
    std::vector<int64_t> row_ptr;        // CSR
    std::vector<int32_t> col;
    std::vector<double> val;
    std::vector<unsigned char> raw_val;  // CSR values in jtype, sorted order
    std::vector<unsigned char> right, down;  // TORUS2D (int8)
    std::vector<unsigned char> dense;    // DENSE raw jtype
    std::vector<double> h;               // empty when h = 0
    std::vector<unsigned char> raw_h;
    int htype = 0;
    int64_t l_rows = 0, l_cols = 0;
};

ising_status_t load_problem(const ising_problem_t *p, bool validate, HostProblem &hp);

// ELL rows -> CSR on the host (empty slots, col = -1, dropped), then the CSR path
ising_status_t load_ell(const ising_problem_t *p, bool validate, HostProblem &hp) {
    const int64_t n = p->n, w = p->ell_width;
    if (w < 0 || (w > 0 && (!p->col || !p->val))) return fail(ISING_ERR_INVALID_ARG, "ELL arrays are NULL");
    if (p->jtype == ISING_FP8E4M3 || p->jtype == ISING_BF16)
        return fail(ISING_ERR_UNSUPPORTED, "ELL values must be I8/I16/I32/F32/F64");
    const size_t jsz = dtype_size(p->jtype);
    std::vector<unsigned char> col_raw, val_raw;
    DOCH_CHECK(to_host(p->col, sizeof(int32_t) * n * w, col_raw));
    DOCH_CHECK(to_host(p->val, jsz * n * w, val_raw));
    const int32_t *cl = reinterpret_cast<const int32_t *>(col_raw.data());
    std::vector<int64_t> rp(n + 1, 0);
    std::vector<int32_t> col;
    std::vector<unsigned char> val;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t k = 0; k < w; ++k) {
            const int32_t j = cl[i * w + k];
            if (j == -1) continue;
            if (j < 0 || j >= n) return fail(ISING_ERR_INDEX_RANGE, "ELL column out of range in row " + std::to_string(i));
            col.push_back(j);
            val.insert(val.end(), &val_raw[(i * w + k) * jsz], &val_raw[(i * w + k) * jsz] + jsz);
        }
        rp[i + 1] = static_cast<int64_t>(col.size());
    }
    ising_problem_t q = *p;
    q.format = ISING_FMT_CSR;
    q.row_ptr = rp.data();
    q.col = col.data();
    q.val = val.data();
    q.ell_width = 0;
    DOCH_CHECK(load_problem(&q, validate, hp));
    return ISING_OK;
}

ising_status_t load_problem(const ising_problem_t *p, bool validate, HostProblem &hp) {
    if (!p) return fail(ISING_ERR_INVALID_ARG, "problem is NULL");
    if (p->n < 1) return fail(ISING_ERR_INVALID_ARG, "n must be >= 1");
    if (p->format == ISING_FMT_ELL) return load_ell(p, validate, hp);
    hp.n = p->n;
    hp.format = p->format;
    hp.jtype = p->jtype;
    const int64_t n = p->n;
    const size_t jsz = dtype_size(p->jtype);
    if (!jsz) return fail(ISING_ERR_INVALID_ARG, "unknown jtype");
    // instances
    hp.n_inst = p->n_instances > 1 ? p->n_instances : 1;
    if (p->n_instances > 65535) return fail(ISING_ERR_INVALID_ARG, "at most 65535 instances");
    if (hp.n_inst > 1) {
        if (p->format != ISING_FMT_CSR) return fail(ISING_ERR_UNSUPPORTED, "batched instances need CSR");
        if (!p->inst_offset) return fail(ISING_ERR_INVALID_ARG, "inst_offset is NULL");
        std::vector<unsigned char> buf;
        DOCH_CHECK(to_host(p->inst_offset, sizeof(int64_t) * (hp.n_inst + 1), buf));
        hp.off.assign(reinterpret_cast<int64_t *>(buf.data()),
                      reinterpret_cast<int64_t *>(buf.data()) + hp.n_inst + 1);
        if (hp.off[0] != 0 || hp.off[hp.n_inst] != n)
            return fail(ISING_ERR_INVALID_ARG, "inst_offset must run from 0 to n");
        for (int b = 0; b < hp.n_inst; ++b)
            if (hp.off[b + 1] <= hp.off[b]) return fail(ISING_ERR_INVALID_ARG, "empty or decreasing instance");
    } else {
        hp.off = {0, n};
    }
    if (p->format == ISING_FMT_CSR) {
        if (!p->row_ptr || (!p->col && n > 0)) return fail(ISING_ERR_INVALID_ARG, "CSR arrays are NULL");
        if (p->jtype == ISING_FP8E4M3 || p->jtype == ISING_BF16)
            return fail(ISING_ERR_UNSUPPORTED, "CSR values must be I8/I16/I32/F32/F64");
        std::vector<unsigned char> rp_raw;
        DOCH_CHECK(to_host(p->row_ptr, sizeof(int64_t) * (n + 1), rp_raw));
        const int64_t *rp = reinterpret_cast<const int64_t *>(rp_raw.data());
        if (rp[0] != 0) return fail(ISING_ERR_INDEX_RANGE, "row_ptr[0] must be 0");
        for (int64_t i = 0; i < n; ++i)
            if (rp[i + 1] < rp[i]) return fail(ISING_ERR_INDEX_RANGE, "row_ptr is not monotone");
        const int64_t nnz = rp[n];
        if (nnz > 0 && !p->val) return fail(ISING_ERR_INVALID_ARG, "CSR values are NULL");
        std::vector<unsigned char> col_raw, val_raw;
        DOCH_CHECK(to_host(p->col, sizeof(int32_t) * nnz, col_raw));
        DOCH_CHECK(to_host(p->val, jsz * nnz, val_raw));
        const int32_t *cl = reinterpret_cast<const int32_t *>(col_raw.data());
        hp.row_ptr.assign(rp, rp + n + 1);
        hp.col.resize(nnz);
        hp.val.resize(nnz);
        hp.raw_val.resize(jsz * nnz);
        std::vector<int64_t> order;
        int b = 0;
        for (int64_t i = 0; i < n; ++i) {
            while (i >= hp.off[b + 1]) ++b;
            const int64_t e0 = rp[i], e1 = rp[i + 1];
            order.resize(e1 - e0);
            std::iota(order.begin(), order.end(), e0);
            std::sort(order.begin(), order.end(), [&](int64_t a, int64_t c) { return cl[a] < cl[c]; });
            for (int64_t k = 0; k < e1 - e0; ++k) {
                const int64_t e = order[k];
                const int32_t j = cl[e];
                // index checks always run: a bad column would make the kernels read out of bounds
                if (j < hp.off[b] || j >= hp.off[b + 1])
                    return fail(ISING_ERR_INDEX_RANGE, "column index out of range in row " + std::to_string(i));
                if (k > 0 && cl[order[k - 1]] == j)
                    return fail(ISING_ERR_INVALID_ARG, "duplicate column in row " + std::to_string(i));
                hp.col[e0 + k] = j;
                hp.val[e0 + k] = value_at(val_raw.data(), p->jtype, e);
                std::memcpy(&hp.raw_val[(e0 + k) * jsz], &val_raw[e * jsz], jsz);
                if (validate) {
                    if (!std::isfinite(hp.val[e0 + k]))
                        return fail(ISING_ERR_NONFINITE, "non-finite coupling in row " + std::to_string(i));
                    if (j == i && hp.val[e0 + k] != 0.0)
                        return fail(ISING_ERR_NONZERO_DIAG, "J_ii != 0 at i = " + std::to_string(i));
                }
            }
        }
        if (validate) {
            for (int64_t i = 0; i < n; ++i)
                for (int64_t e = hp.row_ptr[i]; e < hp.row_ptr[i + 1]; ++e) {
                    const int64_t j = hp.col[e];
                    const auto beg = hp.col.begin() + hp.row_ptr[j], end = hp.col.begin() + hp.row_ptr[j + 1];
                    const auto it = std::lower_bound(beg, end, static_cast<int32_t>(i));
                    const double back = (it != end && *it == i) ? hp.val[it - hp.col.begin()] : 0.0;
                    if (back != hp.val[e])
                        return fail(ISING_ERR_NOT_SYMMETRIC, "J_ij != J_ji at (" + std::to_string(i) + ", " + std::to_string(j) + ")");
                }
        }
    } else if (p->format == ISING_FMT_TORUS2D) {
        if (p->jtype != ISING_I8) return fail(ISING_ERR_UNSUPPORTED, "TORUS2D couplings must be I8");
        if (p->l_rows < 2 || p->l_cols < 2 || p->l_rows * p->l_cols != n)
            return fail(ISING_ERR_INVALID_ARG, "TORUS2D needs l_rows, l_cols >= 2 and n = l_rows * l_cols");
        if (!p->right || !p->down) return fail(ISING_ERR_INVALID_ARG, "TORUS2D arrays are NULL");
        if (p->h) return fail(ISING_ERR_UNSUPPORTED, "TORUS2D takes no field");
        hp.l_rows = p->l_rows;
        hp.l_cols = p->l_cols;
        DOCH_CHECK(to_host(p->right, n, hp.right));
        DOCH_CHECK(to_host(p->down, n, hp.down));
    } else if (p->format == ISING_FMT_DENSE) {
        if (!p->dense) return fail(ISING_ERR_INVALID_ARG, "dense array is NULL");
        DOCH_CHECK(to_host(p->dense, jsz * n * n, hp.dense));
        // the storage (2-bit codes or BF16) is exact only for integers of magnitude <= 256: checked
        // for every type, with or without validation
        for (int64_t e = 0; e < n * n; ++e) {
            const double v = value_at(hp.dense.data(), p->jtype, e);
            if (!(std::fabs(v) <= 256.0) || v != std::floor(v))
                return fail(ISING_ERR_UNSUPPORTED,
                            "DENSE couplings must be integers with |J_ij| <= 256 (held exactly in BF16)");
        }
        if (validate) {
            for (int64_t i = 0; i < n; ++i) {
                if (value_at(hp.dense.data(), p->jtype, i * n + i) != 0.0)
                    return fail(ISING_ERR_NONZERO_DIAG, "J_ii != 0 at i = " + std::to_string(i));
                for (int64_t j = i + 1; j < n; ++j) {
                    const double a = value_at(hp.dense.data(), p->jtype, i * n + j);
                    const double c = value_at(hp.dense.data(), p->jtype, j * n + i);
                    if (std::fabs(a) > 256.0)
                        return fail(ISING_ERR_UNSUPPORTED, "DENSE couplings must satisfy |J_ij| <= 256 (exact in BF16)");
                    if (!std::isfinite(a)) return fail(ISING_ERR_NONFINITE, "non-finite coupling");
                    if (a != c) return fail(ISING_ERR_NOT_SYMMETRIC, "J_ij != J_ji");
                }
            }
        }
    } else {
        return fail(ISING_ERR_INVALID_ARG, "unknown format");
    }
    if (p->h) {
        const size_t hsz = dtype_size(p->htype);
        if (!hsz || p->htype == ISING_FP8E4M3 || p->htype == ISING_BF16)
            return fail(ISING_ERR_INVALID_ARG, "htype must be I8/I16/I32/F32/F64");
        hp.htype = p->htype;
        DOCH_CHECK(to_host(p->h, hsz * n, hp.raw_h));
        hp.h.resize(n);
        for (int64_t i = 0; i < n; ++i) {
            hp.h[i] = value_at(hp.raw_h.data(), p->htype, i);
            if (validate && !std::isfinite(hp.h[i])) return fail(ISING_ERR_NONFINITE, "non-finite field");
        }
    }
    return ISING_OK;
}

// y = J v for one instance [lo, hi) of a host problem (FP64), for the power method
void host_matvec(const HostProblem &hp, int64_t lo, int64_t hi, const std::vector<double> &v,
                 std::vector<double> &y) {
    const int64_t m = hi - lo;
    std::fill(y.begin(), y.end(), 0.0);
    if (hp.format == ISING_FMT_CSR) {
        for (int64_t i = lo; i < hi; ++i) {
            double s = 0.0;
            for (int64_t e = hp.row_ptr[i]; e < hp.row_ptr[i + 1]; ++e) s += hp.val[e] * v[hp.col[e] - lo];
            y[i - lo] = s;
        }
    } else if (hp.format == ISING_FMT_TORUS2D) {
        const int64_t Lr = hp.l_rows, Lc = hp.l_cols;
        for (int64_t r = 0; r < Lr; ++r)
            for (int64_t c = 0; c < Lc; ++c) {
                const int64_t a = r * Lc + c, br = r * Lc + (c + 1) % Lc, bd = ((r + 1) % Lr) * Lc + c;
                const double wr = static_cast<int8_t>(hp.right[a]), wd = static_cast<int8_t>(hp.down[a]);
                y[a] += wr * v[br]; y[br] += wr * v[a];
                y[a] += wd * v[bd]; y[bd] += wd * v[a];
            }
    } else {
        for (int64_t i = 0; i < m; ++i) {
            double s = 0.0;
            for (int64_t j = 0; j < m; ++j) s += value_at(hp.dense.data(), hp.jtype, i * m + j) * v[j];
            y[i] = s;
        }
    }
}

// per-instance sums: off-diagonal sum, sum of squares, max row |J| sum
void host_stats(const HostProblem &hp, int64_t lo, int64_t hi, double &s1, double &s2, double &rowmax) {
    s1 = s2 = rowmax = 0.0;
    if (hp.format == ISING_FMT_CSR) {
        for (int64_t i = lo; i < hi; ++i) {
            double ra = 0.0;
            for (int64_t e = hp.row_ptr[i]; e < hp.row_ptr[i + 1]; ++e) {
                s1 += hp.val[e]; s2 += hp.val[e] * hp.val[e]; ra += std::fabs(hp.val[e]);
            }
            rowmax = std::max(rowmax, ra);
        }
    } else if (hp.format == ISING_FMT_TORUS2D) {
        const int64_t Lr = hp.l_rows, Lc = hp.l_cols;
        for (int64_t r = 0; r < Lr; ++r)
            for (int64_t c = 0; c < Lc; ++c) {
                const int64_t a = r * Lc + c;
                const double wr = static_cast<int8_t>(hp.right[a]), wd = static_cast<int8_t>(hp.down[a]);
                s1 += 2 * (wr + wd); s2 += 2 * (wr * wr + wd * wd);
                const double wl = static_cast<int8_t>(hp.right[r * Lc + (c + Lc - 1) % Lc]);
                const double wu = static_cast<int8_t>(hp.down[((r + Lr - 1) % Lr) * Lc + c]);
                rowmax = std::max(rowmax, std::fabs(wr) + std::fabs(wd) + std::fabs(wl) + std::fabs(wu));
            }
    } else {
        const int64_t m = hi - lo;
        for (int64_t i = 0; i < m; ++i) {
            double ra = 0.0;
            for (int64_t j = 0; j < m; ++j) {
                const double w = value_at(hp.dense.data(), hp.jtype, i * m + j);
                s1 += w; s2 += w * w; ra += std::fabs(w);
            }
            rowmax = std::max(rowmax, ra);
        }
    }
}

// lambda_max(-J) by power iteration on M = -J + sigma I, sigma = ||J||_inf
double power_lambda_neg(const HostProblem &hp, int64_t lo, int64_t hi, double sigma) {
    const int64_t m = hi - lo;
    std::vector<double> v(m), y(m);
    uint64_t s = 0x9E3779B97F4A7C15ull ^ static_cast<uint64_t>(lo);
    for (int64_t i = 0; i < m; ++i) {  // deterministic start (xorshift)
        s ^= s << 13; s ^= s >> 7; s ^= s << 17;
        v[i] = static_cast<double>(s >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    }
    double nv = 0.0;
    for (double t : v) nv += t * t;
    nv = std::sqrt(nv);
    for (double &t : v) t /= nv;
    double lam = 0.0, prev = -1.0;
    for (int it = 0; it < 20000; ++it) {
        host_matvec(hp, lo, hi, v, y);
        double rq = 0.0, ny = 0.0;
        for (int64_t i = 0; i < m; ++i) {
            y[i] = -y[i] + sigma * v[i];
            rq += v[i] * y[i];
            ny += y[i] * y[i];
        }
        lam = rq;
        ny = std::sqrt(ny);
        if (ny == 0.0) break;
        for (int64_t i = 0; i < m; ++i) v[i] = y[i] / ny;
        if (it > 10 && std::fabs(lam - prev) <= 1e-13 * std::fabs(lam)) break;
        prev = lam;
    }
    return lam - sigma;
}

ising_status_t finish(ising_context *c, cudaStream_t st, bool must_sync) {
    if (!must_sync && (c->flags & ISING_FLAG_ASYNC)) return ISING_OK;
    DOCH_CUDA(cudaMemcpyAsync(c->err_host, c->err_word, sizeof(int), cudaMemcpyDeviceToHost, st));
    DOCH_CUDA(cudaStreamSynchronize(st));
    if (*c->err_host) {
        const int w = *c->err_host;
        *c->err_host = 0;
        cudaMemsetAsync(c->err_word, 0, sizeof(int), st);
        cudaStreamSynchronize(st);
        if (w & DEV_ERR_TIMEOUT) return fail(ISING_ERR_TIMEOUT, "a bounded device-side wait ran out");
    }
    return ISING_OK;
}

void destroy_ctx(ising_context *c) {
    if (!c) return;
    c->tune.release();
    cudaFree(c->inst_off);
    cudaFree(c->row_ptr);
    cudaFree(c->col);
    cudaFree(c->val);
    cudaFree(c->right);
    cudaFree(c->down);
    cudaFree(c->dense);
    cudaFree(c->h_f32);
    cudaFree(c->h_f64);
    cudaFree(c->h_i64);
    cudaFree(c->err_word);
    if (c->err_host) cudaFreeHost(c->err_host);
    if (c->count_host) cudaFreeHost(c->count_host);
    cudaFree(c->batch_order);
    cudaFree(c->ell_col);
    cudaFree(c->ell_val);
    cudaFree(c->ell_off);
    cudaFree(c->batch_queue);
    if (c->batch_exec) cudaGraphExecDestroy(c->batch_exec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    c->ping.release();
    c->stage_x.release();
    c->stage_out.release();
    c->partials.release();
    c->params.release();
    c->ckpt.release();
    c->work.release();
    c->res_items[0].buf.release();
    c->res_items[1].buf.release();
    c->res_scratch.release();
    c->proc_units.release();
    c->proc_acc.release();
    c->proc_u.release();
    delete c;
}

ising_status_t build_context(const HostProblem &hp, int flags, ising_context *c) {
    DOCH_CUDA(cudaGetDevice(&c->device));
    DOCH_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
    c->flags = flags;
    c->format = hp.format;
    c->jtype = hp.jtype;
    c->n = hp.n;
    c->n_inst = hp.n_inst;
    c->inst_off_h = hp.off;
    c->max_inst_n = 0;
    for (int b = 0; b < hp.n_inst; ++b) c->max_inst_n = std::max(c->max_inst_n, hp.off[b + 1] - hp.off[b]);
    c->has_h = !hp.h.empty();
    // DENSE values are integers whatever their storage type (checked on load)
    c->integer = (dtype_integer(hp.jtype) || hp.format == ISING_FMT_DENSE) && (!c->has_h || dtype_integer(hp.htype));
    DOCH_CHECK(upload(&c->inst_off, hp.off.data(), sizeof(int64_t) * hp.off.size()));
    if (hp.format == ISING_FMT_CSR && hp.n_inst > 1) {
        // longest-first queue order for the persistent batched kernel
        std::vector<int64_t> work(hp.n_inst);
        for (int b = 0; b < hp.n_inst; ++b)
            work[b] = (hp.off[b + 1] - hp.off[b]) + (hp.row_ptr[hp.off[b + 1]] - hp.row_ptr[hp.off[b]]);
        c->inst_nnz_h.resize(hp.n_inst);
        for (int b = 0; b < hp.n_inst; ++b) c->inst_nnz_h[b] = hp.row_ptr[hp.off[b + 1]] - hp.row_ptr[hp.off[b]];
        std::vector<int32_t> order(hp.n_inst);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return work[a] > work[b]; });
        DOCH_CHECK(upload(&c->batch_order, order.data(), sizeof(int32_t) * order.size()));
        void *qp = nullptr;
        DOCH_CUDA(cudaMalloc(&qp, sizeof(int)));
        c->batch_queue = static_cast<int *>(qp);
    }
    if (hp.format == ISING_FMT_CSR) {
        c->nnz = hp.row_ptr.back();
        for (int64_t i = 0; i < hp.n; ++i)
            c->max_row_nnz = std::max(c->max_row_nnz, hp.row_ptr[i + 1] - hp.row_ptr[i]);
        DOCH_CHECK(upload(&c->row_ptr, hp.row_ptr.data(), sizeof(int64_t) * hp.row_ptr.size()));
        DOCH_CHECK(upload(&c->col, hp.col.data(), sizeof(int32_t) * hp.col.size()));
        if (hp.n_inst > 1 && c->max_inst_n <= 65536) {
            // transposed ELL copy for the shared-memory resident batched kernel, in slot
            // pairs: slots 2p and 2p + 1 of row i sit side by side at pair p, row i
            // ([pair][row][2]), so one 4-byte load gives a row two columns and one 8-byte
            // load two weights. Slots past a row's entries (and the one that makes the
            // width even) hold the row itself with weight 0.
            std::vector<int64_t> eoff(hp.n_inst + 1, 0);
            c->ell_deg_h.assign(hp.n_inst, 0);
            for (int b = 0; b < hp.n_inst; ++b) {
                int d = 0;
                for (int64_t i = hp.off[b]; i < hp.off[b + 1]; ++i)
                    d = std::max<int>(d, static_cast<int>(hp.row_ptr[i + 1] - hp.row_ptr[i]));
                d += d & 1;
                c->ell_deg_h[b] = d;
                eoff[b + 1] = eoff[b] + static_cast<int64_t>(d) * (hp.off[b + 1] - hp.off[b]);
            }
            std::vector<uint16_t> ec(eoff.back());
            std::vector<float> ev(eoff.back());
            for (int b = 0; b < hp.n_inst; ++b) {
                const int64_t lo = hp.off[b], nb = hp.off[b + 1] - lo;
                for (int64_t i = 0; i < nb; ++i) {
                    const int64_t e0 = hp.row_ptr[lo + i], cnt = hp.row_ptr[lo + i + 1] - e0;
                    for (int k = 0; k < c->ell_deg_h[b]; ++k) {
                        const size_t at = static_cast<size_t>(eoff[b] + ((k >> 1) * nb + i) * 2 + (k & 1));
                        ec[at] = static_cast<uint16_t>(k < cnt ? hp.col[e0 + k] - lo : i);
                        ev[at] = k < cnt ? static_cast<float>(hp.val[e0 + k]) : 0.f;
                    }
                }
            }
            DOCH_CHECK(upload(&c->ell_col, ec.data(), sizeof(uint16_t) * ec.size()));
            DOCH_CHECK(upload(&c->ell_val, ev.data(), sizeof(float) * ev.size()));
            DOCH_CHECK(upload(&c->ell_off, eoff.data(), sizeof(int64_t) * eoff.size()));
        }
        if (hp.jtype == ISING_I16) {  // held as I32 on the device
            std::vector<int32_t> v(hp.val.size());
            for (size_t e = 0; e < v.size(); ++e) v[e] = static_cast<int32_t>(hp.val[e]);
            DOCH_CHECK(upload(&c->val, v.data(), sizeof(int32_t) * v.size()));
            c->jtype = ISING_I32;
        } else {
            DOCH_CHECK(upload(&c->val, hp.raw_val.data(), hp.raw_val.size()));
        }
    } else if (hp.format == ISING_FMT_TORUS2D) {
        c->l_rows = hp.l_rows;
        c->l_cols = hp.l_cols;
        DOCH_CHECK(upload(&c->right, hp.right.data(), hp.right.size()));
        DOCH_CHECK(upload(&c->down, hp.down.data(), hp.down.size()));
    } else {
        // Tensor-core tile order [row tile of 128][K block of 64][128][64], zero padded. Entries
        // all in {-1, 0, +1}: packed 2-bit codes (2 KB per tile, expanded on chip); otherwise a
        // BF16 copy, each 16 KB block 128-byte swizzled (chunk c of row r at c ^ (r & 7)).
        const int64_t n = hp.n, ld = (n + 63) / 64 * 64, mt = (n + 127) / 128, kbs = ld / 64;
        bool ternary = true;
        for (int64_t e = 0; e < n * n && ternary; ++e) {
            const double v = value_at(hp.dense.data(), hp.jtype, e);
            ternary = v == 0.0 || v == 1.0 || v == -1.0;
        }
        long long jsum = 0;
        if (ternary) {
            std::vector<uint8_t> packed(static_cast<size_t>(mt) * kbs * 2048, 0);
            for (int64_t i = 0; i < n; ++i) {
                const int64_t ti = i / 128, ri = i % 128;
                for (int64_t j = 0; j < n; ++j) {
                    const double v = value_at(hp.dense.data(), hp.jtype, i * n + j);
                    const int64_t kb = j / 64, cc = j % 64;
                    const uint8_t code = v > 0 ? 1 : (v < 0 ? 2 : 0);
                    packed[static_cast<size_t>((ti * kbs + kb) * 2048 + ri * 16 + cc / 4)] |=
                        static_cast<uint8_t>(code << (2 * (cc % 4)));
                    jsum += static_cast<long long>(v);
                }
            }
            DOCH_CHECK(upload(&c->dense, packed.data(), packed.size()));
            c->dense_ternary = true;
            c->dense_type = ISING_I8;
            c->dense_ld = ld;
            c->dense_jsum = jsum;
        }
        std::vector<uint16_t> bf(ternary ? 0 : static_cast<size_t>(mt) * 128 * ld, 0);
        for (int64_t i = 0; i < (ternary ? 0 : n); ++i) {
            const int64_t ti = i / 128, ri = i % 128;
            for (int64_t j = 0; j < n; ++j) {
                const double v = value_at(hp.dense.data(), hp.jtype, i * n + j);
                float f = static_cast<float>(v);
                uint32_t u;
                std::memcpy(&u, &f, 4);
                const int64_t kb = j / 64, cc = j % 64;
                const size_t off = static_cast<size_t>(((ti * kbs + kb) * 128 + ri) * 64 +
                                                       ((((cc >> 3) ^ ri) & 7) << 3) + (cc & 7));
                bf[off] = static_cast<uint16_t>(u >> 16);  // exact: |v| <= 256 integer
                jsum += static_cast<long long>(v);
            }
        }
        if (!ternary) {
            DOCH_CHECK(upload(&c->dense, bf.data(), bf.size() * 2));
            c->dense_type = ISING_BF16;
            c->dense_ld = ld;
            c->dense_jsum = jsum;
        }
    }
    if (c->has_h) {
        std::vector<float> hf(hp.n);
        for (int64_t i = 0; i < hp.n; ++i) hf[i] = static_cast<float>(hp.h[i]);
        DOCH_CHECK(upload(&c->h_f32, hf.data(), sizeof(float) * hp.n));
        DOCH_CHECK(upload(&c->h_f64, hp.h.data(), sizeof(double) * hp.n));
        if (dtype_integer(hp.htype)) {
            std::vector<int64_t> hi(hp.n);
            for (int64_t i = 0; i < hp.n; ++i) hi[i] = static_cast<int64_t>(hp.h[i]);
            DOCH_CHECK(upload(&c->h_i64, hi.data(), sizeof(int64_t) * hp.n));
        }
    }
    void *ew = nullptr;
    DOCH_CUDA(cudaMalloc(&ew, sizeof(int)));
    c->err_word = static_cast<int *>(ew);
    DOCH_CUDA(cudaMemset(c->err_word, 0, sizeof(int)));
    void *eh = nullptr;
    DOCH_CUDA(cudaMallocHost(&eh, sizeof(int)));
    c->err_host = static_cast<int *>(eh);
    *c->err_host = 0;
    return ISING_OK;
}

size_t xtype_size(int t) { return dtype_size(t); }

// upload the per-instance parameter tables and return views of them
ising_status_t upload_params(ising_context *c, const double *alpha, int alpha_len, const double *beta,
                             ParamTabs &out, cudaStream_t st) {
    const int ni = c->n_inst;
    const size_t na = static_cast<size_t>(ni) * alpha_len;
    std::vector<double> a(na), b(ni);
    std::vector<unsigned char> tmp;
    DOCH_CHECK(to_host(alpha, sizeof(double) * na, tmp));
    std::memcpy(a.data(), tmp.data(), sizeof(double) * na);
    DOCH_CHECK(to_host(beta, sizeof(double) * ni, tmp));
    std::memcpy(b.data(), tmp.data(), sizeof(double) * ni);
    for (double v : a) if (!std::isfinite(v)) return fail(ISING_ERR_NONFINITE, "alpha is not finite");
    for (double v : b) {
        if (!std::isfinite(v)) return fail(ISING_ERR_NONFINITE, "beta is not finite");
        if (v <= 0.0) return fail(ISING_ERR_INVALID_ARG, "beta must be > 0");
    }
    // layout: alpha_d | beta_d | alpha_f | inv_beta_f | zscale_f | xscale_f (each 256-byte aligned)
    auto al = [](size_t v) { return (v + 255) & ~static_cast<size_t>(255); };
    const size_t o1 = al(na * 8), o2 = o1 + al(ni * 8), o3 = o2 + al(na * 4), o4 = o3 + al(ni * 4),
                 o5 = o4 + al(ni * 4), tot = o5 + al(ni * 4);
    std::vector<unsigned char> host(tot);
    std::memcpy(host.data(), a.data(), na * 8);
    std::memcpy(host.data() + o1, b.data(), ni * 8);
    for (size_t i = 0; i < na; ++i) reinterpret_cast<float *>(host.data() + o2)[i] = static_cast<float>(a[i]);
    for (int i = 0; i < ni; ++i) {
        const double ib = 1.0 / b[i];
        const int k = cbrt_prescale_exp(ib);
        reinterpret_cast<float *>(host.data() + o3)[i] = static_cast<float>(ib);
        reinterpret_cast<float *>(host.data() + o4)[i] = static_cast<float>(std::ldexp(ib, 3 * k));
        reinterpret_cast<float *>(host.data() + o5)[i] = std::ldexp(1.0f, -k);
    }
    DOCH_CHECK(c->params.ensure(tot));
    DOCH_CUDA(cudaMemcpyAsync(c->params.ptr, host.data(), tot, cudaMemcpyHostToDevice, st));
    // the source is pageable: make sure the copy has consumed it
    DOCH_CUDA(cudaStreamSynchronize(st));
    unsigned char *base = c->params.as<unsigned char>();
    out.alpha_d = reinterpret_cast<const double *>(base);
    out.beta_d = reinterpret_cast<const double *>(base + o1);
    out.alpha_f = reinterpret_cast<const float *>(base + o2);
    out.inv_beta_f = reinterpret_cast<const float *>(base + o3);
    out.zscale_f = reinterpret_cast<const float *>(base + o4);
    out.xscale_f = reinterpret_cast<const float *>(base + o5);
    out.alpha_len = alpha_len;
    return ISING_OK;
}

// one DOCH step of the handle's storage form
ising_status_t step(ising_context *c, const void *xi, void *xo, int xtype, int R, const ParamTabs &p,
                    const std::vector<double> &alpha_h, const std::vector<double> &beta_h, int k,
                    cudaStream_t st) {
    if (c->format == ISING_FMT_TORUS2D) {
        const double a = alpha_h[p.alpha_len == 1 ? 0 : k];
        if (xtype == ISING_F32)
            return torus_step_f32(c, static_cast<const float *>(xi), static_cast<float *>(xo), R,
                                  static_cast<float>(a), 1.0 / beta_h[0], st);
        return torus_step_f64(c, static_cast<const double *>(xi), static_cast<double *>(xo), R, a,
                              beta_h[0], st);
    }
    if (c->format == ISING_FMT_CSR) return csr_step(c, xi, xo, xtype, R, p, k, st);
    if (c->format == ISING_FMT_PROCEDURAL)
        return proc_step(c, static_cast<const float *>(xi), static_cast<float *>(xo), R,
                         alpha_h[p.alpha_len == 1 ? 0 : k], 1.0 / beta_h[0], st);
    return fail(ISING_ERR_UNSUPPORTED, "this storage form has no iteration kernel yet");
}


// Autotuner for the batched persistent kernel: times each candidate shape for
// a few steps on scratch copies of x and keeps the fastest, per R.
ising_status_t tune_batched(ising_context *c, const float *x, int R, const ParamTabs &p, cudaStream_t st,
                            BatchedConfig *out) {
    auto it = c->batch_tuned.find(R);
    if (it != c->batch_tuned.end()) {
        *out = it->second;
        return ISING_OK;
    }
    const size_t xbytes = static_cast<size_t>(c->n) * R * sizeof(float);
    DOCH_CHECK(c->work.ensure(2 * xbytes));
    float *ta = c->work.as<float>();
    float *tb = reinterpret_cast<float *>(c->work.as<unsigned char>() + xbytes);
    std::vector<BatchedConfig> cand;
    for (int threads : {256, 512, 1024})
        for (int vec : {4, 2, 1}) {
            if (R % vec) continue;
            for (int cps : {1, 2, 4}) {
                if (threads * cps > 2048) continue;
                BatchedConfig k;
                k.threads = threads;
                k.vec = vec;
                k.ctas_per_sm = cps;
                cand.push_back(k);
            }
        }
    cudaEvent_t e0, e1;
    DOCH_CUDA(cudaEventCreate(&e0));
    DOCH_CUDA(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    BatchedConfig best = cand.front();
    const int probe = 8;
    bool any = false;
    for (const BatchedConfig &k : cand) {
        DOCH_CUDA(cudaMemcpyAsync(ta, x, xbytes, cudaMemcpyDeviceToDevice, st));
        const ising_status_t ws = batched_launch(c, k, ta, tb, R, p, 2, st);  // warm-up
        if (ws == ISING_ERR_UNSUPPORTED) continue;                              // shape not launchable
        DOCH_CHECK(ws);
        any = true;
        DOCH_CUDA(cudaEventRecord(e0, st));
        DOCH_CHECK(batched_launch(c, k, ta, tb, R, p, probe, st));
        DOCH_CUDA(cudaEventRecord(e1, st));
        DOCH_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        DOCH_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best_ms) {
            best_ms = ms;
            best = k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!any) return fail(ISING_ERR_CUDA, "batched: no launchable shape");
    g_err.clear();
    c->batch_tuned[R] = best;
    *out = best;
    return ISING_OK;
}

// Autotuner for the shared-memory resident kernel: times each variant (threads
// per CTA; one or two iterate copies in shared memory) for a few steps on a
// scratch copy of x and keeps the fastest, per R.
ising_status_t tune_resident(ising_context *c, const float *x, int R, const ParamTabs &p, cudaStream_t st,
                             ResidentConfig *out) {
    auto it = c->res_tuned.find(R);
    if (it != c->res_tuned.end()) {
        *out = it->second;
        return ISING_OK;
    }
    // ISING_RESIDENT_VARIANT=<threads>:<copies> (512 or 1024 : 1 or 2) fixes the variant
    // instead of timing the candidates (to test each variant)
    if (const char *env = std::getenv("ISING_RESIDENT_VARIANT")) {
        int t = 0, cp = 0;
        if (std::sscanf(env, "%d:%d", &t, &cp) == 2 && (t == 512 || t == 1024) && (cp == 1 || cp == 2)) {
            ResidentConfig k;
            k.threads = t;
            k.one_copy = cp == 1;
            DOCH_CHECK(resident_items(c, R, k.one_copy));
            c->res_tuned[R] = k;
            *out = k;
            return ISING_OK;
        }
    }
    const size_t xbytes = static_cast<size_t>(c->n) * R * sizeof(float);
    DOCH_CHECK(c->work.ensure(xbytes));
    float *tx = c->work.as<float>();
    cudaEvent_t e0, e1;
    DOCH_CUDA(cudaEventCreate(&e0));
    DOCH_CUDA(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    ResidentConfig best;
    bool any = false;
    const int probe = 16;
    for (int threads : {1024, 512})
        for (bool one : {false, true}) {
            ResidentConfig k;
            k.threads = threads;
            k.one_copy = one;
            DOCH_CUDA(cudaMemcpyAsync(tx, x, xbytes, cudaMemcpyDeviceToDevice, st));
            const ising_status_t ws = batched_resident_launch(c, k, tx, R, p, 2, st);  // warm-up
            if (ws == ISING_ERR_UNSUPPORTED) continue;
            DOCH_CHECK(ws);
            any = true;
            DOCH_CUDA(cudaEventRecord(e0, st));
            DOCH_CHECK(batched_resident_launch(c, k, tx, R, p, probe, st));
            DOCH_CUDA(cudaEventRecord(e1, st));
            DOCH_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            DOCH_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best_ms) {
                best_ms = ms;
                best = k;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!any) return ISING_ERR_UNSUPPORTED;
    g_err.clear();
    c->res_tuned[R] = best;
    *out = best;
    return ISING_OK;
}

// capture `launch` (enqueued on the handle's capture stream) into the handle's
// graph unless the graph for `key` exists, then replay it on st
template <typename F>
ising_status_t graph_replay(ising_context *c, const std::vector<uintptr_t> &key, F &&launch, cudaStream_t st) {
    if (!c->batch_exec || c->batch_key != key) {
        if (c->batch_exec) {
            cudaGraphExecDestroy(c->batch_exec);
            c->batch_exec = nullptr;
        }
        if (!c->cap_stream) DOCH_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        DOCH_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        const ising_status_t s = launch(c->cap_stream);
        cudaGraph_t graph = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &graph);
        if (s != ISING_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        DOCH_CUDA(ee);
        const cudaError_t ei = cudaGraphInstantiate(&c->batch_exec, graph, 0);
        cudaGraphDestroy(graph);
        DOCH_CUDA(ei);
        c->batch_key = key;
    }
    DOCH_CUDA(cudaGraphLaunch(c->batch_exec, st));
    return ISING_OK;
}

// All steps of all instances: one persistent launch, captured once into a
// CUDA graph (queue reset + kernel [+ copy back]) and replayed while the
// buffers, parameters and shape stay the same.
ising_status_t batched_iterate(ising_context *c, float *x, int R, const ParamTabs &p, int iters,
                               cudaStream_t st) {
    // every (instance, replica group) resident in shared memory when they fit
    if (batched_resident_ok(c, x, R)) {
        ResidentConfig rc;
        DOCH_CHECK(tune_resident(c, x, R, p, st, &rc));
        DOCH_CHECK(resident_items(c, R, rc.one_copy));   // built here, never inside the capture
        if (rc.one_copy) DOCH_CHECK(c->res_scratch.ensure(static_cast<size_t>(c->n) * R * sizeof(float)));
        const ResidentItems &its = c->res_items[rc.one_copy ? 1 : 0];
        const std::vector<uintptr_t> key = {1, static_cast<uintptr_t>(its.gen), reinterpret_cast<uintptr_t>(x),
                                            static_cast<uintptr_t>(R),
                                            static_cast<uintptr_t>(iters), static_cast<uintptr_t>(p.alpha_len),
                                            reinterpret_cast<uintptr_t>(p.alpha_f),
                                            reinterpret_cast<uintptr_t>(p.zscale_f),
                                            reinterpret_cast<uintptr_t>(p.xscale_f),
                                            static_cast<uintptr_t>(rc.threads), static_cast<uintptr_t>(rc.one_copy),
                                            reinterpret_cast<uintptr_t>(its.buf.ptr),
                                            reinterpret_cast<uintptr_t>(c->res_scratch.ptr)};
        return graph_replay(c, key, [&](cudaStream_t cs) { return batched_resident_launch(c, rc, x, R, p, iters, cs); },
                            st);
    }
    BatchedConfig cfg;
    DOCH_CHECK(tune_batched(c, x, R, p, st, &cfg));
    const size_t xbytes = static_cast<size_t>(c->n) * R * sizeof(float);
    DOCH_CHECK(c->ping.ensure(xbytes));
    float *xb = c->ping.as<float>();
    const std::vector<uintptr_t> key = {2, reinterpret_cast<uintptr_t>(x), reinterpret_cast<uintptr_t>(xb),
                                        static_cast<uintptr_t>(R), static_cast<uintptr_t>(iters),
                                        static_cast<uintptr_t>(p.alpha_len), reinterpret_cast<uintptr_t>(p.alpha_f),
                                        reinterpret_cast<uintptr_t>(p.inv_beta_f), static_cast<uintptr_t>(cfg.threads),
                                        static_cast<uintptr_t>(cfg.vec), static_cast<uintptr_t>(cfg.ctas_per_sm)};
    if (!c->batch_exec || c->batch_key != key) {
        if (c->batch_exec) {
            cudaGraphExecDestroy(c->batch_exec);
            c->batch_exec = nullptr;
        }
        if (!c->cap_stream) DOCH_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        DOCH_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        ising_status_t s = batched_launch(c, cfg, x, xb, R, p, iters, c->cap_stream);
        if (s == ISING_OK && (iters & 1)) {
            const cudaError_t e = cudaMemcpyAsync(x, xb, xbytes, cudaMemcpyDeviceToDevice, c->cap_stream);
            if (e != cudaSuccess) s = cuda_fail(e, "cudaMemcpyAsync (capture)");
        }
        cudaGraph_t graph = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &graph);
        if (s != ISING_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        DOCH_CUDA(ee);
        const cudaError_t ei = cudaGraphInstantiate(&c->batch_exec, graph, 0);
        cudaGraphDestroy(graph);
        DOCH_CUDA(ei);
        c->batch_key = key;
    }
    DOCH_CUDA(cudaGraphLaunch(c->batch_exec, st));
    return ISING_OK;
}

}  // namespace
}  // namespace doch

using namespace doch;

extern "C" {

const char *ising_status_string(ising_status_t s) {
    switch (s) {
        case ISING_OK: return "ok";
        case ISING_ERR_INVALID_ARG: return "invalid argument";
        case ISING_ERR_NOT_SYMMETRIC: return "coupling matrix is not symmetric";
        case ISING_ERR_NONZERO_DIAG: return "coupling matrix has a nonzero diagonal";
        case ISING_ERR_INDEX_RANGE: return "index out of range";
        case ISING_ERR_NONFINITE: return "non-finite value";
        case ISING_ERR_OOM: return "out of device memory";
        case ISING_ERR_CUDA: return "CUDA error";
        case ISING_ERR_TIMEOUT: return "device-side wait timed out";
        case ISING_ERR_NOT_MONOTONE: return "Hamiltonian increased";
        case ISING_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char *ising_last_error(void) { return g_err.c_str(); }

ising_status_t ising_default_params(const ising_problem_t *p, double eta, int32_t method,
                                    double *alpha_out, double *beta_out) {
    return doch::guarded([&]() -> ising_status_t {
        g_err.clear();
        if (!alpha_out || !beta_out) return fail(ISING_ERR_INVALID_ARG, "output pointers are NULL");
        if (!(eta > 0.0) || !std::isfinite(eta)) return fail(ISING_ERR_INVALID_ARG, "eta must be > 0");
        if (method < 0 || method > 2) return fail(ISING_ERR_INVALID_ARG, "method must be 0, 1 or 2");
        HostProblem hp;
        DOCH_CHECK(load_problem(p, true, hp));
        for (int b = 0; b < hp.n_inst; ++b) {
            const int64_t lo = hp.off[b], hi = hp.off[b + 1], m = hi - lo;
            double s1, s2, rowmax;
            host_stats(hp, lo, hi, s1, s2, rowmax);
            int meth = method;
            if (meth == 0) meth = m < 10000 ? 1 : 2;
            double lam;
            if (meth == 1) {
                lam = power_lambda_neg(hp, lo, hi, rowmax);
            } else {
                const double cnt = static_cast<double>(m) * (m - 1.0);
                const double mean = cnt > 0 ? s1 / cnt : 0.0;
                const double var = cnt > 0 ? std::max(0.0, s2 / cnt - mean * mean) : 0.0;
                lam = 2.0 * std::sqrt(var) * std::sqrt(static_cast<double>(m));
            }
            const double alpha = eta * lam;
            alpha_out[b] = alpha;
            beta_out[b] = std::pow(static_cast<double>(m), 1.5) * (alpha + rowmax);
        }
        return ISING_OK;
    });
}

ising_status_t ising_create(const ising_problem_t *p, int32_t flags, ising_handle_t *out) {
    return doch::guarded([&]() -> ising_status_t {
        g_err.clear();
        if (!out) return fail(ISING_ERR_INVALID_ARG, "out is NULL");
        *out = nullptr;
        HostProblem hp;
        DOCH_CHECK(load_problem(p, !(flags & ISING_FLAG_SKIP_VALIDATION), hp));
        ising_context *c = new ising_context();
        ising_status_t s = build_context(hp, flags, c);
        if (s != ISING_OK) {
            destroy_ctx(c);
            return s;
        }
        *out = c;
        return ISING_OK;
    });
}

ising_status_t ising_create_s5(int64_t n, double p, uint64_t seed, int32_t flags, ising_handle_t *out) {
    return doch::guarded([&]() -> ising_status_t {
        g_err.clear();
        if (!out) return fail(ISING_ERR_INVALID_ARG, "out is NULL");
        *out = nullptr;
        if (n < 2 || n >= (int64_t(1) << 31)) return fail(ISING_ERR_INVALID_ARG, "n must be in 2 .. 2^31 - 1");
        if (!(p > 0.0) || p > 100.0) return fail(ISING_ERR_INVALID_ARG, "p (percent) must be in (0, 100]");
        // N_p = floor(102300 / p); keep u < T = ceil(1022 * 2^64 / N_p) (exact in 128-bit integers)
        const uint64_t np = static_cast<uint64_t>(std::floor(102300.0 / p));
        const unsigned __int128 num = static_cast<unsigned __int128>(1022) << 64;
        const uint64_t thr = static_cast<uint64_t>((num + np - 1) / np);
        ising_context *c = new ising_context();
        auto bail = [&](ising_status_t s) {
            destroy_ctx(c);
            return s;
        };
        ising_status_t s;
        if ((s = [&]() -> ising_status_t {
                 DOCH_CUDA(cudaGetDevice(&c->device));
                 DOCH_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
                 c->flags = flags;
                 c->format = ISING_FMT_CSR;
                 c->jtype = ISING_I32;
                 c->n = n;
                 c->n_inst = 1;
                 c->inst_off_h = {0, n};
                 c->max_inst_n = n;
                 c->has_h = false;
                 c->integer = true;
                 DOCH_CHECK(upload(&c->inst_off, c->inst_off_h.data(), sizeof(int64_t) * 2));
                 constexpr uint64_t kTagS5 = 13;  // sub-stream tag of the S5 draws
                 DOCH_CHECK(s5_generate(c, n, s5_stream_seed(seed, kTagS5), thr, np));
                 void *ew = nullptr;
                 DOCH_CUDA(cudaMalloc(&ew, sizeof(int)));
                 c->err_word = static_cast<int *>(ew);
                 DOCH_CUDA(cudaMemset(c->err_word, 0, sizeof(int)));
                 void *eh = nullptr;
                 DOCH_CUDA(cudaMallocHost(&eh, sizeof(int)));
                 c->err_host = static_cast<int *>(eh);
                 *c->err_host = 0;
                 return ISING_OK;
             }()) != ISING_OK)
            return bail(s);
        *out = c;
        return ISING_OK;
    });
}

ising_status_t ising_create_procedural(int64_t n, int64_t cst, int32_t flags, ising_handle_t *out) {
    return doch::guarded([&]() -> ising_status_t {
        g_err.clear();
        if (!out) return fail(ISING_ERR_INVALID_ARG, "out is NULL");
        *out = nullptr;
        if (n < 2 || n > (int64_t(1) << 30)) return fail(ISING_ERR_INVALID_ARG, "n must be in 2 .. 2^30");
        if (cst < 0 || cst > (int64_t(1) << 40)) return fail(ISING_ERR_INVALID_ARG, "c must be in 0 .. 2^40");
        ising_context *c = new ising_context();
        ising_status_t s = [&]() -> ising_status_t {
            DOCH_CUDA(cudaGetDevice(&c->device));
            DOCH_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
            c->flags = flags;
            c->format = ISING_FMT_PROCEDURAL;
            c->jtype = ISING_F32;
            c->n = n;
            c->n_inst = 1;
            c->inst_off_h = {0, n};
            c->max_inst_n = n;
            c->has_h = false;
            c->integer = false;
            c->proc_offset = cst;
            proc_closed_sums(n, cst, &c->proc_s1, &c->proc_s2);
            DOCH_CHECK(upload(&c->inst_off, c->inst_off_h.data(), sizeof(int64_t) * 2));
            void *ew = nullptr;
            DOCH_CUDA(cudaMalloc(&ew, sizeof(int)));
            c->err_word = static_cast<int *>(ew);
            DOCH_CUDA(cudaMemset(c->err_word, 0, sizeof(int)));
            void *eh = nullptr;
            DOCH_CUDA(cudaMallocHost(&eh, sizeof(int)));
            c->err_host = static_cast<int *>(eh);
            *c->err_host = 0;
            return ISING_OK;
        }();
        if (s != ISING_OK) {
            destroy_ctx(c);
            return s;
        }
        *out = c;
        return ISING_OK;
    });
}

ising_status_t ising_params_device(ising_handle_t h, double eta, int32_t method, double *alpha_out,
                                   double *beta_out) {
    return doch::guarded([&]() -> ising_status_t {
        g_err.clear();
        if (!h || !alpha_out || !beta_out) return fail(ISING_ERR_INVALID_ARG, "NULL argument");
        if (!(eta > 0.0) || !std::isfinite(eta)) return fail(ISING_ERR_INVALID_ARG, "eta must be > 0");
        if (method < 0 || method > 2) return fail(ISING_ERR_INVALID_ARG, "method must be 0, 1 or 2");
        if (h->n_inst != 1) return fail(ISING_ERR_UNSUPPORTED, "device parameters run on one instance");
        if (h->format == ISING_FMT_PROCEDURAL) {
            if (method == 1) return fail(ISING_ERR_UNSUPPORTED, "PROCEDURAL couplings take the Wigner estimate");
            return proc_params(h, eta, alpha_out, beta_out);
        }
        return params_device(h, eta, method, alpha_out, beta_out);
    });
}

ising_status_t ising_csr_export(ising_handle_t h, int64_t *row_ptr, int32_t *col, void *val, int64_t *nnz_out,
                                int32_t *jtype_out) {
    return doch::guarded([&]() -> ising_status_t {
        g_err.clear();
        if (!h) return fail(ISING_ERR_INVALID_ARG, "handle is NULL");
        if (h->format != ISING_FMT_CSR) return fail(ISING_ERR_UNSUPPORTED, "the handle does not hold CSR couplings");
        if (nnz_out) *nnz_out = h->nnz;
        if (jtype_out) *jtype_out = h->jtype;
        if (row_ptr) DOCH_CUDA(cudaMemcpy(row_ptr, h->row_ptr, sizeof(int64_t) * (h->n + 1), cudaMemcpyDefault));
        if (col && h->nnz) DOCH_CUDA(cudaMemcpy(col, h->col, sizeof(int32_t) * h->nnz, cudaMemcpyDefault));
        if (val && h->nnz) DOCH_CUDA(cudaMemcpy(val, h->val, dtype_size(h->jtype) * h->nnz, cudaMemcpyDefault));
        return ISING_OK;
    });
}

void ising_destroy(ising_handle_t h) { destroy_ctx(h); }

ising_status_t ising_selftest_wait(ising_handle_t h, int32_t arrive, int64_t limit_ns, void *stream) {
    return doch::guarded([&]() -> ising_status_t {
        g_err.clear();
        if (!h) return fail(ISING_ERR_INVALID_ARG, "handle is NULL");
        if (limit_ns < 1000 || limit_ns > 1000000000LL)
            return fail(ISING_ERR_INVALID_ARG, "limit_ns must be in 1e3 .. 1e9");
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        DOCH_CHECK(selftest_wait_launch(h->err_word, arrive != 0, static_cast<uint64_t>(limit_ns), st));
        return finish(h, st, true);
    });
}

ising_status_t ising_get_size(ising_handle_t h, int64_t *n, int32_t *n_instances) {
    return doch::guarded([&]() -> ising_status_t {
        if (!h) return fail(ISING_ERR_INVALID_ARG, "handle is NULL");
        if (n) *n = h->n;
        if (n_instances) *n_instances = h->n_inst;
        return ISING_OK;
    });
}

ising_status_t ising_synchronize(ising_handle_t h, void *stream) {
    return doch::guarded([&]() -> ising_status_t {
        if (!h) return fail(ISING_ERR_INVALID_ARG, "handle is NULL");
        return finish(h, static_cast<cudaStream_t>(stream), true);
    });
}

ising_status_t ising_iterate(ising_handle_t h, void *x, int32_t xtype, int32_t R, const double *alpha,
                             int32_t alpha_len, const double *beta, int32_t iters, double *H_trace,
                             void *stream) {
    return doch::guarded([&]() -> ising_status_t {
        g_err.clear();
        if (!h || !x || !alpha || !beta) return fail(ISING_ERR_INVALID_ARG, "NULL argument");
        if (R < 1 || iters < 0) return fail(ISING_ERR_INVALID_ARG, "R must be >= 1 and iters >= 0");
        if (alpha_len != 1 && alpha_len != iters) return fail(ISING_ERR_INVALID_ARG, "alpha_len must be 1 or iters");
        if (h->format == ISING_FMT_DENSE) {
            if (xtype != ISING_BF16 && xtype != ISING_F32)
                return fail(ISING_ERR_INVALID_ARG, "DENSE iterates are BF16 (tensor cores) or F32 (plain FP32 form)");
        } else if (h->format == ISING_FMT_PROCEDURAL) {
            if (xtype != ISING_F32) return fail(ISING_ERR_INVALID_ARG, "PROCEDURAL iterates are F32");
        } else if (xtype != ISING_F32 && xtype != ISING_F64) {
            return fail(ISING_ERR_INVALID_ARG, "iterates must be F32 or F64");
        }
        if (R > 65535) return fail(ISING_ERR_INVALID_ARG, "R must be <= 65535");
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        ising_context *c = h;
        const int64_t count = c->n * R;
        const size_t xbytes = static_cast<size_t>(count) * xtype_size(xtype);
        std::vector<double> alpha_h(static_cast<size_t>(c->n_inst) * alpha_len), beta_h(c->n_inst);
        {
            std::vector<unsigned char> tmp;
            DOCH_CHECK(to_host(alpha, sizeof(double) * alpha_h.size(), tmp));
            std::memcpy(alpha_h.data(), tmp.data(), tmp.size());
            DOCH_CHECK(to_host(beta, sizeof(double) * beta_h.size(), tmp));
            std::memcpy(beta_h.data(), tmp.data(), tmp.size());
        }
        ParamTabs p;
        DOCH_CHECK(upload_params(c, alpha, alpha_len, beta, p, st));
    
        const bool x_dev = is_device_ptr(x);
        void *xd = x;
        if (!x_dev) {
            DOCH_CHECK(c->stage_x.ensure(xbytes));
            xd = c->stage_x.ptr;
            DOCH_CUDA(cudaMemcpyAsync(xd, x, xbytes, cudaMemcpyHostToDevice, st));
        }
        const int pairs = c->n_inst * R;
        double *Hd = nullptr;
        if (H_trace) {
            DOCH_CHECK(c->work.ensure(sizeof(double) * pairs * (static_cast<size_t>(iters) + 1)));
            Hd = c->work.as<double>();
        }
        bool done = false;
        if (c->format == ISING_FMT_DENSE) {
            if (H_trace) return fail(ISING_ERR_UNSUPPORTED, "H trace is not available for DENSE couplings");
            if (c->n_inst != 1) return fail(ISING_ERR_UNSUPPORTED, "DENSE runs one instance");
            if (iters > 0 && xtype == ISING_BF16)
                DOCH_CHECK(dense_iterate(c, xd, R, alpha_h.data(), alpha_len, beta_h[0], iters, st));
            if (iters > 0 && xtype == ISING_F32)
                DOCH_CHECK(dense_iterate_f32(c, static_cast<float *>(xd), R, alpha_h.data(), alpha_len, beta_h[0],
                                             iters, st));
            done = true;
        }
        if (!done && !H_trace && c->format == ISING_FMT_CSR && c->n_inst > 1 && xtype == ISING_F32 && iters > 0) {
            DOCH_CHECK(batched_iterate(c, static_cast<float *>(xd), R, p, iters, st));
            done = true;
        }
        if (!done && !H_trace && c->format == ISING_FMT_CSR && iters > 0) {
            ising_status_t s = csr_fused(c, xd, xtype, R, p, iters, st);
            if (s == ISING_OK) done = true;
            else if (s != ISING_ERR_UNSUPPORTED) return s;
        }
        if (!done && iters > 0) {
            DOCH_CHECK(c->ping.ensure(xbytes));
            void *cur = xd, *nxt = c->ping.ptr;
            const bool pairs_ok = !Hd && c->format == ISING_FMT_TORUS2D && xtype == ISING_F32 &&
                                  !(c->flags & ISING_FLAG_SINGLE_STEP) &&
                                  torus_pair_ok(c, static_cast<const float *>(cur), static_cast<const float *>(nxt), R);
            // steps per lattice pass: at most 3 (default) or ISING_LATTICE_PASS = 1, 2 or 3
            int per_pass = 3;
            if (const char *env = std::getenv("ISING_LATTICE_PASS")) {
                const int v = std::atoi(env);
                if (v >= 1 && v <= 3) per_pass = v;
            }
            const bool triples_ok = pairs_ok && per_pass >= 3 && c->l_rows >= 6;
            for (int k = 0; k < iters;) {
                if (triples_ok && k + 2 < iters) {  // three steps in one pass over the lattice
                    const double a1 = alpha_h[alpha_len == 1 ? 0 : k], a2 = alpha_h[alpha_len == 1 ? 0 : k + 1],
                                 a3 = alpha_h[alpha_len == 1 ? 0 : k + 2];
                    DOCH_CHECK(torus_triple_f32(c, static_cast<const float *>(cur), static_cast<float *>(nxt),
                                                static_cast<float>(a1), static_cast<float>(a2), static_cast<float>(a3),
                                                1.0 / beta_h[0], st));
                    std::swap(cur, nxt);
                    k += 3;
                    continue;
                }
                if (pairs_ok && per_pass >= 2 && k + 1 < iters) {  // two steps in one pass over the lattice
                    const double a1 = alpha_h[alpha_len == 1 ? 0 : k], a2 = alpha_h[alpha_len == 1 ? 0 : k + 1];
                    DOCH_CHECK(torus_pair_f32(c, static_cast<const float *>(cur), static_cast<float *>(nxt),
                                              static_cast<float>(a1), static_cast<float>(a2), 1.0 / beta_h[0], st));
                    std::swap(cur, nxt);
                    k += 2;
                    continue;
                }
                // H monitor fused into the step where the step kernel supports it (the exact
                // separate FP64 reduction for FP32 iterates under ISING_FLAG_STRICT_MONOTONE)
                bool fused = false;
                if (Hd && !(xtype == ISING_F32 && (c->flags & ISING_FLAG_STRICT_MONOTONE))) {
                    const double ak = alpha_h[alpha_len == 1 ? 0 : k];
                    double *Hk = Hd + static_cast<size_t>(k) * pairs;
                    ising_status_t fs = ISING_ERR_UNSUPPORTED;
                    if (c->format == ISING_FMT_CSR)
                        fs = csr_step_traced(c, cur, nxt, xtype, R, p, k, ak, beta_h[0], Hk, st);
                    else if (c->format == ISING_FMT_TORUS2D && xtype == ISING_F32)
                        fs = torus_step_f32_traced(c, static_cast<const float *>(cur), static_cast<float *>(nxt), R,
                                                   static_cast<float>(ak), 1.0 / beta_h[0], ak, beta_h[0], Hk, st);
                    if (fs != ISING_OK && fs != ISING_ERR_UNSUPPORTED) return fs;
                    fused = fs == ISING_OK;
                }
                if (!fused) {
                    if (Hd) DOCH_CHECK(hamiltonian_reduce(c, cur, xtype, R, p, k, Hd + static_cast<size_t>(k) * pairs, st));
                    DOCH_CHECK(step(c, cur, nxt, xtype, R, p, alpha_h, beta_h, k, st));
                }
                std::swap(cur, nxt);
                ++k;
            }
            if (Hd) DOCH_CHECK(hamiltonian_reduce(c, cur, xtype, R, p, iters - 1, Hd + static_cast<size_t>(iters) * pairs, st));
            if (cur != xd) DOCH_CUDA(cudaMemcpyAsync(xd, cur, xbytes, cudaMemcpyDeviceToDevice, st));
        } else if (!done && Hd) {
            DOCH_CHECK(hamiltonian_reduce(c, xd, xtype, R, p, 0, Hd, st));
        }
        bool must_sync = !x_dev;
        if (!x_dev) DOCH_CUDA(cudaMemcpyAsync(x, xd, xbytes, cudaMemcpyDeviceToHost, st));
        if (Hd) {
            const size_t hb = sizeof(double) * pairs * (static_cast<size_t>(iters) + 1);
            DOCH_CUDA(cudaMemcpyAsync(H_trace, Hd, hb, cudaMemcpyDefault, st));
            if (!is_device_ptr(H_trace)) must_sync = true;
            if (c->flags & ISING_FLAG_STRICT_MONOTONE) {
                DOCH_CHECK(finish(c, st, true));
                std::vector<double> Hh(pairs * (static_cast<size_t>(iters) + 1));
                DOCH_CUDA(cudaMemcpy(Hh.data(), Hd, hb, cudaMemcpyDeviceToHost));
                for (int k = 0; k < iters; ++k)
                    for (int t = 0; t < pairs; ++t) {
                        const double a = Hh[static_cast<size_t>(k) * pairs + t], b = Hh[static_cast<size_t>(k + 1) * pairs + t];
                        if (b > a + 1e-6 * std::fabs(a))
                            return fail(ISING_ERR_NOT_MONOTONE, "H rose at step " + std::to_string(k));
                    }
            }
        }
        return finish(c, st, must_sync);
    });
}

ising_status_t ising_iterate_adoch(ising_handle_t h, void *x, int32_t xtype, int32_t R, const double *alpha,
                                   const double *beta, int32_t iters, int32_t q, int8_t *accepted,
                                   double *H_trace, void *stream) {
    return doch::guarded([&]() -> ising_status_t {
        g_err.clear();
        if (!h || !x || !alpha || !beta) return fail(ISING_ERR_INVALID_ARG, "NULL argument");
        if (R < 1 || R > 65535 || iters < 0 || q < 0)
            return fail(ISING_ERR_INVALID_ARG, "R must be in 1..65535, iters >= 0 and q >= 0");
        if (xtype != ISING_F32 && xtype != ISING_F64) return fail(ISING_ERR_INVALID_ARG, "iterates must be F32 or F64");
        ising_context *c = h;
        if (c->format != ISING_FMT_CSR && c->format != ISING_FMT_TORUS2D && c->format != ISING_FMT_PROCEDURAL)
            return fail(ISING_ERR_UNSUPPORTED, "ADOCH runs on CSR, TORUS2D or PROCEDURAL couplings");
        if (c->format == ISING_FMT_PROCEDURAL && xtype != ISING_F32)
            return fail(ISING_ERR_INVALID_ARG, "PROCEDURAL iterates are F32");
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        const int64_t count = c->n * R;
        const size_t xbytes = static_cast<size_t>(count) * xtype_size(xtype);
        ParamTabs p;
        DOCH_CHECK(upload_params(c, alpha, 1, beta, p, st));
        const bool x_dev = is_device_ptr(x);
        void *xd = x;
        if (!x_dev) {
            DOCH_CHECK(c->stage_x.ensure(xbytes));
            xd = c->stage_x.ptr;
            DOCH_CUDA(cudaMemcpyAsync(xd, x, xbytes, cudaMemcpyHostToDevice, st));
        }
        const int pairs = c->n_inst * R;
        const size_t ab = static_cast<size_t>(pairs) * iters;
        const size_t hb = sizeof(double) * pairs * (static_cast<size_t>(iters) + 1);
        int8_t *acc_dev = nullptr;
        double *H_dev = nullptr;
        const bool acc_on_dev = accepted && is_device_ptr(accepted);
        const bool H_on_dev = H_trace && is_device_ptr(H_trace);
        if (accepted) {
            if (acc_on_dev) {
                acc_dev = accepted;
            } else {
                DOCH_CHECK(c->stage_out.ensure(ab + 1));
                acc_dev = c->stage_out.as<int8_t>();
            }
        }
        if (H_trace) {
            if (H_on_dev) {
                H_dev = H_trace;
            } else {
                DOCH_CHECK(c->work.ensure(hb));
                H_dev = c->work.as<double>();
            }
        }
        if (iters > 0) DOCH_CHECK(adoch_iterate(c, xd, xtype, R, p, iters, q, acc_dev, H_dev, st));
        if (H_dev) DOCH_CHECK(hamiltonian_reduce(c, xd, xtype, R, p, 0, H_dev + static_cast<size_t>(iters) * pairs, st));
        bool must_sync = false;
        if (!x_dev) {
            DOCH_CUDA(cudaMemcpyAsync(x, xd, xbytes, cudaMemcpyDeviceToHost, st));
            must_sync = true;
        }
        if (accepted && !acc_on_dev && ab > 0) {
            DOCH_CUDA(cudaMemcpyAsync(accepted, acc_dev, ab, cudaMemcpyDeviceToHost, st));
            must_sync = true;
        }
        if (H_trace && !H_on_dev) {
            DOCH_CUDA(cudaMemcpyAsync(H_trace, H_dev, hb, cudaMemcpyDeviceToHost, st));
            must_sync = true;
        }
        return finish(c, st, must_sync);
    });
}

ising_status_t ising_iterate_until(ising_handle_t h, void *x, int32_t xtype, int32_t R, const double *alpha,
                                   const double *beta, int32_t max_iters, double eps, int32_t *steps_out,
                                   void *stream) {
    return doch::guarded([&]() -> ising_status_t {
        g_err.clear();
        if (!h || !x || !alpha || !beta) return fail(ISING_ERR_INVALID_ARG, "NULL argument");
        if (R < 1 || R > 65535 || max_iters < 0) return fail(ISING_ERR_INVALID_ARG, "R must be in 1..65535, max_iters >= 0");
        if (!std::isfinite(eps) || eps < 0.0) return fail(ISING_ERR_INVALID_ARG, "eps must be finite and >= 0");
        if (xtype != ISING_F32 && xtype != ISING_F64) return fail(ISING_ERR_INVALID_ARG, "iterates must be F32 or F64");
        ising_context *c = h;
        if (c->format == ISING_FMT_DENSE)
            return fail(ISING_ERR_UNSUPPORTED, "the stopping rule runs on CSR, TORUS2D or PROCEDURAL");
        if (c->format == ISING_FMT_PROCEDURAL && xtype != ISING_F32)
            return fail(ISING_ERR_INVALID_ARG, "PROCEDURAL iterates are F32");
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        const int64_t count = c->n * R;
        const size_t xbytes = static_cast<size_t>(count) * xtype_size(xtype);
        const int pairs = c->n_inst * R;
        std::vector<double> alpha_h(c->n_inst), beta_h(c->n_inst);
        {
            std::vector<unsigned char> tmp;
            DOCH_CHECK(to_host(alpha, sizeof(double) * alpha_h.size(), tmp));
            std::memcpy(alpha_h.data(), tmp.data(), tmp.size());
            DOCH_CHECK(to_host(beta, sizeof(double) * beta_h.size(), tmp));
            std::memcpy(beta_h.data(), tmp.data(), tmp.size());
        }
        ParamTabs p;
        DOCH_CHECK(upload_params(c, alpha, 1, beta, p, st));
        const bool x_dev = is_device_ptr(x);
        void *xd = x;
        if (!x_dev) {
            DOCH_CHECK(c->stage_x.ensure(xbytes));
            xd = c->stage_x.ptr;
            DOCH_CUDA(cudaMemcpyAsync(xd, x, xbytes, cudaMemcpyHostToDevice, st));
        }
        // work: result | partials | running | steps | stopped_now | n_running (256-byte aligned)
        auto al = [](size_t v) { return (v + 255) & ~static_cast<size_t>(255); };
        const size_t o1 = al(xbytes), o2 = o1 + al(stop_partials_bytes(c, R)), o3 = o2 + al(sizeof(int) * pairs),
                     o4 = o3 + al(sizeof(int32_t) * pairs), o5 = o4 + al(sizeof(int) * pairs), tot = o5 + 256;
        DOCH_CHECK(c->work.ensure(tot));
        unsigned char *wb = c->work.as<unsigned char>();
        void *res = wb;
        StopState s;
        s.partials = reinterpret_cast<double *>(wb + o1);
        s.running = reinterpret_cast<int *>(wb + o2);
        s.steps = reinterpret_cast<int32_t *>(wb + o3);
        s.stopped_now = reinterpret_cast<int *>(wb + o4);
        s.n_running = reinterpret_cast<int *>(wb + o5);
        {
            std::vector<int> ones(pairs, 1), st0(pairs, max_iters);
            DOCH_CUDA(cudaMemcpyAsync(s.running, ones.data(), sizeof(int) * pairs, cudaMemcpyHostToDevice, st));
            DOCH_CUDA(cudaMemcpyAsync(s.steps, st0.data(), sizeof(int32_t) * pairs, cudaMemcpyHostToDevice, st));
            DOCH_CUDA(cudaMemcpyAsync(s.n_running, &pairs, sizeof(int), cudaMemcpyHostToDevice, st));
            DOCH_CUDA(cudaMemsetAsync(s.stopped_now, 0, sizeof(int) * pairs, st));
            DOCH_CUDA(cudaStreamSynchronize(st));  // the sources are pageable
        }
        // batched FP32 instances: the rule runs inside the shared-memory resident kernel, which
        // ends each (instance, replica group) as soon as all of its replicas stopped
        ising_status_t rs = ISING_ERR_UNSUPPORTED;
        if (c->format == ISING_FMT_CSR && c->n_inst > 1 && xtype == ISING_F32 && max_iters > 0)
            if (batched_resident_ok(c, static_cast<float *>(xd), R)) {
            ResidentConfig rc;
            rs = tune_resident(c, static_cast<float *>(xd), R, p, st, &rc);
            if (rs == ISING_OK)
                rs = batched_resident_launch(c, rc, static_cast<float *>(xd), R, p, max_iters, st,
                                             static_cast<float>(eps), s.steps);
        }
        if (rs != ISING_OK && rs != ISING_ERR_UNSUPPORTED) return rs;
        if (rs == ISING_ERR_UNSUPPORTED) {
            if (!c->count_host) DOCH_CUDA(cudaHostAlloc(reinterpret_cast<void **>(&c->count_host), sizeof(int), 0));
            DOCH_CHECK(c->ping.ensure(xbytes));
            void *cur = xd, *nxt = c->ping.ptr;
            constexpr int kPoll = 8;  // steps between host checks of the running-pair count
            for (int k = 0; k < max_iters; ++k) {
                DOCH_CHECK(step(c, cur, nxt, xtype, R, p, alpha_h, beta_h, k, st));
                DOCH_CHECK(stop_step(c, cur, nxt, res, xtype, R, eps, k, s, st));
                std::swap(cur, nxt);
                if ((k + 1) % kPoll == 0 && k + 1 < max_iters) {
                    DOCH_CUDA(cudaMemcpyAsync(c->count_host, s.n_running, sizeof(int), cudaMemcpyDeviceToHost, st));
                    DOCH_CUDA(cudaStreamSynchronize(st));
                    if (*c->count_host == 0) break;
                }
            }
            DOCH_CHECK(stop_finish(c, cur, res, xtype, R, s, st));
            DOCH_CUDA(cudaMemcpyAsync(xd, res, xbytes, cudaMemcpyDeviceToDevice, st));
        }
        bool must_sync = false;
        if (!x_dev) {
            DOCH_CUDA(cudaMemcpyAsync(x, xd, xbytes, cudaMemcpyDeviceToHost, st));
            must_sync = true;
        }
        if (steps_out) {
            DOCH_CUDA(cudaMemcpyAsync(steps_out, s.steps, sizeof(int32_t) * pairs, cudaMemcpyDefault, st));
            if (!is_device_ptr(steps_out)) must_sync = true;
        }
        return finish(c, st, must_sync);
    });
}

ising_status_t ising_energy(ising_handle_t h, const void *x, int32_t xtype, int32_t R, int64_t *E_int,
                            int64_t *cut_int, double *E_f64, double *cut_f64, int32_t *best, int8_t *spins,
                            void *stream) {
    return doch::guarded([&]() -> ising_status_t {
        g_err.clear();
        if (!h || !x) return fail(ISING_ERR_INVALID_ARG, "NULL argument");
        if (R < 1 || R > 65535) return fail(ISING_ERR_INVALID_ARG, "R out of range");
        if (xtype != ISING_F32 && xtype != ISING_F64 && xtype != ISING_BF16 && xtype != ISING_I8)
            return fail(ISING_ERR_INVALID_ARG, "x must be F32, F64, BF16 or I8");
        ising_context *c = h;
        if ((E_int || cut_int) && !c->integer)
            return fail(ISING_ERR_INVALID_ARG, "integer energies need integer couplings and field");
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        const int64_t count = c->n * R;
        const size_t xbytes = static_cast<size_t>(count) * xtype_size(xtype);
        const void *xd = x;
        bool must_sync = false;
        if (!is_device_ptr(x)) {
            DOCH_CHECK(c->stage_x.ensure(xbytes));
            DOCH_CUDA(cudaMemcpyAsync(c->stage_x.ptr, x, xbytes, cudaMemcpyHostToDevice, st));
            xd = c->stage_x.ptr;
            must_sync = true;
        }
        const size_t pairs = static_cast<size_t>(c->n_inst) * R;
        // staging of the outputs: E_i | cut_i | E_d | cut_d | best
        DOCH_CHECK(c->stage_out.ensure(pairs * 8 * 4 + c->n_inst * 4 + 64));
        int64_t *Ei = c->stage_out.as<int64_t>();
        int64_t *Ci = Ei + pairs;
        double *Ed = reinterpret_cast<double *>(Ci + pairs);
        double *Cd = Ed + pairs;
        int32_t *Bd = reinterpret_cast<int32_t *>(Cd + pairs);
        if (c->format == ISING_FMT_DENSE)
            DOCH_CHECK(dense_energy(c, xd, xtype, R, Ei, Ci, Ed, Cd, st));
        else if (c->format == ISING_FMT_PROCEDURAL)
            DOCH_CHECK(proc_energy(c, xd, xtype, R, Ed, Cd, st));
        else
            DOCH_CHECK(energy_reduce(c, xd, xtype, R, c->integer ? Ei : nullptr, c->integer ? Ci : nullptr, Ed, Cd, st));
        if (best) DOCH_CHECK(best_replica(c, c->integer ? Ei : nullptr, Ed, R, Bd, st));
        auto put = [&](void *dst, const void *src, size_t bytes) -> ising_status_t {
            if (!dst) return ISING_OK;
            if (!is_device_ptr(dst)) must_sync = true;
            DOCH_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
            return ISING_OK;
        };
        DOCH_CHECK(put(E_int, Ei, pairs * 8));
        DOCH_CHECK(put(cut_int, Ci, pairs * 8));
        DOCH_CHECK(put(E_f64, Ed, pairs * 8));
        DOCH_CHECK(put(cut_f64, Cd, pairs * 8));
        DOCH_CHECK(put(best, Bd, c->n_inst * 4));
        if (spins) {
            if (is_device_ptr(spins)) {
                DOCH_CHECK(write_spins(c, xd, xtype, R, spins, st));
            } else {
                DOCH_CHECK(c->work.ensure(count));
                DOCH_CHECK(write_spins(c, xd, xtype, R, c->work.as<int8_t>(), st));
                DOCH_CUDA(cudaMemcpyAsync(spins, c->work.ptr, count, cudaMemcpyDeviceToHost, st));
                must_sync = true;
            }
        }
        return finish(c, st, must_sync);
    });
}

ising_status_t ising_tune_eta(ising_handle_t h, const void *x0, int32_t xtype, int32_t R, const double *etas,
                              int32_t n_etas, int32_t probe_iters, double alpha1, double beta1, double *score_best,
                              double *score_mean, int32_t *best_index, double *alpha_out, double *beta_out,
                              void *stream) {
    return doch::guarded([&]() -> ising_status_t {
        g_err.clear();
        if (!h || !x0 || !etas) return fail(ISING_ERR_INVALID_ARG, "NULL argument");
        ising_context *c = h;
        if (c->n_inst != 1) return fail(ISING_ERR_UNSUPPORTED, "ising_tune_eta runs on one instance");
        if (R < 1 || R > 65535 || n_etas < 1 || n_etas > 4096 || probe_iters < 0)
            return fail(ISING_ERR_INVALID_ARG, "need 1 <= R <= 65535, 1 <= n_etas <= 4096, probe_iters >= 0");
        if (!std::isfinite(alpha1) || !std::isfinite(beta1) || beta1 <= 0.0)
            return fail(ISING_ERR_INVALID_ARG, "alpha1 and beta1 must be finite, beta1 > 0");
        std::vector<double> eta_h(n_etas);
        {
            std::vector<unsigned char> tmp;
            DOCH_CHECK(to_host(etas, sizeof(double) * n_etas, tmp));
            std::memcpy(eta_h.data(), tmp.data(), tmp.size());
        }
        const double n15 = std::pow(static_cast<double>(c->n), 1.5);
        std::vector<double> a_h(n_etas), b_h(n_etas);
        for (int k = 0; k < n_etas; ++k) {
            if (!std::isfinite(eta_h[k])) return fail(ISING_ERR_NONFINITE, "eta is not finite");
            a_h[k] = eta_h[k] * alpha1;
            b_h[k] = beta1 + n15 * (eta_h[k] - 1.0) * alpha1;   // beta is affine in alpha (Eq. alphabeta)
            if (!(b_h[k] > 0.0)) return fail(ISING_ERR_INVALID_ARG, "beta of a candidate eta is not > 0");
        }
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        const size_t xbytes = static_cast<size_t>(c->n) * R * xtype_size(xtype);
        const size_t eb = ((sizeof(double) * static_cast<size_t>(R) * n_etas + 255) / 256) * 256;
        const size_t xoff = 2 * eb;
        DOCH_CHECK(c->tune.ensure(xoff + 2 * xbytes));
        unsigned char *base = c->tune.as<unsigned char>();
        int64_t *Ei = reinterpret_cast<int64_t *>(base);       // [n_etas][R] (integer J)
        double *Ed = reinterpret_cast<double *>(base + eb);     // [n_etas][R]
        void *x0d = base + xoff;                                // the start, kept for every candidate
        void *xw = base + xoff + xbytes;                        // the probe iterate
        DOCH_CUDA(cudaMemcpyAsync(x0d, x0, xbytes, cudaMemcpyDefault, st));
        const bool integer = c->integer;
        for (int k = 0; k < n_etas; ++k) {
            DOCH_CUDA(cudaMemcpyAsync(xw, x0d, xbytes, cudaMemcpyDeviceToDevice, st));
            DOCH_CHECK(ising_iterate(h, xw, xtype, R, &a_h[k], 1, &b_h[k], probe_iters, nullptr, stream));
            DOCH_CHECK(ising_energy(h, xw, xtype, R, integer ? Ei + static_cast<size_t>(k) * R : nullptr, nullptr,
                                    integer ? nullptr : Ed + static_cast<size_t>(k) * R, nullptr, nullptr, nullptr,
                                    stream));
        }
        std::vector<int64_t> Ei_h(integer ? static_cast<size_t>(n_etas) * R : 0);
        std::vector<double> Ed_h(static_cast<size_t>(n_etas) * R);
        if (integer) {
            DOCH_CUDA(cudaMemcpyAsync(Ei_h.data(), Ei, sizeof(int64_t) * Ei_h.size(), cudaMemcpyDeviceToHost, st));
        } else {
            DOCH_CUDA(cudaMemcpyAsync(Ed_h.data(), Ed, sizeof(double) * Ed_h.size(), cudaMemcpyDeviceToHost, st));
        }
        DOCH_CHECK(finish(c, st, true));
        if (integer)
            for (size_t t = 0; t < Ei_h.size(); ++t) Ed_h[t] = static_cast<double>(Ei_h[t]);
        // score = best energy over the replicas; ties: lower mean, then the earlier candidate
        std::vector<double> best(n_etas), mean(n_etas);
        int pick = 0;
        for (int k = 0; k < n_etas; ++k) {
            const double *e = Ed_h.data() + static_cast<size_t>(k) * R;
            double mn = e[0], sum = 0.0;
            long long isum = 0;
            for (int r = 0; r < R; ++r) {
                mn = std::min(mn, e[r]);
                if (integer) isum += Ei_h[static_cast<size_t>(k) * R + r];
                else sum += e[r];
            }
            best[k] = mn;
            mean[k] = (integer ? static_cast<double>(isum) : sum) / R;
            if (best[k] < best[pick] || (best[k] == best[pick] && mean[k] < mean[pick])) pick = k;
        }
        auto put = [&](void *dst, const void *src, size_t bytes) -> ising_status_t {
            if (dst) DOCH_CUDA(cudaMemcpy(dst, src, bytes, cudaMemcpyDefault));
            return ISING_OK;
        };
        DOCH_CHECK(put(score_best, best.data(), sizeof(double) * n_etas));
        DOCH_CHECK(put(score_mean, mean.data(), sizeof(double) * n_etas));
        DOCH_CHECK(put(best_index, &pick, sizeof(int32_t)));
        DOCH_CHECK(put(alpha_out, &a_h[pick], sizeof(double)));
        DOCH_CHECK(put(beta_out, &b_h[pick], sizeof(double)));
        return ISING_OK;
    });
}

ising_status_t ising_backward(ising_handle_t h, const void *x0, int32_t xtype, int32_t R, const double *alpha,
                              int32_t iters, double beta, int32_t ckpt_every, double *grad_alpha,
                              void *grad_x0, double *loss, int64_t *zero_events, void *stream) {
    return doch::guarded([&]() -> ising_status_t {
        g_err.clear();
        if (!h || !x0 || !alpha) return fail(ISING_ERR_INVALID_ARG, "NULL argument");
        ising_context *c = h;
        if (c->format != ISING_FMT_CSR || c->n_inst != 1)
            return fail(ISING_ERR_UNSUPPORTED, "ising_backward runs on one CSR instance");
        if (xtype != ISING_F32 && xtype != ISING_F64)
            return fail(ISING_ERR_INVALID_ARG, "ising_backward iterates are F32 or F64");
        const size_t xel = xtype == ISING_F64 ? 8 : 4;
        if (R < 1 || R > 65535 || iters < 1 || ckpt_every < 1)
            return fail(ISING_ERR_INVALID_ARG, "need 1 <= R <= 65535, iters >= 1, ckpt_every >= 1");
        if (!std::isfinite(beta) || beta <= 0.0) return fail(ISING_ERR_INVALID_ARG, "beta must be finite and > 0");
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        const int C = ckpt_every < iters ? ckpt_every : iters;
        const int S = (iters + C - 1) / C;                   // checkpoints x^(sC), s = 0..S-1
        std::vector<double> alpha_h(iters);
        {
            std::vector<unsigned char> tmp;
            DOCH_CHECK(to_host(alpha, sizeof(double) * iters, tmp));
            std::memcpy(alpha_h.data(), tmp.data(), tmp.size());
        }
        ParamTabs p;
        DOCH_CHECK(upload_params(c, alpha_h.data(), iters, &beta, p, st));
        const int V = (R % 4 == 0) ? 4 : (R % 2 == 0 ? 2 : 1);
        if (R / V > 256) return fail(ISING_ERR_UNSUPPORTED, "ising_backward: R / vector width must be <= 256");
        const int64_t rows_per_block = 256 / (R / V);
        int64_t grid64 = (c->n + rows_per_block - 1) / rows_per_block;
        // one resident wave: each thread pipelines the loads of its rows
        if (grid64 > static_cast<int64_t>(kAdjointBlocksPerSm) * c->num_sms)
            grid64 = static_cast<int64_t>(kAdjointBlocksPerSm) * c->num_sms;
        const int grid = static_cast<int>(grid64 < 1 ? 1 : grid64);
        // layout of the handle's checkpoint buffer
        auto al = [](size_t v) { return (v + 255) & ~static_cast<size_t>(255); };
        const size_t A = al(static_cast<size_t>(c->n) * R * xel);        // one iterate
        const size_t G = al(static_cast<size_t>(c->n) * R * sizeof(float)); // one adjoint state
        const size_t part_b = al(sizeof(double) * static_cast<size_t>(iters) * grid);
        const size_t lpart_b = al(sizeof(double) * grid);
        const size_t out_b = al(sizeof(double) * (static_cast<size_t>(iters) + 1) + 8);
        const size_t wide_b = xtype == ISING_F64 ? A : 0;                   // FP64 copy of dL/dx0
        DOCH_CHECK(c->ckpt.ensure(A * (S + C) + 2 * G + wide_b + part_b + lpart_b + out_b));
        unsigned char *base = c->ckpt.as<unsigned char>();
        auto ck = [&](int sg_i) { return static_cast<void *>(base + A * sg_i); };
        auto sg = [&](int m) { return static_cast<void *>(base + A * (S + m)); };
        unsigned char *tail = base + A * (S + C);
        float *gbuf[2] = {reinterpret_cast<float *>(tail), reinterpret_cast<float *>(tail + G)};
        double *wide = reinterpret_cast<double *>(tail + 2 * G);
        double *part = reinterpret_cast<double *>(tail + 2 * G + wide_b);
        double *lpart = reinterpret_cast<double *>(tail + 2 * G + wide_b + part_b);
        double *ga_d = reinterpret_cast<double *>(tail + 2 * G + wide_b + part_b + lpart_b);
        double *loss_d = ga_d + iters;
        unsigned long long *zeros_d = reinterpret_cast<unsigned long long *>(loss_d + 1);
        DOCH_CUDA(cudaMemsetAsync(zeros_d, 0, 8, st));
        const size_t xbytes = static_cast<size_t>(c->n) * R * xel;
        DOCH_CUDA(cudaMemcpyAsync(ck(0), x0, xbytes, cudaMemcpyDefault, st));
        // x^(sC + m) of segment s: checkpoint, recomputed iterate, or the next checkpoint
        auto seg_len = [&](int sg_i) { return std::min(C, iters - sg_i * C); };
        auto xs = [&](int sg_i, int m) -> void * {
            if (m == 0) return ck(sg_i);
            if (m == seg_len(sg_i) && sg_i + 1 < S) return ck(sg_i + 1);
            return sg(m - 1);
        };
        // forward: all segments, storing the checkpoints
        for (int sg_i = 0; sg_i < S; ++sg_i)
            for (int m = 1; m <= seg_len(sg_i); ++m)
                DOCH_CHECK(csr_step(c, xs(sg_i, m - 1), xs(sg_i, m), xtype, R, p, sg_i * C + m - 1, st));
        // loss and g^N (x^N is the last iterate of the last segment)
        int gc = 0;
        DOCH_CHECK(csr_loss_w(c, xs(S - 1, seg_len(S - 1)), xtype, gbuf[gc], R, V, grid, lpart, zeros_d, st));
        const float inv_beta = static_cast<float>(1.0 / beta);
        for (int sg_i = S - 1; sg_i >= 0; --sg_i) {
            const int len = seg_len(sg_i);
            if (sg_i < S - 1)  // the last segment's iterates are still in place from the forward pass
                for (int m = 1; m < len; ++m)
                    DOCH_CHECK(csr_step(c, xs(sg_i, m - 1), xs(sg_i, m), xtype, R, p, sg_i * C + m - 1, st));
            for (int m = len - 1; m >= 0; --m) {
                const int k = sg_i * C + m;
                DOCH_CHECK(csr_adjoint_step(c, gbuf[gc], xs(sg_i, m), xtype, gbuf[1 - gc], R, V,
                                            static_cast<float>(alpha_h[k]), inv_beta, k == 0, grid,
                                            part + static_cast<size_t>(k) * grid, zeros_d, st));
                gc = 1 - gc;
            }
        }
        DOCH_CHECK(adjoint_finish_launch(part, iters, grid, beta, lpart, grid, R, ga_d, loss_d, st));
        bool must_sync = false;
        auto put = [&](void *dst, const void *src, size_t bytes) -> ising_status_t {
            if (!dst) return ISING_OK;
            if (!is_device_ptr(dst)) must_sync = true;
            DOCH_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
            return ISING_OK;
        };
        if (xtype == ISING_F64) {
            DOCH_CHECK(widen_f32_to_f64(gbuf[gc], wide, c->n * R, c->num_sms, st));
            DOCH_CHECK(put(grad_x0, wide, xbytes));
        } else {
            DOCH_CHECK(put(grad_x0, gbuf[gc], xbytes));
        }
        DOCH_CHECK(put(grad_alpha, ga_d, sizeof(double) * iters));
        DOCH_CHECK(put(loss, loss_d, sizeof(double)));
        DOCH_CHECK(put(zero_events, zeros_d, sizeof(int64_t)));
        if (!is_device_ptr(x0)) must_sync = true;
        return finish(c, st, must_sync);
    });
}

}  // extern "C"
