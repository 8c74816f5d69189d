// Internal declarations of libising_doch.so (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <exception>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/ising.h"

namespace doch {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
void set_error(const std::string &msg);
ising_status_t fail(ising_status_t s, const std::string &msg);
ising_status_t cuda_fail(cudaError_t e, const char *what);

// Runs the body of a C-ABI entry point: a host exception (a failed allocation, ...) becomes a
// status instead of leaving through extern "C".
template <typename F>
ising_status_t guarded(F &&f) {
    try {
        return f();
    } catch (const std::bad_alloc &) {
        return fail(ISING_ERR_OOM, "host memory allocation failed");
    } catch (const std::exception &e) {
        return fail(ISING_ERR_INVALID_ARG, std::string("host error: ") + e.what());
    } catch (...) {
        return fail(ISING_ERR_INVALID_ARG, "host error");
    }
}

// (the locals carry a long prefix so that they cannot capture a name used in the argument)
#define DOCH_CUDA(call)                                                          \
    do {                                                                         \
        cudaError_t doch_macro_err_ = (call);                                    \
        if (doch_macro_err_ != cudaSuccess)                                      \
            return ::doch::cuda_fail(doch_macro_err_, #call);                    \
    } while (0)

#define DOCH_CHECK(expr)                                                         \
    do {                                                                         \
        ising_status_t doch_macro_status_ = (expr);                              \
        if (doch_macro_status_ != ISING_OK) return doch_macro_status_;           \
    } while (0)

// ---------------------------------------------------------------------------
// device buffer owned by a handle (grown on demand, never shrunk)
// ---------------------------------------------------------------------------
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    ising_status_t ensure(size_t want);
    void release();
    template <typename T> T *as() const { return static_cast<T *>(ptr); }
};

// device-side error word: bit 0 = a bounded wait ran out
enum { DEV_ERR_TIMEOUT = 1 };

// launch shape of the batched persistent kernel (picked by the autotuner)
struct BatchedConfig {
    int threads = 512;
    int vec = 4;
    int ctas_per_sm = 2;
};

// variant of the shared-memory resident batched kernel (picked by the autotuner):
// threads per CTA, and whether both Jacobi copies of an item's iterate sit in
// shared memory or only x^(k) (the new iterate then goes through global scratch,
// and items hold twice as many replicas)
struct ResidentConfig {
    int threads = 1024;
    bool one_copy = false;
};

// work items of the resident kernel for one variant: (instance, first replica, G,
// ELL slots) as int4, built for R replicas; smem = the largest item's bytes
struct ResidentItems {
    DevBuf buf;
    int gen = 0;  // rebuild counter (part of the key of a captured launch)
    int R = 0;
    int count = 0;
    size_t smem = 0;
};

// Bounded-wait self-test (k_selftest.cu): one mbarrier wait of limit_ns that
// nobody satisfies (arrive = false) or that is satisfied at once.
ising_status_t selftest_wait_launch(int *err, bool arrive, uint64_t limit_ns, cudaStream_t st);

}  // namespace doch

// the opaque handle of the C ABI
struct ising_context {
    int device = 0;
    int num_sms = 0;
    int flags = 0;
    int format = 0;
    int jtype = 0;
    int64_t n = 0;
    int n_inst = 1;
    bool integer = false;  // J and h integer: exact int64 energies available
    bool has_h = false;
    // batched instances
    std::vector<int64_t> inst_off_h;
    int64_t *inst_off = nullptr;  // device [n_inst + 1]
    int64_t max_inst_n = 0;
    // CSR
    int64_t nnz = 0;
    int64_t *row_ptr = nullptr;
    int32_t *col = nullptr;
    void *val = nullptr;  // jtype
    int64_t max_row_nnz = 0;
    // TORUS2D
    int64_t l_rows = 0, l_cols = 0;
    int8_t *right = nullptr, *down = nullptr;
    // DENSE: integer couplings held as BF16 (exact for |J| <= 256) in the
    // tensor-core tile order [ceil(n/128)][dense_ld/64][128][64], 128-byte
    // swizzled; dense_ld = n rounded up to 64 (zero padded)
    // dense_ternary: every entry is -1, 0 or +1 and J is held instead as packed
    // 2-bit codes in the same tile order (2 KB per 128 x 64 tile, row-major,
    // 4 codes per byte from the low bits: 0 -> 0, 1 -> +1, 2 -> -1)
    void *dense = nullptr;
    bool dense_ternary = false;
    int dense_type = 0;
    int64_t dense_ld = 0;
    long long dense_jsum = 0;  // sum_ij J_ij, for the cut
    // PROCEDURAL: J_ij = sin(i j + proc_offset) (1-based, J_ii = 0), generated on
    // the fly; proc_s1 / proc_s2 = sums of J_ij and J_ij^2 over i != j (FP64)
    int64_t proc_offset = 0;
    double proc_s1 = 0.0, proc_s2 = 0.0;
    // one-replica symmetric product: work units (int4) and the fixed-point
    // accumulators (int64 [n], zero between products) plus the max |x| word
    doch::DevBuf proc_units;
    int proc_units_count = 0;
    doch::DevBuf proc_acc;
    doch::DevBuf proc_u;  // J x for the H monitor
    // field (both precisions; integer copy when integral)
    float *h_f32 = nullptr;
    double *h_f64 = nullptr;
    int64_t *h_i64 = nullptr;
    // scratch
    doch::DevBuf ping;      // second iterate buffer for the Jacobi ping-pong
    doch::DevBuf stage_x;   // staging of host iterates
    doch::DevBuf stage_out; // staging of host outputs
    doch::DevBuf partials;  // reduction partials
    doch::DevBuf params;    // alpha/beta tables on the device
    doch::DevBuf ckpt;      // checkpoints of the adjoint
    doch::DevBuf work;      // misc. work space
    doch::DevBuf tune;      // eta tuning: the probe iterate and its energies
    int *err_word = nullptr;  // device error word
    int *err_host = nullptr;  // pinned mirror
    int *count_host = nullptr;  // pinned: running-pair count of the stopping rule
    // batched instances: longest-first queue order, queue counter, tuned shapes,
    // and the captured graph of the persistent launch with the key it was built for
    int32_t *batch_order = nullptr;
    int *batch_queue = nullptr;
    std::map<int, doch::BatchedConfig> batch_tuned;  // by R
    // shared-memory resident kernel: per-instance nnz (host), work items
    // (instance, first replica, G) for batch_items_R replicas, their shared memory
    std::vector<int64_t> inst_nnz_h;
    // transposed ELL copy of batched instances of at most 65536 spins: per
    // instance b, ell_deg[b] slots (the largest row degree) x n_b rows from
    // entry ell_off[b], slot k of row i at ell_off[b] + k n_b + i; 16-bit
    // instance-local columns, FP32 weights; a row's entries in CSR order,
    // padded with (i, 0)
    uint16_t *ell_col = nullptr;
    float *ell_val = nullptr;
    int64_t *ell_off = nullptr;
    std::vector<int> ell_deg_h;
    doch::ResidentItems res_items[2];                   // [two copies, one copy]
    doch::DevBuf res_scratch;                           // one-copy variant: x^(k+1) of every item
    std::map<int, doch::ResidentConfig> res_tuned;      // by R
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t batch_exec = nullptr;
    std::vector<uintptr_t> batch_key;
};

namespace doch {

// ---------------------------------------------------------------------------
// launchers implemented in the kernel translation units
// ---------------------------------------------------------------------------

// TORUS2D, one DOCH step, x_out = T(x_in) (Eq. FPE). XT = float or double.
ising_status_t torus_step_f32(const ising_context *c, const float *x_in, float *x_out, int R,
                              float alpha, double inv_beta, cudaStream_t st);
ising_status_t torus_step_f64(const ising_context *c, const double *x_in, double *x_out, int R,
                              double alpha, double beta, cudaStream_t st);
// TORUS2D, two DOCH steps in one pass (alpha1 then alpha2), FP32, R = 1; only
// when torus_pair_ok() holds.
bool torus_pair_ok(const ising_context *c, const float *x_in, const float *x_out, int R);
ising_status_t torus_pair_f32(const ising_context *c, const float *x_in, float *x_out, float alpha1,
                              float alpha2, double inv_beta, cudaStream_t st);
// TORUS2D, three DOCH steps in one pass (alpha1, alpha2, alpha3), same conditions
// as the two-step pass and l_rows >= 6.
ising_status_t torus_triple_f32(const ising_context *c, const float *x_in, float *x_out, float alpha1, float alpha2,
                                float alpha3, double inv_beta, cudaStream_t st);

// Per-instance parameter tables on the device (filled by ising_iterate):
// alpha [n_inst][alpha_len] and beta [n_inst] in FP64, plus FP32 copies of
// alpha and of 1/beta for the FP32 kernels.
struct ParamTabs {
    const double *alpha_d = nullptr;
    const double *beta_d = nullptr;
    const float *alpha_f = nullptr;
    const float *inv_beta_f = nullptr;
    // per instance, for the prescaled fast cube root: cbrt(z / beta) =
    // cbrt(z * zscale) * xscale with zscale = 2^(3k) / beta, xscale = 2^-k
    const float *zscale_f = nullptr;
    const float *xscale_f = nullptr;
    int alpha_len = 1;
};

// CSR, one DOCH step for all instances (alpha of step k), xtype F32 or F64.
ising_status_t csr_step(const ising_context *c, const void *x_in, void *x_out, int xtype, int R,
                        const ParamTabs &p, int k, cudaStream_t st);
// The same step with the H monitor fused (one instance): H(x^(k)) of Eq. Hamilton
// per replica into H_out [R] (device), alpha_k and beta of the step.
// ISING_ERR_UNSUPPORTED when the fused form does not apply (batched instances,
// R / vector width > 256).
ising_status_t csr_step_traced(ising_context *c, const void *xi, void *xo, int xtype, int R, const ParamTabs &p,
                               int k, double alpha_k, double beta, double *H_out, cudaStream_t st);
// TORUS2D single step (R = 1, FP32 fast path) with the fused H monitor; UNSUPPORTED otherwise.
ising_status_t torus_step_f32_traced(ising_context *c, const float *x_in, float *x_out, int R, float alpha,
                                     double inv_beta, double alpha_k, double beta, double *H_out, cudaStream_t st);
// H per replica from fused per-block partials [blocks][R][4] (x^4, x^2, x u, h x)
ising_status_t ham_fused_finish_launch(const double *hpart, int blocks, int R, double alpha, double beta, double *H,
                                       cudaStream_t st);
// CSR, all `iters` steps in one launch: one CTA per (instance, replica) with
// the iterate in shared memory. ISING_ERR_UNSUPPORTED when an instance does
// not fit (the caller then uses csr_step).
ising_status_t csr_fused(const ising_context *c, void *x, int xtype, int R, const ParamTabs &p,
                         int iters, cudaStream_t st);
size_t csr_fused_max_spins(int xtype);

// Reductions (sign rounding + energy/cut, Hamiltonian monitor, best replica).
// xtype: ISING_F32 / ISING_F64 / ISING_BF16 / ISING_I8.
ising_status_t energy_reduce(ising_context *c, const void *x, int xtype, int R, int64_t *E_i,
                             int64_t *cut_i, double *E_d, double *cut_d, cudaStream_t st);
ising_status_t best_replica(const ising_context *c, const int64_t *E_i, const double *E_d, int R,
                            int32_t *best, cudaStream_t st);
ising_status_t write_spins(const ising_context *c, const void *x, int xtype, int R, int8_t *s,
                           cudaStream_t st);
// H(x) of Eq. Hamilton per (instance, replica), FP64, into H_out [n_inst][R] (device).
// alpha of step k is taken from the tables (k clamped to alpha_len - 1).
ising_status_t hamiltonian_reduce(ising_context *c, const void *x, int xtype, int R,
                                  const ParamTabs &p, int k, double *H_out, cudaStream_t st);

// Batched persistent kernel (k_batched.cu): FP32 iterates, ping-pong xa <-> xb;
// after `iters` steps the result is in xa (iters even) or xb (odd).
// ADOCH (Algorithm 2) for CSR or TORUS2D couplings, F32 or F64 iterates, all
// instances: `iters` steps with history window q; per step and (instance,
// replica) pair the acceptance flag (acc_dev[k][pair], may be NULL) and H(x^k)
// (H_dev[k][pair], may be NULL) are written; x is updated in place.
ising_status_t adoch_iterate(ising_context *c, void *x, int xtype, int R, const ParamTabs &p, int iters, int q,
                             int8_t *acc_dev, double *H_dev, cudaStream_t st);

// Algorithm S5 on the device (k_gen.cu): fills c->row_ptr, col, val (I32),
// nnz and max_row_nnz for n spins; sd = stream seed, thr = keep threshold,
// np = N_p. s5_stream_seed(seed, tag) is the generator's stream seed.
ising_status_t s5_generate(ising_context *c, int64_t n, uint64_t sd, uint64_t thr, uint64_t np);
uint64_t s5_stream_seed(uint64_t seed, uint64_t tag);
// Eq. alphabeta on the device for one instance (CSR or TORUS2D).
ising_status_t params_device(const ising_context *c, double eta, int method, double *alpha, double *beta);

// Stopping rule of Remark S2 (k_stop.cu): device state per (instance,
// replica) pair and the kernels run after each step x^(k) -> x^(k+1).
struct StopState {
    double *partials = nullptr;    // [pair][chunk][2]: sums of (x^(k+1) - x^(k))^2 and (x^(k))^2
    int *running = nullptr;        // [pair] 1 while the pair runs
    int32_t *steps = nullptr;      // [pair] steps taken (max_iters for a pair that never stops)
    int *stopped_now = nullptr;    // [pair] 1 if the pair stopped at this step
    int *n_running = nullptr;      // pairs still running
};
size_t stop_partials_bytes(const ising_context *c, int R);
// r^(k) per pair; pairs stopping now record k + 1 and copy x^(k+1) (xn) into res
ising_status_t stop_step(ising_context *c, const void *xc, const void *xn, void *res, int xtype, int R, double eps,
                         int k, StopState &s, cudaStream_t st);
// pairs still running take xc into res
ising_status_t stop_finish(ising_context *c, const void *xc, void *res, int xtype, int R, StopState &s,
                           cudaStream_t st);

// Batched instances with each (instance, replica group) resident in shared
// memory for all steps (k_batched.cu); ISING_ERR_UNSUPPORTED when an instance
// does not fit or x is not 16-byte aligned. Updates x in place. eps > 0
// applies the stopping rule of Remark S2 per (instance, replica) inside the
// kernel (steps: [pair] steps taken, may be NULL).
ising_status_t batched_resident_launch(ising_context *c, const ResidentConfig &cfg, float *x, int R,
                                       const ParamTabs &p, int iters, cudaStream_t st, float eps = 0.f,
                                       int32_t *steps = nullptr);
// every instance fits the resident kernel (two-copy variant) and x is 16-byte aligned
bool batched_resident_ok(ising_context *c, float *x, int R);
// build (or keep) the resident kernel's work items of a variant for R replicas
ising_status_t resident_items(ising_context *c, int R, bool one_copy);
ising_status_t batched_launch(const ising_context *c, const BatchedConfig &cfg, float *xa, float *xb, int R,
                              const ParamTabs &p, int iters, cudaStream_t st);

// Dense couplings on the tcgen05 tensor cores (k_dense_tc.cu): BF16 iterates.
ising_status_t dense_iterate(ising_context *c, void *x, int R, const double *alpha_h, int alpha_len,
                             double beta, int iters, cudaStream_t st);
ising_status_t dense_energy(ising_context *c, const void *x, int xtype, int R, int64_t *E_i, int64_t *cut_i,
                            double *E_d, double *cut_d, cudaStream_t st);
// Dense couplings, plain FP32 form on the CUDA cores (k_dense_f32.cu): FP32
// iterates [n][R] updated in place, FP32 products and accumulation.
ising_status_t dense_iterate_f32(ising_context *c, float *x, int R, const double *alpha_h, int alpha_len,
                                 double beta, int iters, cudaStream_t st);

// Procedural couplings (k_proc.cu), FP32 iterates, one instance, no field.
// One DOCH step x_out = T(x_in); energies into E_d / cut_d (device, R each);
// Eq. alphabeta with the Wigner estimate; the closed-form sums of J and J^2.
ising_status_t proc_step(ising_context *c, const float *x_in, float *x_out, int R, double alpha, double inv_beta,
                         cudaStream_t st);
ising_status_t proc_energy(ising_context *c, const void *x, int xtype, int R, double *E_d, double *cut_d,
                           cudaStream_t st);
ising_status_t proc_params(ising_context *c, double eta, double *alpha, double *beta);
// u = J x (FP32, [n][R], device), the coupling product alone (ADOCH passes)
ising_status_t proc_product(ising_context *c, const float *x, float *u, int R, cudaStream_t st);
ising_status_t proc_hamiltonian(ising_context *c, const float *x, int R, const ParamTabs &p, int k, double *H_out,
                                cudaStream_t st);
void proc_closed_sums(int64_t n, int64_t c, double *s1, double *s2);

// Adjoint (k_backward.cu): CSR couplings, one instance; iterates F32 or F64
// (xtype), adjoint quantities in FP32. csr_loss_w: g^N = -(J x^N + h)/R with
// per-block loss partials, stored as w^(N-1) = g^N / (3 (x^N)^2); one adjoint
// step from w^k and x^k to w^(k-1) (or g^0 when final_step); FP32 -> FP64
// widening; the fixed-order finish. zeros counts components x^(k) = 0, k >= 1.
// The adjoint step kernel is compiled for kAdjointBlocksPerSm resident blocks of
// 256 threads per SM; its grid is one such wave (grid-stride over the rows).
constexpr int kAdjointBlocksPerSm = 3;
// The CSR step for short rows (nnz <= kPipeAvgDeg * n) is compiled for
// kCsrPipeBlocksPerSm resident blocks of 256 threads per SM (FP32 iterates;
// FP64 iterates, which need more registers: one block fewer).
constexpr int kCsrPipeBlocksPerSm = 4;
constexpr int kPipeAvgDeg = 8;
ising_status_t csr_loss_w(const ising_context *c, const void *x, int xtype, float *w, int R, int V, int grid,
                          double *part, unsigned long long *zeros, cudaStream_t st);
ising_status_t csr_adjoint_step(const ising_context *c, const float *w_in, const void *x_cur, int xtype,
                                float *w_out, int R, int V, float alpha_k, float inv_beta, bool final_step,
                                int grid, double *part, unsigned long long *zeros, cudaStream_t st);
ising_status_t widen_f32_to_f64(const float *a, double *b, int64_t count, int num_sms, cudaStream_t st);
ising_status_t adjoint_finish_launch(const double *part, int iters, int blocks, double beta,
                                     const double *lpart, int lblocks, int R, double *grad_alpha,
                                     double *loss, cudaStream_t st);

// Bounded-wait self-test (k_selftest.cu): one mbarrier wait of limit_ns that
// nobody satisfies (arrive = false) or that is satisfied at once.
ising_status_t selftest_wait_launch(int *err, bool arrive, uint64_t limit_ns, cudaStream_t st);

}  // namespace doch
