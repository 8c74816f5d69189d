/*
 * ising.h -- C ABI of the GB300 (sm_103a) DOCH Ising solver library
 * (libising_doch.so).
 *
 * The library runs the difference-of-convex fixed-point iteration of
 * "A Continuous Energy Ising Machine Leveraging Difference-of-Convex
 * Programming" (arXiv 2509.01928):
 *
 *   x^(k+1) = T(x^(k)),  T(x) = cbrt( beta^-1 ((J + alpha I) x + h) )
 *
 * (Eq. FPE, Methods; Algorithm 1 "DOCH"), followed by sign rounding and an
 * Ising-energy / Max-Cut reduction (Eq. IsingModel; Supplementary Note 5).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Status: every call returns an ising_status_t; nothing aborts or traps.
 *    ising_last_error() returns a message for the calling thread's last
 *    failed call.
 *  - Pointers: array arguments may be host or device pointers; the library
 *    tells them apart with cudaPointerGetAttributes. Host arrays are staged
 *    through device memory owned by the handle and the call synchronises the
 *    stream before returning. Device arrays are used in place.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream). Work is enqueued on that stream. Unless the handle was
 *    created with ISING_FLAG_ASYNC, every call synchronises the stream before
 *    returning and reports device-side errors (bounded-wait timeouts, CUDA
 *    faults) in its status. With ISING_FLAG_ASYNC, calls on device arrays
 *    return after enqueueing; ising_synchronize() reports the errors.
 *  - Layout: an iterate or spin array is [n][R] row-major: the R replicas of
 *    spin i are contiguous. Batched instances are concatenated along n.
 *  - Ownership: ising_create copies J and h into device memory owned by the
 *    handle; the caller may free its copies when it returns. x, outputs and
 *    streams stay the caller's. The handle also owns its scratch buffers
 *    (ping-pong state, reduction partials, checkpoints).
 *  - Threads: one handle must not be used by two threads at once.
 *  - Tuning knobs (environment, read when a handle first needs them):
 *    ISING_LATTICE_PASS = 1, 2 or 3 caps the DOCH steps one pass over a
 *    TORUS2D lattice computes (default 3; every setting gives the same
 *    iterates bit for bit). ISING_RESIDENT_VARIANT = <threads>:<copies>
 *    (512 or 1024 : 1 or 2) fixes the variant of the shared-memory resident
 *    kernel for batched instances instead of the handle's autotuner (every
 *    variant gives the same iterates bit for bit).
 */
#ifndef ISING_DOCH_H
#define ISING_DOCH_H

#include <stdint.h>

#if defined(__GNUC__)
#define ISING_API __attribute__((visibility("default")))
#else
#define ISING_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ISING_OK = 0,
    ISING_ERR_INVALID_ARG = 1,   /* null/negative size, unknown enum, size mismatch   */
    ISING_ERR_NOT_SYMMETRIC = 2, /* J_ij != J_ji (Eq. IsingModel requires symmetry)   */
    ISING_ERR_NONZERO_DIAG = 3,  /* J_ii != 0 (no self-coupling, Eq. IsingModel)      */
    ISING_ERR_INDEX_RANGE = 4,   /* CSR column out of range / row_ptr not monotone    */
    ISING_ERR_NONFINITE = 5,     /* NaN or Inf in J, h, alpha or beta                 */
    ISING_ERR_OOM = 6,           /* device allocation failed                          */
    ISING_ERR_CUDA = 7,          /* a CUDA runtime call or kernel failed              */
    ISING_ERR_TIMEOUT = 8,       /* a bounded device-side wait ran out                */
    ISING_ERR_NOT_MONOTONE = 9,  /* H rose while ISING_FLAG_STRICT_MONOTONE was set   */
    ISING_ERR_UNSUPPORTED = 10   /* valid request this build does not implement       */
} ising_status_t;

/* Storage form of the coupling matrix J. */
typedef enum {
    ISING_FMT_CSR = 0,     /* compressed sparse rows (Supplementary Note 9)            */
    ISING_FMT_TORUS2D = 1, /* periodic 2-D lattice, one coupling per lattice edge      */
    ISING_FMT_DENSE = 2,   /* full n x n row-major matrix                               */
    ISING_FMT_PROCEDURAL = 3,/* J_ij = sin(i j + c), generated on the fly (handles from
                                ising_create_procedural only)                           */
    ISING_FMT_ELL = 4        /* fixed-width rows (converted to CSR by ising_create)      */
} ising_format_t;

/* Element types. */
typedef enum {
    ISING_I8 = 0,
    ISING_I16 = 1,
    ISING_I32 = 2,
    ISING_FP8E4M3 = 3,
    ISING_BF16 = 4,
    ISING_F32 = 5,
    ISING_F64 = 6
} ising_dtype_t;

/* Creation flags. */
enum {
    ISING_FLAG_ASYNC = 1,            /* do not synchronise inside calls on device arrays */
    ISING_FLAG_SKIP_VALIDATION = 2,  /* skip the symmetry, diagonal and finiteness checks of
                                        J and h (index and size checks always run)        */
    ISING_FLAG_STRICT_MONOTONE = 4,  /* ising_iterate fails with ISING_ERR_NOT_MONOTONE
                                        when a recorded H trace rises                    */
    ISING_FLAG_SINGLE_STEP = 8       /* TORUS2D: one kernel pass per step instead of the
                                        fused two-step pass (same results, more traffic) */
};

/*
 * Problem statement (Eq. IsingModel): couplings J (n x n, symmetric,
 * J_ii = 0) and an optional external field h (n). Only the members of the
 * chosen format are read; unused members must be zero/NULL.
 *
 * CSR: row i holds columns col[row_ptr[i] .. row_ptr[i+1]) with values
 *   val[] of type jtype (I8, I16, I32, F32 or F64). Both triangles are stored.
 * TORUS2D: n = l_rows * l_cols; spin index of site (r, c) is r * l_cols + c;
 *   right[r][c] couples (r, c) with (r, (c+1) mod l_cols) and down[r][c]
 *   couples (r, c) with ((r+1) mod l_rows, c); jtype I8. l_rows, l_cols >= 2
 *   (on a 2-wide side both edges of a pair add up to one J_ij).
 * ELL: row i holds the ell_width slots col[i * ell_width + k] (int32; -1
 *   marks an empty slot) with values val[i * ell_width + k] of jtype (I8, I16,
 *   I32, F32 or F64); converted to CSR on create, so everything CSR accepts
 *   (batches included) applies.
 * DENSE: dense[i * n + j] = J_ij, jtype I8, I16, I32, FP8E4M3, BF16, F32 or
 *   F64; every value must be an integer with |J_ij| <= 256 (held exactly in
 *   BF16, or as 2-bit codes when all are -1, 0 or +1).
 * Field: h[n] of type htype (I8, I16, I32, F32, F64), or NULL for h = 0
 *   (CSR and DENSE; a TORUS2D lattice takes no field).
 * Batches: n_instances > 1 (CSR or ELL) concatenates independent problems;
 *   instance b owns spins [inst_offset[b], inst_offset[b+1]) and its rows may
 *   only reference columns of that range. n_instances = 0 or 1 means one
 *   instance and inst_offset may be NULL.
 */
typedef struct {
    int64_t n;
    int32_t format;          /* ising_format_t */
    int32_t jtype;           /* ising_dtype_t of the coupling values */
    const int64_t *row_ptr;  /* CSR: [n + 1] */
    const int32_t *col;      /* CSR: [nnz]; ELL: [n][ell_width] */
    const void *val;         /* CSR: [nnz]; ELL: [n][ell_width] */
    int64_t l_rows, l_cols;  /* TORUS2D */
    const void *right;       /* TORUS2D: [l_rows][l_cols] */
    const void *down;        /* TORUS2D: [l_rows][l_cols] */
    const void *dense;       /* DENSE: [n][n] */
    const void *h;           /* [n] or NULL */
    int32_t htype;           /* ising_dtype_t of h */
    int32_t n_instances;     /* 0 or 1: single instance */
    const int64_t *inst_offset; /* [n_instances + 1] or NULL */
    int64_t ell_width;       /* ELL: slots per row */
} ising_problem_t;

typedef struct ising_context *ising_handle_t;

/*
 * Parameter rule of Eq. alphabeta (Supplementary Note 6), host-side FP64:
 *   alpha = eta * lambda_max(-J),
 *   beta  = n^1.5 * max_j ( alpha + sum_{i != j} |J_ij| ).
 * method 0 = auto (power iteration below n = 1e4, Wigner estimate of
 * Eq. estimate_eig_J from there on, as the paper does), 1 = power
 * iteration on -J shifted by ||J||_inf, 2 = Wigner estimate
 * 2 <J> sqrt(n) with <J> the standard deviation of the n(n-1) off-diagonal
 * entries. Per instance for batched problems: alpha_out and beta_out hold
 * max(1, n_instances) values. Arrays of p must be host pointers here.
 */
ISING_API ising_status_t ising_default_params(const ising_problem_t *p, double eta, int32_t method,
                                    double *alpha_out, double *beta_out);

/*
 * Validate J and h (symmetry, zero diagonal, index ranges, finite values;
 * skipped with ISING_FLAG_SKIP_VALIDATION) and copy them to device memory
 * owned by a new handle. Dense couplings must be integers with |J| <= 256
 * (ISING_ERR_UNSUPPORTED otherwise, whatever their storage type); they are
 * held in the tensor-core tile order, as packed 2-bit codes when every entry
 * is -1, 0 or +1 and as BF16 otherwise (both exact). On failure *out is NULL.
 */
ISING_API ising_status_t ising_create(const ising_problem_t *p, int32_t flags, ising_handle_t *out);

/*
 * Algorithm S5 (Supplementary Note 9) generated on the device, straight into
 * a new handle's CSR arrays (no host copy of J): n spins, p in percent; for
 * every pair i > j, z in {1, ..., N_p} with N_p = floor(102300 / p), and
 * J_ij = J_ji = z - 511 where z < 1023 (stored even when 0). The draw of pair
 * (i, j) is value t = i (i - 1) / 2 + j of the counter-based SplitMix64
 * stream s = mix(seed * 0x9E3779B97F4A7C15 + 13 * 0x94D049BB133111EB):
 * u = mix(s + (t + 1) * 0x9E3779B97F4A7C15), z = 1 + floor(u N_p / 2^64).
 * Couplings are held as int32 (integer energies are exact). Cost: n^2 draws.
 */
ISING_API ising_status_t ising_create_s5(int64_t n, double p, uint64_t seed, int32_t flags, ising_handle_t *out);

/*
 * Procedural dense couplings of Supplementary Note 9 (the benchmark matrix of
 * the paper's 10^6- and 10^7-spin fully connected runs): J_ij = sin(i j + c)
 * for 1-based indices i != j, J_ii = 0, no field. Nothing of J is stored: the
 * kernels generate every coupling where it is used (Algorithm S6's blocks, on
 * one GPU) from an exact integer phase and a minimax polynomial (each FP32
 * coupling within 3.3e-7 of the exact value, rms 6e-8): n^2 / 2 couplings per
 * product for one replica (each serves J_ij x_j and J_ji x_i; order-independent
 * int64 fixed-point sums), n^2 for more.
 *   n       2 .. 2^30 spins;  c  0 .. 2^40 (the paper uses 100).
 * The handle supports ising_iterate (F32 iterates),
 * ising_iterate_adoch (F32), ising_iterate_until (F32), ising_energy (E_f64, cut_f64, best, spins; the
 * sum of J in the cut is evaluated in closed form in FP64) and
 * ising_params_device (Wigner estimate; method 1 is ISING_ERR_UNSUPPORTED).
 * Creation costs O(n) host work (closed-form sums of J and J^2).
 */
ISING_API ising_status_t ising_create_procedural(int64_t n, int64_t c, int32_t flags, ising_handle_t *out);

/*
 * Eq. alphabeta on the device for a one-instance CSR or TORUS2D handle (for
 * problems that exist only on the device): the same rule as
 * ising_default_params (method 0 = auto, 1 = power iteration on -J +
 * ||J||_inf I, 2 = Wigner estimate), with FP64 reductions on the device.
 * PROCEDURAL handles take the Wigner estimate for methods 0 and 2, with the
 * sums of J and J^2 in closed form and the row sums of |J_ij| from one pass
 * over the generated couplings.
 */
ISING_API ising_status_t ising_params_device(ising_handle_t h, double eta, int32_t method, double *alpha_out,
                                   double *beta_out);

/*
 * Copy a CSR handle's device arrays to the caller (host or device): row_ptr
 * [n+1] int64, col [nnz] int32, val [nnz] of the storage type *jtype_out
 * (I8, I32, F32 or F64). Any output may be NULL (nnz_out alone sizes them).
 */
ISING_API ising_status_t ising_csr_export(ising_handle_t h, int64_t *row_ptr, int32_t *col, void *val,
                                int64_t *nnz_out, int32_t *jtype_out);

/* Release the handle and everything it owns. NULL is accepted. */
ISING_API void ising_destroy(ising_handle_t h);

/*
 * DOCH, Algorithm 1, steps 2-4: apply T (Eq. FPE) `iters` times to the R
 * replicas in x, in place (Jacobi: every component of x^(k+1) is computed
 * from x^(k)).
 *   x      [n][R] iterate of type xtype (F32 or F64; BF16 for DENSE), x^(0)
 *          on entry, x^(iters) on return.
 *   alpha  [max(1,n_instances)][alpha_len] host array, alpha_len = 1 (constant
 *          alpha) or iters (a schedule alpha_k, one value per iteration).
 *   beta   [max(1,n_instances)] host array, beta > 0.
 *   H_trace  NULL, or [iters + 1][max(1,n_instances)][R] FP64 receiving
 *          H(x^(k)) of Eq. Hamilton (with -h^T x for a field), each with the
 *          alpha of step k (the last step's for k = iters). Computed in FP64
 *          on the device, fused into the iteration kernel.
 * For DENSE a BF16 iterate runs the coupling product on the tcgen05 tensor
 * cores (FP32 accumulation, BF16 state); an F32 iterate runs the plain FP32
 * form (FP32 products and accumulation on the CUDA cores, FP32 state, CUDA's
 * cbrtf), the reference the BF16 form is compared with. For PROCEDURAL the iterate is
 * F32 and each step generates the couplings; an H_trace costs one more
 * coupling product per step.
 */
ISING_API ising_status_t ising_iterate(ising_handle_t h, void *x, int32_t xtype, int32_t R,
                             const double *alpha, int32_t alpha_len, const double *beta,
                             int32_t iters, double *H_trace, void *stream);

/*
 * ADOCH, Algorithm 2: DOCH with an extrapolated point that is kept only when
 * it passes a non-monotone test on H (Eq. Hamilton):
 *   t_0 = 1, t_(k+1) = (1 + sqrt(1 + 4 t_k^2)) / 2,
 *   y^k = x^k + ((t_k - 1) / t_(k+1)) (x^k - x^(k-1)),  y^0 = x^0,
 *   v^k = y^k if H(y^k) <= max(H(x^max(0,k-q)), ..., H(x^k)), else x^k,
 *   x^(k+1) = T(v^k)  (Eq. FPE).
 * Each step costs one coupling product (J y^k = (1 + c_k) J x^k - c_k J x^(k-1)),
 * FP64 reductions of H(x^k) and H(y^k) per (instance, replica), and the
 * update; the acceptance test runs per (instance, replica) on the device.
 *   x      [n][R] F32 or F64, x^(0) on entry, x^(iters) on return (in place).
 *   alpha, beta  [max(1,n_instances)] host arrays (constant alpha; beta > 0).
 *   q      window of the non-monotone test (q >= 0; q = 0 compares with
 *          H(x^k) alone).
 *   accepted  NULL, or [iters][max(1,n_instances)][R] int8 (host or device):
 *          1 where v^k = y^k.
 *   H_trace   NULL, or [iters + 1][max(1,n_instances)][R] FP64 (host or
 *          device): H(x^(k)) for k = 0 .. iters.
 * CSR, TORUS2D and PROCEDURAL (F32) couplings; ISING_ERR_UNSUPPORTED for
 * DENSE. Device scratch: four iterate-sized buffers plus O(R) reduction
 * space, owned by the handle (two for an FP32 lattice with R = 1, whose
 * passes recompute both coupling products instead of storing them).
 */
ISING_API ising_status_t ising_iterate_adoch(ising_handle_t h, void *x, int32_t xtype, int32_t R,
                                   const double *alpha, const double *beta, int32_t iters, int32_t q,
                                   int8_t *accepted, double *H_trace, void *stream);

/*
 * DOCH (Algorithm 1) with the stopping rule of Remark S2, per (instance,
 * replica) pair: after each step, r^(k) = ||x^(k+1) - x^(k)||_2 / ||x^(k)||_2
 * (compensated FP32 per thread for F32 iterates, FP64 across threads and for
 * F64 iterates); the pair stops at the first k with
 * r^(k) < eps and keeps x^(k+1). Pairs that never meet the rule run
 * max_iters steps.
 *   x      [n][R] F32 or F64 (in place): each pair's last iterate on return.
 *   alpha, beta  [max(1,n_instances)] host arrays (constant alpha).
 *   eps    >= 0 (0 never stops).
 *   steps_out  NULL, or [max(1,n_instances)][R] int32 (host or device): the
 *          steps each pair took.
 * Batched FP32 instances that fit the shared-memory resident kernel apply
 * the rule inside it (FP32 sums per thread and warp, FP64 across warps) and
 * end each instance's replica group once all of its replicas stopped;
 * otherwise the host checks every 8 steps whether any pair still runs and
 * ends the loop when none does. CSR, TORUS2D and PROCEDURAL (F32);
 * ISING_ERR_UNSUPPORTED for DENSE.
 */
ISING_API ising_status_t ising_iterate_until(ising_handle_t h, void *x, int32_t xtype, int32_t R,
                                   const double *alpha, const double *beta, int32_t max_iters, double eps,
                                   int32_t *steps_out, void *stream);

/*
 * Sign rounding (Algorithm 1, step 5: s = sign(x^(N)), sign(0) = +1) and the
 * Ising energy E_r = -1/2 s_r^T J s_r - h^T s_r (Eq. IsingModel) with the cut
 * value cut_r = 1/4 sum_ij (1 - s_i s_j) W_ij for W = -2J (Supplementary
 * Note 5), per instance and replica, plus the best replica argmin_r E_r per
 * instance (first minimum).
 *   x        [n][R] of type xtype: F32/F64/BF16 iterates (rounded here), or
 *            I8 spins (+1/-1).
 *   E_int, cut_int  [max(1,n_instances)][R] int64, exact integer arithmetic;
 *            only for integer J and h (else ISING_ERR_INVALID_ARG). May be NULL.
 *   E_f64, cut_f64  [max(1,n_instances)][R] FP64 with a fixed reduction
 *            order (run-to-run identical). May be NULL.
 *   best     [max(1,n_instances)] int32, or NULL.
 *   spins    [n][R] int8 receiving s, or NULL.
 */
ISING_API ising_status_t ising_energy(ising_handle_t h, const void *x, int32_t xtype, int32_t R,
                            int64_t *E_int, int64_t *cut_int, double *E_f64, double *cut_f64,
                            int32_t *best, int8_t *spins, void *stream);

/*
 * Choice of eta in alpha = eta * lambda_max(-J) by probe iterations
 * (Supplementary Note 6: eta in (0, 2] is tuned by examining the Ising energy
 * over the first few iterations -- 5 to 10 for large graphs, 1 to 3 for
 * ultra-large ones). For a one-instance handle:
 *   alpha1, beta1  Eq. alphabeta at eta = 1 (from ising_default_params or
 *          ising_params_device); beta is affine in alpha, so candidate k uses
 *          alpha_k = etas[k] alpha1 and beta_k = beta1 + n^1.5 (etas[k] - 1) alpha1.
 *   x0     [n][R] start of every probe (xtype as ising_iterate accepts for the
 *          handle's format; host or device); not modified.
 * For each candidate in order: probe_iters DOCH steps from x0 (ising_iterate),
 * then the Ising energies of sign(x) per replica (exact int64 for integer J,
 * FP64 otherwise, as ising_energy). score_best[k] = the lowest energy over the
 * replicas, score_mean[k] = the mean energy; the chosen candidate has the
 * lowest score_best (ties: lower score_mean, then the earlier candidate).
 *   score_best, score_mean  [n_etas] FP64 or NULL;  best_index int32 or NULL;
 *   alpha_out, beta_out     the chosen candidate's alpha and beta, or NULL.
 * Outputs may be host or device pointers. n_etas 1 .. 4096. The handle keeps
 * two iterate-sized scratch buffers for the probes. Synchronises the stream.
 */
ISING_API ising_status_t ising_tune_eta(ising_handle_t h, const void *x0, int32_t xtype, int32_t R,
                                        const double *etas, int32_t n_etas, int32_t probe_iters, double alpha1,
                                        double beta1, double *score_best, double *score_mean, int32_t *best_index,
                                        double *alpha_out, double *beta_out, void *stream);

/*
 * Adjoint of `iters` DOCH steps (derived from Eq. FPE; the paper has no
 * gradients). Loss: the mean relaxed energy of the final iterates,
 *   L = (1/R) sum_r ( -1/2 x_r^T J x_r - h^T x_r ) at x^(iters)
 * (Supplementary Note 2, Eq. E, plus the field term). Computes
 *   grad_alpha[k] = dL/dalpha_k  (k = 0..iters-1)  and  grad_x0 = dL/dx^(0)
 * by the reverse recursion
 *   g^N = -(1/R)(J x^N + h);  w^k = g^(k+1) / (3 (x^(k+1))^2) (0 where x^(k+1) = 0);
 *   dL/dalpha_k = sum w^k x^k / beta;  g^k = (J w^k + alpha_k w^k) / beta,
 * keeping x^(k) only every ckpt_every steps and recomputing each segment.
 *   x0       [n][R] F32 or F64 (CSR, one instance). The forward iterates
 *            (checkpoints and recomputed segments) run in x0's precision; the
 *            adjoint recursion runs in FP32; its sums (dL/dalpha, the loss)
 *            are compensated FP32 per thread for F32 iterates and FP64 across
 *            threads (FP64 throughout for F64 iterates). d x^(k+1)/d x^k
 *            contains 1/(3 (x^(k+1))^2), so components passing near zero in
 *            the transient make the gradient sensitive to the trajectory: F64
 *            gives gradients within ~1e-6 of the exact adjoint from any start,
 *            F32 is exact to ~1e-5 only where the trajectory avoids such
 *            crossings (e.g. from a converged state).
 *   alpha    [iters] (the schedule); beta > 0 host scalar.
 *   grad_alpha  [iters] FP64;  grad_x0  [n][R] of x0's type;  loss  FP64
 *            scalar (all may be host or device; NULL skips an output).
 *   zero_events  int64 scalar or NULL: components where x^(k+1) was exactly 0.
 */
ISING_API ising_status_t ising_backward(ising_handle_t h, const void *x0, int32_t xtype, int32_t R,
                              const double *alpha, int32_t iters, double beta, int32_t ckpt_every,
                              double *grad_alpha, void *grad_x0, double *loss,
                              int64_t *zero_events, void *stream);

/* Wait for the handle's work on `stream` and report deferred device errors. */
ISING_API ising_status_t ising_synchronize(ising_handle_t h, void *stream);

/* Problem size of a handle: total spins and instance count. */
ISING_API ising_status_t ising_get_size(ising_handle_t h, int64_t *n, int32_t *n_instances);

/*
 * Energy and cut of a TORUS2D lattice that allocates no device memory.
 * (The paper has no counterpart: this is a deployment variant of the
 * readout of ising_energy.)
 *
 * For callers that cannot call cudaMalloc -- code whose device memory is
 * owned by another allocator that has reserved the device, or loops in which
 * an allocation (which may synchronise the device) is not acceptable. It
 * needs no handle: the caller passes the lattice couplings right/down
 * ([l_rows][l_cols] int8, as in ising_problem_t), the FP32 iterates x
 * ([n][R], n = l_rows * l_cols) and the outputs E_out / cut_out ([R] int64,
 * either may be NULL), all as DEVICE arrays; host arrays are rejected with
 * ISING_ERR_INVALID_ARG. Computes s = sign(x) (sign(0) = +1), E_r =
 * -1/2 s_r^T J s_r and cut_r with W = -2J exactly in int64, as ising_energy.
 *
 * Its reduction partials live in a fixed device array inside the library
 * (131,072 bytes: two int64 per (replica, chunk of sites), held on every
 * device that loads the library until the process exits), so R is limited
 * to 8192; larger R fails with ISING_ERR_INVALID_ARG. Every array must be
 * memory of the current device; the library cannot check their lengths, so
 * the caller guarantees right/down hold l_rows * l_cols values, x
 * l_rows * l_cols * R and each given output R. The first call on a device looks up that array's
 * address (cudaGetSymbolAddress, with the device current) and caches it;
 * make that first call before any stream capture. Every call shares the
 * array: two calls whose work overlaps on the GPU (different streams, or
 * different host threads) race and may return wrong values. Work is
 * enqueued on `stream` and not waited for.
 */
ISING_API ising_status_t ising_energy_torus_noalloc(const int8_t *right, const int8_t *down,
                                                    int64_t l_rows, int64_t l_cols, const float *x,
                                                    int32_t R, int64_t *E_out, int64_t *cut_out,
                                                    void *stream);

/*
 * Diagnostic: the FP32 cube root of the CSR, batched, dense, procedural and
 * ADOCH kernels, sign(z) 2^(log2|z|/3) evaluated on z 2^(-3k) and rescaled by
 * 2^k, written to ours[i], next to CUDA's cbrtf(z[i]) in ref[i]. z, ours, ref
 * are device arrays of n floats; -40 <= k <= 40. Synchronises the stream.
 */
ISING_API ising_status_t ising_selftest_cbrt(const float *z, float *ours, float *ref, int64_t n,
                                             int32_t k, void *stream);

/*
 * Diagnostic: the FP32 cube root of the lattice DOCH kernels (Eq. FPE's update
 * cbrt(z / beta)), sign(z) 2^(log2|z|/3 + c3) with c3 = log2(1/beta)/3, one
 * FMA between the hardware base-2 logarithm and exponential, written to
 * out[i]. z and out are device arrays of n floats; c3 finite with |c3| <= 64.
 * Synchronises the stream.
 */
ISING_API ising_status_t ising_selftest_cbrt_log(const float *z, float *out, int64_t n, float c3, void *stream);

/*
 * Diagnostic: the procedural couplings J_ij = sin(i j + c) (1-based i, j;
 * J_ii = 0) for rows row0 .. row0 + rows - 1 and columns col0 .. col0 + cols - 1
 * (0-based indices), evaluated on the device exactly as the product kernels of
 * an ising_create_procedural handle generate them (64-bit phase every 32nd
 * column from col0, 32-bit increments in between), into J_out [rows][cols]
 * FP32 (device array). Indices below 2^30, c in 0 .. 2^40. Synchronises the
 * stream.
 */
ISING_API ising_status_t ising_selftest_procedural(int64_t row0, int32_t rows, int64_t col0, int32_t cols,
                                                   int64_t c, float *J_out, void *stream);

/*
 * Diagnostic of the failure path of bounded device waits (the paper has no
 * counterpart): launches one thread that waits on a shared-memory mbarrier
 * with the bounded wait the tensor-core kernel uses, limit limit_ns
 * (1e3 .. 1e9 ns). With arrive = 0 nothing ever arrives, the wait gives up
 * after the limit, sets the timeout bit of the handle's device error word,
 * and the call returns ISING_ERR_TIMEOUT; the error word is then cleared and
 * the handle stays usable. With arrive != 0 the thread arrives first and the
 * call returns ISING_OK. No trap, no fault: the kernel simply returns.
 * Synchronises the stream.
 */
ISING_API ising_status_t ising_selftest_wait(ising_handle_t h, int32_t arrive, int64_t limit_ns, void *stream);

/* Static description of a status code. */
ISING_API const char *ising_status_string(ising_status_t s);

/* Message of the calling thread's last failed call ("" if none). */
ISING_API const char *ising_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ISING_DOCH_H */
