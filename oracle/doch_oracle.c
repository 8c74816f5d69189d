/*
 * FP64 oracle for the DOCH Ising solver -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded restatement of what the method computes,
 * used to check the CUDA path. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the product path never does.
 * It shares no code, header or table with the CUDA library.
 *
 * Paper: "A Continuous Energy Ising Machine Leveraging Difference-of-Convex
 * Programming" (arXiv 2509.01928). Notation follows the paper:
 *   E(s) = -1/2 s^T J s - h^T s                       (Eq. IsingModel)
 *   H(x) = beta/4 sum x^4 - alpha/2 sum x^2 - 1/2 x^T J x  (Eq. Hamilton)
 *        = f(x) - g(x),  f = beta/4 sum x^4,  g = 1/2 x^T (J + alpha I) x
 *   T(x) = cbrt( beta^-1 (J + alpha I) x )             (Eq. FPE)
 *   DOCH: x^(k+1) = T(x^(k)), k = 0..N-1; s = sign(x^(N))  (Algorithm 1)
 *
 * Readings where the paper is silent:
 *   - external field h: kept inside the convex part g (g = 1/2 x^T(J+aI)x + h^T x),
 *     so the DCA first-order condition of Eq. optcon gives
 *     beta x^3 = (J + alpha I) x + h, i.e. T(x) = cbrt((Jx + alpha x + h)/beta).
 *   - sign(0) = +1.
 *   - cut weights: W = -2 J (Supplementary Note 5 sets J = -W/2).
 *   - alpha may follow a schedule alpha_k (one value per iteration); beta is fixed.
 *   - relaxed-energy loss for the adjoint: L = (1/R) sum_r (-1/2 x_r^T J x_r - h^T x_r)
 *     at x^(N) (relaxed energy of Supplementary Note 2, Eq. E, plus the field term).
 *
 * Layout: every state array is [n][R] row-major (the R replicas of spin i
 * are contiguous), R >= 1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Coupling matrix J (symmetric, zero diagonal) in one of three forms. */
enum { ORC_CSR = 0, ORC_TORUS = 1, ORC_DENSE = 2 };

typedef struct {
    int64_t n;
    int32_t form;
    int32_t pad_;
    /* CSR: row i holds col[row_ptr[i] .. row_ptr[i+1]) with values val[] */
    const int64_t *row_ptr;
    const int32_t *col;
    const double *val;
    const int64_t *ival;      /* same values as int64 (integer couplings), or NULL */
    /* torus: right[r][c] couples (r,c)-(r,c+1 mod Lc); down[r][c] couples (r,c)-(r+1 mod Lr,c) */
    int64_t l_rows, l_cols;
    const double *right, *down;
    const int64_t *iright, *idown;
    /* dense: row-major n*n */
    const double *dense;
    const int64_t *idense;
    /* external field h[n], or NULL for h = 0 */
    const double *h;
    const int64_t *ih;
} orc_problem;

/* ------------------------------------------------------------------------
 * Coupling product u = J x for all R replicas (the linear part of Eq. FPE).
 * ---------------------------------------------------------------------- */
void orc_coupling_product(const orc_problem *p, int R, const double *x, double *u)
{
    const int64_t n = p->n;
    memset(u, 0, sizeof(double) * (size_t)n * (size_t)R);
    if (p->form == ORC_CSR) {
        for (int64_t i = 0; i < n; ++i)
            for (int64_t e = p->row_ptr[i]; e < p->row_ptr[i + 1]; ++e) {
                const int64_t j = p->col[e];
                for (int r = 0; r < R; ++r)
                    u[i * R + r] += p->val[e] * x[j * R + r];
            }
    } else if (p->form == ORC_TORUS) {
        /* every lattice edge (a, b) with weight w adds w*x_b to u_a and w*x_a to u_b */
        const int64_t Lr = p->l_rows, Lc = p->l_cols;
        for (int64_t rr = 0; rr < Lr; ++rr)
            for (int64_t c = 0; c < Lc; ++c) {
                const int64_t a = rr * Lc + c;
                const int64_t b_right = rr * Lc + (c + 1) % Lc;
                const int64_t b_down = ((rr + 1) % Lr) * Lc + c;
                const double wr = p->right[a], wd = p->down[a];
                for (int r = 0; r < R; ++r) {
                    u[a * R + r] += wr * x[b_right * R + r];
                    u[b_right * R + r] += wr * x[a * R + r];
                    u[a * R + r] += wd * x[b_down * R + r];
                    u[b_down * R + r] += wd * x[a * R + r];
                }
            }
    } else {
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = 0; j < n; ++j) {
                const double w = p->dense[i * n + j];
                for (int r = 0; r < R; ++r)
                    u[i * R + r] += w * x[j * R + r];
            }
    }
}

/* ------------------------------------------------------------------------
 * Hamiltonian H(x) per replica (Eq. Hamilton, plus -h^T x for the field).
 * ---------------------------------------------------------------------- */
void orc_hamiltonian(const orc_problem *p, int R, const double *x, double alpha,
                     double beta, double *H)
{
    const int64_t n = p->n;
    double *u = (double *)malloc(sizeof(double) * (size_t)n * (size_t)R);
    orc_coupling_product(p, R, x, u);
    for (int r = 0; r < R; ++r) {
        double s4 = 0.0, s2 = 0.0, xjx = 0.0, hx = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            const double xi = x[i * R + r];
            s4 += xi * xi * xi * xi;
            s2 += xi * xi;
            xjx += xi * u[i * R + r];
            if (p->h) hx += p->h[i] * xi;
        }
        H[r] = beta / 4.0 * s4 - alpha / 2.0 * s2 - 0.5 * xjx - hx;
    }
    free(u);
}

/* ------------------------------------------------------------------------
 * DOCH, Algorithm 1: N applications of T (Eq. FPE), Jacobi (every component
 * of x^(k+1) from x^(k)). alpha has alpha_len = 1 (constant) or iters values.
 * H_trace (nullable) receives H(x^(k)) for k = 0..iters, each evaluated with
 * the alpha of step k (the last step's alpha for k = iters); [iters+1][R].
 * x holds x^(0) on entry and x^(N) on return.
 * ---------------------------------------------------------------------- */
int orc_doch(const orc_problem *p, int R, double *x, const double *alpha, int alpha_len,
             double beta, int iters, double *H_trace)
{
    const int64_t n = p->n;
    if (R < 1 || iters < 0 || beta <= 0.0 || (alpha_len != 1 && alpha_len != iters))
        return 1;
    double *u = (double *)malloc(sizeof(double) * (size_t)n * (size_t)R);
    if (!u) return 2;
    for (int k = 0; k < iters; ++k) {
        const double a = alpha[alpha_len == 1 ? 0 : k];
        if (H_trace) orc_hamiltonian(p, R, x, a, beta, H_trace + (size_t)k * R);
        orc_coupling_product(p, R, x, u);
        for (int64_t i = 0; i < n; ++i)
            for (int r = 0; r < R; ++r) {
                const double hi = p->h ? p->h[i] : 0.0;
                const double z = (u[i * R + r] + a * x[i * R + r] + hi) / beta;
                x[i * R + r] = cbrt(z);
            }
    }
    if (H_trace && iters > 0)
        orc_hamiltonian(p, R, x, alpha[alpha_len == 1 ? 0 : iters - 1], beta,
                        H_trace + (size_t)iters * R);
    free(u);
    return 0;
}

/* sign with sign(0) = +1 (Algorithm 1, return step) */
void orc_sign(int64_t count, const double *x, int8_t *s)
{
    for (int64_t t = 0; t < count; ++t) s[t] = x[t] >= 0.0 ? 1 : -1;
}

/* ------------------------------------------------------------------------
 * Ising energy (Eq. IsingModel) and cut (Supplementary Note 5, W = -2J), FP64.
 * E_r = -1/2 sum_{i,j} J_ij s_i s_j - sum_i h_i s_i
 * cut_r = 1/4 sum_{i,j} (1 - s_i s_j) W_ij
 * ---------------------------------------------------------------------- */
void orc_energy(const orc_problem *p, int R, const int8_t *s, double *E, double *cut)
{
    const int64_t n = p->n;
    for (int r = 0; r < R; ++r) {
        double quad = 0.0, field = 0.0, cw = 0.0;
        if (p->form == ORC_TORUS) {
            const int64_t Lr = p->l_rows, Lc = p->l_cols;
            for (int64_t rr = 0; rr < Lr; ++rr)
                for (int64_t c = 0; c < Lc; ++c) {
                    const int64_t a = rr * Lc + c;
                    const int64_t br = rr * Lc + (c + 1) % Lc;
                    const int64_t bd = ((rr + 1) % Lr) * Lc + c;
                    /* each edge appears twice in sum_{i,j}: J_ab and J_ba */
                    quad += 2.0 * p->right[a] * s[a * R + r] * s[br * R + r];
                    quad += 2.0 * p->down[a] * s[a * R + r] * s[bd * R + r];
                    cw += 2.0 * (1 - s[a * R + r] * s[br * R + r]) * (-2.0 * p->right[a]);
                    cw += 2.0 * (1 - s[a * R + r] * s[bd * R + r]) * (-2.0 * p->down[a]);
                }
        } else {
            for (int64_t i = 0; i < n; ++i) {
                if (p->form == ORC_CSR) {
                    for (int64_t e = p->row_ptr[i]; e < p->row_ptr[i + 1]; ++e) {
                        const int64_t j = p->col[e];
                        const double sij = (double)s[i * R + r] * s[j * R + r];
                        quad += p->val[e] * sij;
                        cw += (1.0 - sij) * (-2.0 * p->val[e]);
                    }
                } else {
                    for (int64_t j = 0; j < n; ++j) {
                        const double sij = (double)s[i * R + r] * s[j * R + r];
                        quad += p->dense[i * n + j] * sij;
                        cw += (1.0 - sij) * (-2.0 * p->dense[i * n + j]);
                    }
                }
            }
        }
        if (p->h)
            for (int64_t i = 0; i < n; ++i) field += p->h[i] * s[i * R + r];
        E[r] = -0.5 * quad - field;
        cut[r] = 0.25 * cw;
    }
}

/* Same definitions in exact int64 arithmetic, for integer couplings and field
 * (the i* arrays of the problem). */
void orc_energy_int(const orc_problem *p, int R, const int8_t *s, int64_t *E, int64_t *cut)
{
    const int64_t n = p->n;
    for (int r = 0; r < R; ++r) {
        int64_t quad = 0, field = 0, cw = 0;
        if (p->form == ORC_TORUS) {
            const int64_t Lr = p->l_rows, Lc = p->l_cols;
            for (int64_t rr = 0; rr < Lr; ++rr)
                for (int64_t c = 0; c < Lc; ++c) {
                    const int64_t a = rr * Lc + c;
                    const int64_t br = rr * Lc + (c + 1) % Lc;
                    const int64_t bd = ((rr + 1) % Lr) * Lc + c;
                    const int64_t s_ar = (int64_t)s[a * R + r] * s[br * R + r];
                    const int64_t s_ad = (int64_t)s[a * R + r] * s[bd * R + r];
                    quad += 2 * p->iright[a] * s_ar + 2 * p->idown[a] * s_ad;
                    cw += 2 * (1 - s_ar) * (-2 * p->iright[a]) + 2 * (1 - s_ad) * (-2 * p->idown[a]);
                }
        } else {
            for (int64_t i = 0; i < n; ++i) {
                if (p->form == ORC_CSR) {
                    for (int64_t e = p->row_ptr[i]; e < p->row_ptr[i + 1]; ++e) {
                        const int64_t j = p->col[e];
                        const int64_t sij = (int64_t)s[i * R + r] * s[j * R + r];
                        quad += p->ival[e] * sij;
                        cw += (1 - sij) * (-2 * p->ival[e]);
                    }
                } else {
                    for (int64_t j = 0; j < n; ++j) {
                        const int64_t sij = (int64_t)s[i * R + r] * s[j * R + r];
                        quad += p->idense[i * n + j] * sij;
                        cw += (1 - sij) * (-2 * p->idense[i * n + j]);
                    }
                }
            }
        }
        if (p->ih)
            for (int64_t i = 0; i < n; ++i) field += p->ih[i] * s[i * R + r];
        /* quad = s^T J s is even (J symmetric, zero diagonal), cw is a multiple of 4 */
        E[r] = -(quad / 2) - field;
        cut[r] = cw / 4;
    }
}

/* ------------------------------------------------------------------------
 * Adjoint of N DOCH steps (derived from Eq. FPE; the paper has no gradients).
 * Loss L = (1/R) sum_r ( -1/2 x_r^T J x_r - h^T x_r ) at x^(N).
 *   g^N = dL/dx^N = -(1/R) (J x^N + h)
 *   for k = N-1 .. 0:
 *     x^(k+1) = cbrt(z^k), z^k = (J x^k + alpha_k x^k + h)/beta
 *     w^k = g^(k+1) * d cbrt(z)/dz = g^(k+1) / (3 (x^(k+1))^2)   (0 where x^(k+1) = 0)
 *     dL/dalpha_k = sum_{i,r} w^k_ir x^k_ir / beta
 *     g^k = (J w^k + alpha_k w^k) / beta                (J = J^T)
 *   dL/dx^0 = g^0
 * Replicas are independent, so each replica is processed on its own with all
 * of its iterates stored (no checkpointing); contributions to dL/dalpha are
 * summed in replica order. zero_events counts components with x^(k+1) = 0.
 * alpha has iters values. grad_x0 is [n][R].
 * ---------------------------------------------------------------------- */
int orc_backward(const orc_problem *p, int R, const double *x0, const double *alpha, double beta,
                 int iters, double *grad_alpha, double *grad_x0, double *loss, int64_t *zero_events)
{
    const int64_t n = p->n;
    if (R < 1 || iters < 0 || beta <= 0.0) return 1;
    double *xs = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(iters + 1));
    double *u = (double *)malloc(sizeof(double) * (size_t)n);
    double *g = (double *)malloc(sizeof(double) * (size_t)n);
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    if (!xs || !u || !g || !w) { free(xs); free(u); free(g); free(w); return 2; }
    for (int k = 0; k < iters; ++k) grad_alpha[k] = 0.0;
    double L = 0.0;
    int64_t zeros = 0;
    for (int r = 0; r < R; ++r) {
        /* forward, one replica (R = 1 view of the problem) */
        for (int64_t i = 0; i < n; ++i) xs[i] = x0[i * R + r];
        for (int k = 0; k < iters; ++k) {
            const double *xk = xs + (size_t)k * n;
            double *xk1 = xs + (size_t)(k + 1) * n;
            orc_coupling_product(p, 1, xk, u);
            for (int64_t i = 0; i < n; ++i) {
                const double hi = p->h ? p->h[i] : 0.0;
                xk1[i] = cbrt((u[i] + alpha[k] * xk[i] + hi) / beta);
            }
        }
        /* loss and g^N */
        const double *xN = xs + (size_t)iters * n;
        orc_coupling_product(p, 1, xN, u);
        double lr = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            const double hi = p->h ? p->h[i] : 0.0;
            lr += -0.5 * xN[i] * u[i] - hi * xN[i];
            g[i] = -(u[i] + hi) / R;
        }
        L += lr / R;
        /* backward */
        for (int k = iters - 1; k >= 0; --k) {
            const double *xk = xs + (size_t)k * n;
            const double *xk1 = xs + (size_t)(k + 1) * n;
            double ga = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                if (xk1[i] == 0.0) { w[i] = 0.0; ++zeros; }
                else w[i] = g[i] / (3.0 * xk1[i] * xk1[i]);
                ga += w[i] * xk[i];
            }
            grad_alpha[k] += ga / beta;
            orc_coupling_product(p, 1, w, u);
            for (int64_t i = 0; i < n; ++i) g[i] = (u[i] + alpha[k] * w[i]) / beta;
        }
        for (int64_t i = 0; i < n; ++i) grad_x0[i * R + r] = g[i];
    }
    *loss = L;
    if (zero_events) *zero_events = zeros;
    free(xs); free(u); free(g); free(w);
    return 0;
}

/* ------------------------------------------------------------------------
 * The same adjoint recursion (loss, g^N, then k = N-1 .. 0 as in
 * orc_backward) for ONE replica along a GIVEN trajectory xs = x^(0..N)
 * ([N+1][n], e.g. iterates computed in another precision), instead of the
 * trajectory this file computes itself. R is the replica count of the mean
 * in L (the loss and g^N carry 1/R). Adds this replica's dL/dalpha_k into
 * grad_alpha [N], writes its dL/dx^0 into grad_x0 [n], adds its share of L
 * into *loss and its count of components with x^(k+1) = 0 into *zero_events.
 * ---------------------------------------------------------------------- */
int orc_adjoint_along(const orc_problem *p, int R, const double *xs, const double *alpha,
                      double beta, int iters, double *grad_alpha, double *grad_x0, double *loss,
                      int64_t *zero_events)
{
    const int64_t n = p->n;
    if (R < 1 || iters < 0 || beta <= 0.0) return 1;
    double *u = (double *)malloc(sizeof(double) * (size_t)n);
    double *g = (double *)malloc(sizeof(double) * (size_t)n);
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    if (!u || !g || !w) { free(u); free(g); free(w); return 2; }
    const double *xN = xs + (size_t)iters * n;
    orc_coupling_product(p, 1, xN, u);
    double lr = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double hi = p->h ? p->h[i] : 0.0;
        lr += -0.5 * xN[i] * u[i] - hi * xN[i];
        g[i] = -(u[i] + hi) / R;
    }
    *loss += lr / R;
    int64_t zeros = 0;
    for (int k = iters - 1; k >= 0; --k) {
        const double *xk = xs + (size_t)k * n;
        const double *xk1 = xs + (size_t)(k + 1) * n;
        double ga = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            if (xk1[i] == 0.0) { w[i] = 0.0; ++zeros; }
            else w[i] = g[i] / (3.0 * xk1[i] * xk1[i]);
            ga += w[i] * xk[i];
        }
        grad_alpha[k] += ga / beta;
        orc_coupling_product(p, 1, w, u);
        for (int64_t i = 0; i < n; ++i) g[i] = (u[i] + alpha[k] * w[i]) / beta;
    }
    for (int64_t i = 0; i < n; ++i) grad_x0[i] = g[i];
    if (zero_events) *zero_events += zeros;
    free(u); free(g); free(w);
    return 0;
}
