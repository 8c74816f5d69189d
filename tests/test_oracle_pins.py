"""Pins for the FP64 oracle, against facts the paper and the mathematics fix.

None of these checks re-types the oracle's own formula: each one compares it
with a worked example of the paper, a closed form, a proposition of the
supplementary notes, an independent dense/brute-force computation, or a
finite-difference / forward-mode derivative.
"""
import itertools
import os

import numpy as np
import pytest

import oracle as O
from paper_2509_01928_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *v = line.split()
            out[k] = [float(t) for t in v]
    return out


def _sk(n, seed):
    """Gaussian (SK-like) dense symmetric J with zero diagonal, from the input streams."""
    g = I.gaussian(I.stream_seed(seed, 50), I.stream_seed(seed, 51), 0, n * n).reshape(n, n)
    J = np.triu(g, 1)
    return J + J.T


def _all_spins(n):
    """All 2^n spin vectors as rows, +-1 int8."""
    return np.array(list(itertools.product([-1, 1], repeat=n)), dtype=np.int8)


# ---------------------------------------------------------------------------
# worked example (Figure 3 caption)
# ---------------------------------------------------------------------------

def test_two_spin_worked_example():
    g = _golden("two_spin_fig3.txt")
    J = np.array([[0.0, g["J12"][0]], [g["J12"][0], 0.0]])
    alpha, beta = g["alpha"][0], g["beta"][0]
    p = O.Problem(J)
    ga, gb = np.array(g["ground_state_a"]), np.array(g["ground_state_b"])
    k5 = int(g["iterations_to_converge"][0])
    xs = np.linspace(-1, 1, 9)
    starts = np.array([(a, b) for a in xs for b in xs if abs(a - b) >= 0.2]).T  # [2][R]
    x5 = O.doch(p, starts, alpha, beta, k5)
    x60 = O.doch(p, starts, alpha, beta, 60)
    for r in range(starts.shape[1]):
        target = ga if starts[0, r] > starts[1, r] else gb
        assert np.max(np.abs(x5[:, r] - target)) < 1e-2
        assert np.max(np.abs(x60[:, r] - target)) < 1e-12
    # the returned spins are ground states of E(s) = s1 s2 (energy -1)
    E, _ = O.energy(p, O.sign(x60))
    assert np.all(E == -1.0)


# ---------------------------------------------------------------------------
# closed-form binary fixed points: x = c * s with beta c^2 = alpha + (J s)_i s_i
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d", [3, 4, 7])
def test_ferromagnetic_regular_fixed_point(d):
    g = I.regular_pm1(40, d, seed=11)
    g.val = np.ones_like(g.val)  # J = +1 on every edge
    alpha, beta = O.alpha_beta(g, eta=1.0, method="eig")
    c = np.sqrt((d + alpha) / beta)
    x = np.full((g.n, 2), c)
    x[:, 1] = -c
    out = O.doch(O.Problem(g), x, alpha, beta, 1)
    np.testing.assert_allclose(out, x, rtol=4e-16, atol=0)


def test_antiferromagnetic_checkerboard_fixed_point():
    lr, lc = 6, 8
    t = I.Torus2D(-np.ones((lr, lc), np.int8), -np.ones((lr, lc), np.int8))
    alpha, beta = O.alpha_beta(t, eta=1.0, method="eig")
    c = np.sqrt((4 + alpha) / beta)
    rr, cc = np.meshgrid(np.arange(lr), np.arange(lc), indexing="ij")
    x = (c * np.where((rr + cc) % 2 == 0, 1.0, -1.0)).reshape(-1, 1)
    out = O.doch(O.Problem(t), x, alpha, beta, 1)
    np.testing.assert_allclose(out, x, rtol=4e-16, atol=0)
    # and the checkerboard is the ground state: every edge satisfied, E = -2n
    E, cut = O.energy_int(O.Problem(t), np.sign(x).astype(np.int8))
    assert E[0] == -2 * lr * lc
    assert cut[0] == 2 * 2 * lr * lc  # W = -2J = +2 on every one of the 2n edges


# ---------------------------------------------------------------------------
# three storage forms of one J agree with a dense matrix product
# ---------------------------------------------------------------------------

def test_coupling_product_forms_agree():
    t = I.torus_pm1(5, 7, seed=3)
    csr = t.to_csr()
    dense = csr.to_dense()
    x = I.x0_uniform(t.n, 3, seed=4, dtype=np.float64)
    ref = dense @ x
    for J in (t, csr, dense):
        np.testing.assert_allclose(O.coupling_product(O.Problem(J), x), ref, rtol=0, atol=1e-15)
    # the torus neighbour structure itself: site (r,c) couples to its four neighbours
    lr, lc = t.shape
    for r in range(lr):
        for c in range(lc):
            i = r * lc + c
            expect = {r * lc + (c + 1) % lc: t.right[r, c], r * lc + (c - 1) % lc: t.right[r, c - 1],
                      ((r + 1) % lr) * lc + c: t.down[r, c], ((r - 1) % lr) * lc + c: t.down[r - 1, c]}
            row = {j: dense[i, j] for j in np.nonzero(dense[i])[0]}
            assert row == {k: float(v) for k, v in expect.items()}


# ---------------------------------------------------------------------------
# beta-homogeneity (h = 0): x'^k = c_k x^k with c_(k+1) = (c_k beta/beta')^(1/3)
# ---------------------------------------------------------------------------

def test_beta_homogeneity():
    g = I.erdos_renyi_pm1(50, 0.2, seed=5)
    p = O.Problem(g)
    alpha, beta = O.alpha_beta(g)
    beta2 = beta * 37.0
    x0 = I.x0_uniform(g.n, 4, seed=6, dtype=np.float64)
    c = 1.0
    for k in range(1, 8):
        c = (c * beta / beta2) ** (1.0 / 3.0)
        xa = O.doch(p, x0, alpha, beta, k)
        xb = O.doch(p, x0, alpha, beta2, k)
        np.testing.assert_allclose(xb, c * xa, rtol=1e-12, atol=0)
        assert np.array_equal(np.sign(xa), np.sign(xb))


# ---------------------------------------------------------------------------
# Proposition S5 (monotone descent with the mu/2 ||dx||^2 bound),
# Proposition S6 (vanishing steps), Proposition S8 (bounded iterates)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("beta_scale", ["paper", "small"])
def test_monotone_descent_quantitative(beta_scale):
    J = _sk(40, seed=7)
    p = O.Problem(J)
    eta = 1.3
    alpha, beta = O.alpha_beta(J, eta=eta, method="eig")
    if beta_scale == "small":
        beta = alpha + np.abs(J).sum(axis=1).max()  # ||J + alpha I||_inf, Prop. S8's bound
    mu = np.linalg.eigvalsh(J + alpha * np.eye(40))[0]
    assert mu > 0
    x0 = I.x0_uniform(40, 6, seed=8, dtype=np.float64)
    x = x0.copy()
    for _ in range(60):
        H0 = O.hamiltonian(p, x, alpha, beta)
        x1 = O.doch(p, x, alpha, beta, 1)
        H1 = O.hamiltonian(p, x1, alpha, beta)
        scale = np.abs(H0).max() + 1e-300
        drop = H0 - H1
        bound = mu / 2 * ((x1 - x) ** 2).sum(axis=0)
        assert np.all(drop >= bound - 1e-12 * scale)
        x = x1
    # the H trace returned by the oracle is non-increasing as well
    _, H = O.doch(p, x0, alpha, beta, 5, trace=True)
    assert np.all(np.diff(H, axis=0) <= 1e-12 * np.abs(H).max())


def test_descent_with_field():
    """With a field inside g, DOCH still descends H(x) - h^T x (reading of Eq. optcon)."""
    J = _sk(30, seed=9)
    h = 0.5 * I.gaussian(I.stream_seed(9, 60), I.stream_seed(9, 61), 0, 30)
    p = O.Problem(J, h)
    alpha, beta = O.alpha_beta(J, eta=1.2, method="eig")
    beta = beta / 30 ** 1.5  # a small beta gives a long transient
    x = I.x0_uniform(30, 4, seed=10, dtype=np.float64)
    prev = O.hamiltonian(p, x, alpha, beta)
    for _ in range(40):
        x = O.doch(p, x, alpha, beta, 1)
        cur = O.hamiltonian(p, x, alpha, beta)
        assert np.all(cur <= prev + 1e-12 * np.abs(prev).max())
        prev = cur
    # the limit satisfies beta x^3 = (J + alpha I) x + h (Eq. optcon with h in g)
    x = O.doch(p, x, alpha, beta, 400)
    lhs = beta * x ** 3
    rhs = J @ x + alpha * x + h[:, None]
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-9 * np.abs(rhs).max())


def test_bounded_iterates_any_alpha():
    g = I.erdos_renyi_pm1(60, 0.15, seed=12)
    p = O.Problem(g)
    lam = O.lambda_max_neg(g)
    alpha = 0.3 * lam  # g(x) not convex: only Proposition S8 applies
    beta = alpha + np.abs(g.to_dense()).sum(axis=1).max()
    x0 = 5.0 * I.x0_uniform(60, 5, seed=13, dtype=np.float64)
    bound = max(1.0, np.abs(x0).max())
    x = x0
    for _ in range(50):
        x = O.doch(p, x, alpha, beta, 1)
        assert np.abs(x).max() <= bound * (1 + 1e-15)
    # with the small-beta bound, ||x^(k+1)||_inf <= ||x^k||_inf^(1/3) step by step
    x = x0
    for _ in range(10):
        x1 = O.doch(p, x, alpha, beta, 1)
        assert np.abs(x1).max() <= np.abs(x).max() ** (1 / 3) * (1 + 1e-15)
        x = x1


def test_steps_vanish_and_fixed_point_identity():
    J = _sk(50, seed=14)
    p = O.Problem(J)
    alpha, beta = O.alpha_beta(J, eta=1.0, method="eig")
    x0 = I.x0_uniform(50, 4, seed=15, dtype=np.float64)
    x = O.doch(p, x0, alpha, beta, 300)
    x1 = O.doch(p, x, alpha, beta, 1)
    assert np.all(np.linalg.norm(x1 - x, axis=0) <= 1e-12 * np.linalg.norm(x, axis=0))
    np.testing.assert_allclose(beta * x ** 3, J @ x + alpha * x, rtol=0,
                               atol=1e-10 * np.abs(alpha * x).max())


def test_attractor_minimizers():
    """Proposition S2: with J = 0 the iteration settles on {-lam, +lam}^n, lam = sqrt(alpha/beta)."""
    n = 16
    p = O.Problem(np.zeros((n, n)))
    alpha, beta = 2.5, 40.0
    x0 = I.x0_uniform(n, 3, seed=16, dtype=np.float64)
    x = O.doch(p, x0, alpha, beta, 80)
    lam = np.sqrt(alpha / beta)
    np.testing.assert_allclose(np.abs(x), lam, rtol=1e-12)
    assert np.array_equal(np.sign(x), np.sign(x0))


# ---------------------------------------------------------------------------
# energy and cut: brute force, Max-Cut identity, homogeneous reduction
# ---------------------------------------------------------------------------

def _int_instance(n, seed, with_h=True):
    u = I.splitmix64(I.stream_seed(seed, 70), 0, n * n + n)
    J = np.triu((u[:n * n] % np.uint64(7)).astype(np.int64).reshape(n, n) - 3, 1)
    J = J + J.T
    h = (u[n * n:] % np.uint64(5)).astype(np.int64) - 2 if with_h else None
    return J, h


def test_energy_brute_force_integer():
    n = 14
    J, h = _int_instance(n, seed=17)
    S = _all_spins(n)                     # [2^n][n]
    direct = -0.5 * np.einsum("ri,ij,rj->r", S.astype(np.int64), J, S.astype(np.int64)) - S @ h
    E, cut = O.energy_int(O.Problem(J, h), S.T.copy())
    assert np.array_equal(E, direct.astype(np.int64))
    Ef, _ = O.energy(O.Problem(J, h), S.T.copy())
    assert np.array_equal(Ef, direct.astype(np.float64))


def test_energy_brute_force_gaussian():
    n = 12
    J = _sk(n, seed=18)
    h = I.gaussian(I.stream_seed(18, 80), I.stream_seed(18, 81), 0, n)
    S = _all_spins(n).astype(np.float64)
    direct = -0.5 * np.einsum("ri,ij,rj->r", S, J, S) - S @ h
    E, _ = O.energy(O.Problem(J, h), S.T.astype(np.int8).copy())
    np.testing.assert_allclose(E, direct, rtol=1e-12, atol=1e-12)


def test_cut_identity_and_direct_count():
    g = I.erdos_renyi_pm1(60, 0.1, seed=19)
    p = O.Problem(g)
    W = -2 * g.to_dense().astype(np.int64)
    S = np.where(I.uniform01(I.stream_seed(19, 90), 0, 60 * 16) < 0.5, -1, 1).astype(np.int8)
    S = S.reshape(60, 16)
    E, cut = O.energy_int(p, S)
    w_tot = np.triu(W, 1).sum()            # total weight, each edge once
    assert w_tot % 2 == 0
    assert np.array_equal(cut, w_tot // 2 - E)
    for r in range(16):
        s = S[:, r]
        across = s[:, None] != s[None, :]
        assert cut[r] == np.triu(W * across, 1).sum()
    # torus form gives the same numbers as its CSR form
    t = I.torus_pm1(6, 5, seed=20)
    St = S[:30]
    assert [a.tolist() for a in O.energy_int(O.Problem(t), St)] == \
           [a.tolist() for a in O.energy_int(O.Problem(t.to_csr()), St)]


def test_homogeneous_reduction():
    """Supplementary Note 1, Proposition S1: E_hat((s, t)) = E(t s), and the
    ground state of the (n+1)-spin zero-field model gives that of the field model."""
    n = 11
    J, h = _int_instance(n, seed=21)
    Jhat = np.zeros((n + 1, n + 1), dtype=np.int64)
    Jhat[:n, :n] = J
    Jhat[:n, n] = h
    Jhat[n, :n] = h
    S = _all_spins(n + 1)
    Ehat, _ = O.energy_int(O.Problem(Jhat), S.T.copy())
    ts = (S[:, :n] * S[:, n:n + 1]).astype(np.int8)      # t * s
    E, _ = O.energy_int(O.Problem(J, h), ts.T.copy())
    assert np.array_equal(Ehat, E)
    g = np.argmin(Ehat)
    s_star = S[g, :n] * S[g, n]
    Ef, _ = O.energy_int(O.Problem(J, h), _all_spins(n).T.copy())
    E_star, _ = O.energy_int(O.Problem(J, h), s_star.reshape(-1, 1).astype(np.int8))
    assert E_star[0] == Ef.min()


def test_doch_never_below_ground_state():
    n = 16
    J = _sk(n, seed=22)
    p = O.Problem(J)
    alpha, beta = O.alpha_beta(J, eta=1.0, method="eig")
    Eall, _ = O.energy(p, _all_spins(n).T.copy())
    x = O.doch(p, I.x0_uniform(n, 64, seed=23, dtype=np.float64), alpha, beta, 100)
    E, _ = O.energy(p, O.sign(x))
    assert np.all(E >= Eall.min() - 1e-12)
    assert E.min() <= np.sort(Eall)[int(0.01 * Eall.size)]  # best replica is in the lowest 1 %


def test_sign_of_zero_is_plus_one():
    s = O.sign(np.array([[0.0, -0.0], [1e-300, -1e-300]]))
    assert s.tolist() == [[1, 1], [1, -1]]


# ---------------------------------------------------------------------------
# parameter rule (Eq. alphabeta, Eq. estimate_eig_J)
# ---------------------------------------------------------------------------

def test_params_convexity_and_beta():
    g = I.erdos_renyi_pm1(200, 0.06, seed=24)
    alpha, beta = O.alpha_beta(g, eta=1.0, method="eig")
    D = g.to_dense()
    assert np.linalg.eigvalsh(D + alpha * np.eye(200))[0] >= -1e-9
    assert np.linalg.eigvalsh(D + 0.98 * alpha * np.eye(200))[0] < 0
    assert beta == pytest.approx(200 ** 1.5 * (alpha + np.abs(D).sum(axis=1).max()), rel=1e-15)


def test_wigner_estimate_k2000_c0():
    gld = _golden("k2000_bsb_c0.txt")
    n = int(gld["n"][0])
    J = I.dense_pm1(n, seed=25)
    lam = O.wigner_lambda(J)            # = 2 <J> sqrt(n)
    c0 = 1.0 / lam                      # = 1 / (2 <J> sqrt(n))
    assert c0 == pytest.approx(gld["c0"][0], rel=gld["rel_tol"][0])
    # semicircle edge: the estimate is within a few percent of the true lambda_max(-J)
    assert lam == pytest.approx(O.lambda_max_neg(J), rel=0.05)


# ---------------------------------------------------------------------------
# adjoint: central finite differences and a forward-mode dense Jacobian
# ---------------------------------------------------------------------------

def _loss(p, J, h, x0, alpha, beta, iters):
    x = O.doch(p, x0, alpha, beta, iters)
    hh = 0 if h is None else h[:, None]
    return np.mean(-0.5 * (x * (J @ x)).sum(axis=0) - (hh * x).sum(axis=0))


def test_adjoint_finite_differences():
    g = I.erdos_renyi_pm1(30, 0.2, seed=26)
    J = g.to_dense()
    h = 0.3 * I.gaussian(I.stream_seed(26, 1), I.stream_seed(26, 2), 0, 30)
    p = O.Problem(g, h)
    a0, beta = O.alpha_beta(g, eta=1.0, method="eig")
    beta = beta / 30.0   # smaller beta keeps the late iterations moving
    N = 12
    alpha = a0 * (1.0 + 0.05 * np.sin(np.arange(N)))
    x0 = I.x0_uniform(30, 3, seed=27, dtype=np.float64)
    ga, gx, loss, zeros = O.backward(p, x0, alpha, beta, N)
    assert zeros == 0
    assert loss == pytest.approx(_loss(p, J, h, x0, alpha, beta, N), rel=1e-14)
    for k in (0, 3, N - 1):
        eps = 1e-6 * max(1.0, abs(alpha[k]))
        ap, am = alpha.copy(), alpha.copy()
        ap[k] += eps
        am[k] -= eps
        fd = (_loss(p, J, h, x0, ap, beta, N) - _loss(p, J, h, x0, am, beta, N)) / (2 * eps)
        assert ga[k] == pytest.approx(fd, rel=1e-5, abs=1e-9 * abs(loss))
    for d in range(4):
        v = I.gaussian(I.stream_seed(28, d), I.stream_seed(29, d), 0, 90).reshape(30, 3)
        v /= np.linalg.norm(v)
        eps = 1e-6
        fd = (_loss(p, J, h, x0 + eps * v, alpha, beta, N)
              - _loss(p, J, h, x0 - eps * v, alpha, beta, N)) / (2 * eps)
        assert (gx * v).sum() == pytest.approx(fd, rel=1e-5)


def test_adjoint_matches_forward_mode_jacobian():
    n, N, R = 7, 5, 2
    J = _sk(n, seed=30)
    p = O.Problem(J)
    alpha0, beta = O.alpha_beta(J, eta=1.0, method="eig")
    beta /= 10
    alpha = alpha0 * np.array([1.0, 1.1, 0.9, 1.05, 1.0])
    x0 = I.x0_uniform(n, R, seed=31, dtype=np.float64)
    ga, gx, _, _ = O.backward(p, x0, alpha, beta, N)
    A = J
    ga_ref = np.zeros(N)
    for r in range(R):
        xs = [x0[:, r]]
        for k in range(N):
            xs.append(np.cbrt((A @ xs[-1] + alpha[k] * xs[-1]) / beta))
        gN = -(A @ xs[N]) / R
        # forward mode: M_k = d x^(k+1) / d x^k, m_k = d x^(k+1) / d alpha_k
        M = [np.diag(1 / (3 * xs[k + 1] ** 2)) @ (A + alpha[k] * np.eye(n)) / beta for k in range(N)]
        m = [xs[k] / (3 * xs[k + 1] ** 2) / beta for k in range(N)]
        P = np.eye(n)
        for k in range(N):
            P = M[k] @ P
        np.testing.assert_allclose(gx[:, r], P.T @ gN, rtol=1e-10, atol=1e-14)
        for k in range(N):
            Q = np.eye(n)
            for j in range(k + 1, N):
                Q = M[j] @ Q
            ga_ref[k] += gN @ (Q @ m[k])
    np.testing.assert_allclose(ga, ga_ref, rtol=1e-10)


# ---------------------------------------------------------------------------
# ADOCH (Algorithm 2)
# ---------------------------------------------------------------------------

def test_adoch_nonmonotone_bound_and_one_step():
    J = _sk(30, seed=32)
    p = O.Problem(J)
    alpha, beta = O.alpha_beta(J, eta=1.1, method="eig")
    beta /= 30 ** 1.5
    x0 = I.x0_uniform(30, 3, seed=33, dtype=np.float64)
    # one step: y^0 = x^0 is always accepted, so ADOCH equals DOCH
    x1, acc = O.adoch(p, x0, alpha, beta, 1, q=5)
    np.testing.assert_array_equal(x1, O.doch(p, x0, alpha, beta, 1))
    assert acc[0].tolist() == [1, 1, 1]
    # H(x^(k+1)) <= max window of H (acceptance test of Eq. BBscheme + Prop. S5)
    q = 3
    for N in (2, 5, 9, 15):
        xN, _ = O.adoch(p, x0, alpha, beta, N, q=q)
        hist = [O.hamiltonian(p, O.adoch(p, x0, alpha, beta, k, q=q)[0], alpha, beta)
                for k in range(max(0, N - 1 - q), N)]
        HN = O.hamiltonian(p, xN, alpha, beta)
        assert np.all(HN <= np.max(hist, axis=0) + 1e-12 * np.abs(HN).max())


def test_adoch_two_spin():
    g = _golden("two_spin_fig3.txt")
    J = np.array([[0.0, -1.0], [-1.0, 0.0]])
    x0 = np.array([[0.7, -0.2], [0.1, 0.5]])
    x, _ = O.adoch(O.Problem(J), x0, g["alpha"][0], g["beta"][0], 60, q=5)
    np.testing.assert_allclose(x, [[1.0, -1.0], [-1.0, 1.0]], atol=1e-9)


def test_adoch_decision_replay():
    """Replaying ADOCH's own decisions reproduces it bit for bit; rejecting every
    extrapolation (v^k = x^k throughout) reduces Algorithm 2 to Algorithm 1 (x^(k+1)
    = T(x^k)); the signed margins are infinite at k = 0 (y^0 = x^0) and their sign
    is the test's decision."""
    J = _sk(40, seed=34)
    p = O.Problem(J)
    alpha, beta = O.alpha_beta(J, eta=1.0, method="eig")
    x0 = I.x0_uniform(40, 3, seed=35, dtype=np.float64)
    iters, q = 25, 1
    x, acc, m = O.adoch(p, x0, alpha, beta, iters, q, margins=True)
    xr, accr = O.adoch(p, x0, alpha, beta, iters, q, decisions=acc)
    np.testing.assert_array_equal(xr, x)
    np.testing.assert_array_equal(accr, acc)
    assert 0 < acc[1:].mean() < 1          # both branches occur
    x0s, acc0 = O.adoch(p, x0, alpha, beta, iters, q, decisions=np.zeros((iters, 3), np.int8))
    np.testing.assert_allclose(x0s, O.doch(p, x0, alpha, beta, iters), rtol=0, atol=1e-15)
    assert not acc0.any()
    assert np.isinf(m[0]).all() and np.isfinite(m[1:]).all()
    np.testing.assert_array_equal(acc[1:], (m[1:] >= 0).astype(np.int8))


# ---------------------------------------------------------------------------
# Stopping rule (Remark S2)
# ---------------------------------------------------------------------------

def test_stopping_rule_definition():
    """doch_until stops each replica at the first step whose relative change
    ||x^(k+1) - x^(k)|| / ||x^(k)|| (recomputed here from single DOCH steps) is
    below eps, and returns that step's iterate; eps = 0 never stops (plain
    Algorithm 1) and a huge eps stops after one step."""
    J = _sk(50, seed=36)
    p = O.Problem(J)
    alpha, beta = O.alpha_beta(J, eta=1.0, method="eig")
    x0 = I.x0_uniform(50, 4, seed=37, dtype=np.float64)
    x, steps, rtr = O.doch_until(p, x0, alpha, beta, 200, 1e-6)
    for r in range(4):
        xk = x0[:, r:r + 1]
        for k in range(steps[r]):
            xn = O.doch(p, xk, alpha, beta, 1)
            rk = np.linalg.norm(xn - xk) / np.linalg.norm(xk)
            assert rk == rtr[k, r]
            assert (rk < 1e-6) == (k == steps[r] - 1)
            xk = xn
        np.testing.assert_array_equal(x[:, r:r + 1], xk)
    assert 1 < steps.min() and steps.max() < 200      # stops somewhere in between
    x0s, s0, _ = O.doch_until(p, x0, alpha, beta, 30, 0.0)
    np.testing.assert_array_equal(x0s, O.doch(p, x0, alpha, beta, 30))
    assert (s0 == 30).all()
    x1, s1, _ = O.doch_until(p, x0, alpha, beta, 30, 1e9)
    np.testing.assert_array_equal(x1, O.doch(p, x0, alpha, beta, 1))
    assert (s1 == 1).all()


def test_adjoint_along_a_given_trajectory():
    """adjoint_along runs the recursion on the iterates it is given: on the
    oracle's own FP64 trajectory it reproduces backward bit for bit, and on
    an FP32-rounded trajectory (not a fixed orbit of T) it matches the
    forward-mode products M_k = diag(1/(3 (x^(k+1))^2)) (J + alpha_k I)/beta,
    m_k = x^k / (3 (x^(k+1))^2 beta) formed along that same trajectory."""
    n, N, R = 9, 6, 3
    J = _sk(n, seed=33)
    h = 0.2 * I.gaussian(I.stream_seed(33, 1), I.stream_seed(33, 2), 0, n)
    p = O.Problem(J, h)
    alpha0, beta = O.alpha_beta(J, eta=1.0, method="eig")
    beta /= 10
    alpha = alpha0 * (1.0 + 0.07 * np.cos(np.arange(N)))
    x0 = I.x0_uniform(n, R, seed=34, dtype=np.float64)
    traj = [x0]
    for k in range(N):
        traj.append(O.doch(p, traj[-1], alpha[k], beta, 1))
    ga, gx, loss, z = O.backward(p, x0, alpha, beta, N)
    ga2, gx2, loss2, z2 = O.adjoint_along(p, np.array(traj), alpha, beta)
    assert np.array_equal(ga, ga2) and np.array_equal(gx, gx2) and loss == loss2 and z == z2 == 0
    t32 = [t.astype(np.float32).astype(np.float64) for t in traj]
    ga3, gx3, loss3, _ = O.adjoint_along(p, np.array(t32), alpha, beta, R=5)
    ga_ref = np.zeros(N)
    loss_ref = 0.0
    for r in range(R):
        xs = [t[:, r] for t in t32]
        loss_ref += (-0.5 * xs[N] @ (J @ xs[N]) - h @ xs[N]) / 5
        gN = -(J @ xs[N] + h) / 5
        M = [np.diag(1 / (3 * xs[k + 1] ** 2)) @ (J + alpha[k] * np.eye(n)) / beta for k in range(N)]
        m = [xs[k] / (3 * xs[k + 1] ** 2) / beta for k in range(N)]
        P = np.eye(n)
        for k in range(N):
            P = M[k] @ P
        np.testing.assert_allclose(gx3[:, r], P.T @ gN, rtol=1e-10, atol=1e-14)
        for k in range(N):
            Q = np.eye(n)
            for j in range(k + 1, N):
                Q = M[j] @ Q
            ga_ref[k] += gN @ (Q @ m[k])
    np.testing.assert_allclose(ga3, ga_ref, rtol=1e-10)
    assert loss3 == pytest.approx(loss_ref, rel=1e-13)


# ---------------------------------------------------------------------------
# eta tuning by probe iterations (Supplementary Note 6)
# ---------------------------------------------------------------------------

def test_tune_eta_beta_rule_and_selection():
    """The candidates' beta (affine in alpha) equals Eq. alphabeta evaluated directly at each
    eta; the chosen eta's score is the minimum over the candidates; a candidate list of one
    eta reduces to a plain DOCH run and its energies; and on a 12-spin instance whose
    brute-force ground energy some candidate reaches, the chosen score is that ground energy."""
    g = I.erdos_renyi_pm1(12, 0.5, seed=35)
    P = O.Problem(g)
    a1, b1 = O.alpha_beta(g, eta=1.0, method="eig")
    for eta in (0.3, 1.0, 1.7):
        a, b = O.alpha_beta(g, eta=eta, method="eig")
        assert a == pytest.approx(eta * a1, rel=1e-14)
        assert b == pytest.approx(b1 + 12 ** 1.5 * (eta - 1.0) * a1, rel=1e-14)
    x0 = I.x0_uniform(12, 16, seed=36, dtype=np.float64)
    etas = [0.1, 0.4, 0.7, 1.0, 1.3, 1.6, 2.0]
    best, mean, k = O.tune_eta(P, x0, etas, 40, a1, b1)
    assert best[k] == best.min()
    assert all(mean[k] <= mean[j] for j in range(len(etas)) if best[j] == best[k])
    b_one, m_one, k_one = O.tune_eta(P, x0, [0.7], 40, a1, b1)
    a, b = O.alpha_beta(g, eta=0.7, method="eig")
    E = O.energy_int(P, O.sign(O.doch(P, x0, a, b, 40)))[0]
    assert k_one == 0 and b_one[0] == E.min() and m_one[0] == pytest.approx(E.mean(), rel=1e-15)
    S = _all_spins(12).astype(np.int64)
    Jd = g.to_dense().astype(np.int64)
    ground = int((-(S @ Jd * S).sum(axis=1) // 2).min())   # brute force over all 2^12 states
    assert best.min() >= ground
    assert best[k] == ground, (best, ground)
