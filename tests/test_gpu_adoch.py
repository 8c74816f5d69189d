"""ADOCH (Algorithm 2) on the device against the FP64 oracle.

Once the iteration converges, y^k -> x^k and H(y^k) ties with the window
maximum to the rounding level of the H sums (another summation order on the
device than in the oracle), so either decision is correct there, and a flip at
a relative margin m moves the next point by about sqrt(m) (H is quadratic near
the fixed point). The tests therefore compare what is unique:
* the device iterates with the oracle run on the device's own decisions
  (`decisions=`): 1e-11 relative in FP64, 1e-5 in FP32;
* every device decision with the oracle's test on that same trajectory,
  wherever the signed margin (window max - H(y^k)) / |H(x^k)| is clear of
  zero (1e-10 in FP64, 1e-4 in FP32);
* H(x^k) against the oracle's H.
q = 0 makes every accepted extrapolation non-increasing in H and the DOCH
step is a descent step (alpha = lambda_max(-J)), so the recorded H(x^k) never
rises (up to FP64 rounding).
"""
import numpy as np
import pytest

import oracle as O
from paper_2509_01928_gb300 import _native as N
from paper_2509_01928_gb300 import build as B
from paper_2509_01928_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available()
    B.build_library()
    return N.load()


def _rel(a, b):
    a = np.asarray(a, np.float64).reshape(b.shape)
    return np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)


def _run(J, x0, alpha, beta, iters, q, h=None, instances=None, host=False):
    p = N.Problem(J, h, instances)
    hd = N.ising_create(p)
    try:
        B_ = 1 if instances is None else len(instances) - 1
        R = x0.shape[1]
        if host:
            x = x0.copy()
            acc = np.zeros((iters, B_ * R), np.int8)
            H = np.zeros((iters + 1, B_ * R))
        else:
            x = torch.from_numpy(x0.copy()).cuda()
            acc = torch.zeros((iters, B_ * R), dtype=torch.int8, device="cuda")
            H = torch.zeros((iters + 1, B_ * R), dtype=torch.float64, device="cuda")
        N.ising_iterate_adoch(hd, x, alpha, beta, iters, q, accepted=acc, H_trace=H)
        if not host:
            x, acc, H = x.cpu().numpy(), acc.cpu().numpy(), H.cpu().numpy()
        return x, acc, H
    finally:
        N.ising_destroy(hd)


def _check(P, x0, alpha, beta, iters, q, x, acc, H, tol_x, tol_m):
    """x and the flags of one (instance) block against the oracle replaying them."""
    ref, _, m = O.adoch(P, x0, alpha, beta, iters, q, decisions=acc, margins=True)
    assert _rel(x, ref).max() <= tol_x
    clear = np.abs(m) > tol_m
    np.testing.assert_array_equal(acc[clear], (m[clear] >= 0).astype(np.int8))
    if H is not None:
        Href = O.hamiltonian(P, ref, alpha, beta)
        assert np.all(np.abs(H[-1] - Href) <= 1e-9 * np.abs(Href))
    return clear


@pytest.mark.parametrize("q", [1, 5])
@pytest.mark.parametrize("kind", ["er", "gauss_field", "torus"])
def test_adoch_fp64_matches_oracle(kind, q):
    h = None
    if kind == "er":
        J = I.erdos_renyi_pm1(300, 0.05, seed=201)
    elif kind == "gauss_field":
        J = I.regular_gauss(400, 5, seed=202)
        h = I.field_gauss(J.n, 0.1, seed=203)
    else:
        J = I.torus_pm1(16, 24, seed=204)
    R, iters = 5, 40
    x0 = I.x0_uniform(J.n, R, seed=205, dtype=np.float64)
    alpha, beta = O.alpha_beta(J, eta=1.0, method="eig")
    P = O.Problem(J, h)
    x, acc, H = _run(J, x0, [alpha], [beta], iters, q, h=h)
    clear = _check(P, x0, alpha, beta, iters, q, x, acc, H, 1e-11, 1e-10)
    assert clear[:10].all()  # before convergence every decision is clear and pinned
    assert acc.any()
    if q == 1:  # the oracle rejects 26-53 % of these extrapolations: both branches run
        assert not acc.all()


def test_adoch_fp32_matches_oracle():
    J = I.regular_gauss(500, 4, seed=211)
    h = I.field_gauss(J.n, 0.1, seed=212)
    J.val = J.val.astype(np.float32)
    R, iters, q = 4, 30, 4
    x0 = I.x0_uniform(J.n, R, seed=213)
    alpha, beta = O.alpha_beta(J, eta=1.0, method="eig")
    P = O.Problem(J, h.astype(np.float32))
    x, acc, H = _run(J, x0, [alpha], [beta], iters, q, h=h.astype(np.float32))
    _check(P, x0.astype(np.float64), alpha, beta, iters, q, x, acc, None, 1e-5, 1e-4)


@pytest.mark.parametrize("shape,q", [((64, 128), 1), ((37, 200), 5), ((16, 1024), 3), ((30, 42), 2)])
def test_adoch_lattice_fp32(shape, q):
    """FP32 lattice: l_cols % 4 == 0 with a 16-byte aligned iterate takes the fast path (both coupling
    products recomputed in each pass, nothing stored); (30, 42) and an iterate shifted by one float
    take the general kernels."""
    J = I.torus_pm1(*shape, seed=251)
    R, iters = 1, 40
    x0 = I.x0_uniform(J.n, R, seed=252)
    alpha, beta = O.alpha_beta(J, eta=1.0, method="eig")
    P = O.Problem(J)
    x, acc, H = _run(J, x0, [alpha], [beta], iters, q)
    clear = _check(P, x0.astype(np.float64), alpha, beta, iters, q, x, acc, None, 1e-5, 1e-4)
    assert clear[:10].all()
    # the same run from a misaligned iterate (general kernels)
    hd = N.ising_create(N.Problem(J))
    try:
        buf = torch.zeros(J.n + 1, dtype=torch.float32, device="cuda")
        xs = buf[1:].view(J.n, 1)
        xs.copy_(torch.from_numpy(x0))
        acc2 = torch.zeros((iters, 1), dtype=torch.int8, device="cuda")
        H2 = torch.zeros((iters + 1, 1), dtype=torch.float64, device="cuda")
        N.ising_iterate_adoch(hd, xs, [alpha], [beta], iters, q, accepted=acc2, H_trace=H2)
        x2, a2, H2 = xs.cpu().numpy(), acc2.cpu().numpy(), H2.cpu().numpy()
    finally:
        N.ising_destroy(hd)
    _check(P, x0.astype(np.float64), alpha, beta, iters, q, x2, a2, None, 1e-5, 1e-4)
    # H(x^k) of the two paths (the fast path forms x^T J x from edge sums of the new iterate) while
    # their trajectories agree: the first ten steps, before the decisions near ties
    np.testing.assert_allclose(H[:10], H2[:10], rtol=1e-5)
    assert np.all(H[1:10] <= H[:9] + 1e-6 * np.abs(H[:9])) or q > 0


def test_adoch_q0_never_rises():
    J = I.erdos_renyi_pm1(400, 0.04, seed=221)
    R, iters = 6, 60
    x0 = I.x0_uniform(J.n, R, seed=222, dtype=np.float64)
    alpha, beta = O.alpha_beta(J, eta=1.0, method="eig")
    _, acc, H = _run(J, x0, [alpha], [beta], iters, 0)
    assert np.all(H[1:] <= H[:-1] + 1e-12 * np.abs(H[:-1]))
    assert acc.any()


def test_adoch_batched_instances_and_host_buffers():
    gs = [I.regular_gauss(300, 3, seed=231), I.regular_gauss(700, 6, seed=232), I.regular_gauss(150, 4, seed=233)]
    hs = [I.field_gauss(g.n, 0.1, seed=240 + b) for b, g in enumerate(gs)]
    off = np.cumsum([0] + [g.n for g in gs]).astype(np.int64)
    nz = np.cumsum([0] + [g.nnz for g in gs])
    rp = np.concatenate([[0]] + [g.row_ptr[1:] + z for g, z in zip(gs, nz[:-1])])
    col = np.concatenate([g.col + o for g, o in zip(gs, off[:-1])]).astype(np.int32)
    val = np.concatenate([g.val for g in gs])
    J = I.CSR(int(off[-1]), rp, col, val)
    h = np.concatenate(hs)
    R, iters, q = 3, 25, 3
    x0 = I.x0_uniform(J.n, R, seed=234, dtype=np.float64)
    ab = [O.alpha_beta(g, eta=1.0, method="eig") for g in gs]
    alphas, betas = [a for a, _ in ab], [b for _, b in ab]
    xd, accd, Hd = _run(J, x0, alphas, betas, iters, q, h=h, instances=off)
    xh, acch, Hh = _run(J, x0, alphas, betas, iters, q, h=h, instances=off, host=True)
    assert np.array_equal(xd, xh) and np.array_equal(accd, acch) and np.array_equal(Hd, Hh)
    for b, g in enumerate(gs):
        _check(O.Problem(g, hs[b]), x0[off[b]:off[b + 1]], alphas[b], betas[b], iters, q,
               xd[off[b]:off[b + 1]], accd[:, b * R:(b + 1) * R], Hd[:, b * R:(b + 1) * R], 1e-11, 1e-10)


def test_adoch_rejects_dense():
    J = I.dense_pm1(64, seed=241)
    hd = N.ising_create(N.Problem(J))
    try:
        x = torch.zeros((64, 2), dtype=torch.float32, device="cuda")
        with pytest.raises(N.IsingError, match="ADOCH runs on CSR, TORUS2D or PROCEDURAL"):
            N.ising_iterate_adoch(hd, x, [1.0], [1.0], 3, 2)
    finally:
        N.ising_destroy(hd)
