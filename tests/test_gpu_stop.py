"""The stopping rule of Remark S2 on the device against the FP64 oracle.

A pair's step count is an integer decided by floating point: r^(k) < eps.
The device reduces r^(k) in another order than the oracle (FP64; compensated
FP32 per thread from FP32 iterates on the FP32 path), so the counts are compared where the
oracle's r^(k) stays clear of eps up to its stopping step (relative margin
1e-9 in FP64, 1e-3 in FP32); where the counts agree the iterates are compared
at the parity tolerance of the path (FP64 1e-10, FP32 1e-5).
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


def _run(J, x0, alpha, beta, max_iters, eps, h=None, instances=None, host=False):
    hd = N.ising_create(N.Problem(J, h, instances))
    try:
        pairs = x0.shape[1] * (1 if instances is None else len(instances) - 1)
        if host:
            x, steps = x0.copy(), np.zeros(pairs, np.int32)
        else:
            x = torch.from_numpy(x0.copy()).cuda()
            steps = torch.zeros(pairs, dtype=torch.int32, device="cuda")
        N.ising_iterate_until(hd, x, alpha, beta, max_iters, eps, steps=steps)
        if not host:
            x, steps = x.cpu().numpy(), steps.cpu().numpy()
        return x, steps
    finally:
        N.ising_destroy(hd)


def _compare(P, x0, alpha, beta, max_iters, eps, x, steps, margin, tol):
    ref, ksteps, rtr = O.doch_until(P, x0.astype(np.float64), alpha, beta, max_iters, eps)
    compared = 0
    for r in range(x0.shape[1]):
        K = ksteps[r]
        clear = np.all(np.abs(rtr[:K, r] / eps - 1.0) > margin) if eps > 0 else True
        if not clear:
            continue
        assert steps[r] == K, f"replica {r}: {steps[r]} steps, oracle {K}"
        assert _rel(x[:, r:r + 1], ref[:, r:r + 1]).max() <= tol
        compared += 1
    return compared, ksteps


@pytest.mark.parametrize("kind", ["er", "torus", "gauss_field"])
def test_stop_fp64_matches_oracle(kind):
    h = None
    if kind == "er":
        J = I.erdos_renyi_pm1(300, 0.05, seed=301)
    elif kind == "torus":
        J = I.torus_pm1(20, 24, seed=302)
    else:
        J = I.regular_gauss(400, 5, seed=303)
        h = I.field_gauss(J.n, 0.1, seed=304)
    R = 6
    x0 = I.x0_uniform(J.n, R, seed=305, dtype=np.float64)
    alpha, beta = O.alpha_beta(J, eta=1.0, method="eig")
    x, steps = _run(J, x0, [alpha], [beta], 400, 1e-6, h=h)
    compared, ksteps = _compare(O.Problem(J, h), x0, alpha, beta, 400, 1e-6, x, steps, 1e-9, 1e-10)
    assert compared >= R - 1
    assert 1 < ksteps.min() and ksteps.max() < 400  # the rule fires before max_iters


def test_stop_fp32_matches_oracle():
    J = I.regular_gauss(500, 4, seed=311)
    h = I.field_gauss(J.n, 0.1, seed=312).astype(np.float32)
    J.val = J.val.astype(np.float32)
    R = 5
    x0 = I.x0_uniform(J.n, R, seed=313)
    alpha, beta = O.alpha_beta(J, eta=1.0, method="eig")
    x, steps = _run(J, x0, [alpha], [beta], 300, 1e-4, h=h)
    compared, _ = _compare(O.Problem(J, h), x0, alpha, beta, 300, 1e-4, x, steps, 1e-3, 1e-5)
    assert compared >= R - 1


def test_stop_batched_host_buffers_and_extremes():
    gs = [I.regular_gauss(300, 3, seed=321), I.regular_gauss(700, 6, seed=322), I.regular_gauss(150, 4, seed=323)]
    hs = [I.field_gauss(g.n, 0.1, seed=330 + b) for b, g in enumerate(gs)]
    off = np.cumsum([0] + [g.n for g in gs]).astype(np.int64)
    nz = np.cumsum([0] + [g.nnz for g in gs])
    rp = np.concatenate([[0]] + [g.row_ptr[1:] + z for g, z in zip(gs, nz[:-1])])
    col = np.concatenate([g.col + o for g, o in zip(gs, off[:-1])]).astype(np.int32)
    J = I.CSR(int(off[-1]), rp, col, np.concatenate([g.val for g in gs]))
    h = np.concatenate(hs)
    R = 3
    x0 = I.x0_uniform(J.n, R, seed=324, dtype=np.float64)
    ab = [O.alpha_beta(g, eta=1.0, method="eig") for g in gs]
    alphas, betas = [a for a, _ in ab], [b for _, b in ab]
    xd, sd = _run(J, x0, alphas, betas, 300, 1e-7, h=h, instances=off)
    xh, sh = _run(J, x0, alphas, betas, 300, 1e-7, h=h, instances=off, host=True)
    assert np.array_equal(xd, xh) and np.array_equal(sd, sh)
    for b, g in enumerate(gs):
        compared, _ = _compare(O.Problem(g, hs[b]), x0[off[b]:off[b + 1]], alphas[b], betas[b], 300, 1e-7,
                               xd[off[b]:off[b + 1]], sd[b * R:(b + 1) * R], 1e-9, 1e-10)
        assert compared >= R - 1
    # eps = 0: every pair runs max_iters steps of Algorithm 1
    x0e, s0 = _run(J, x0, alphas, betas, 25, 0.0, h=h, instances=off)
    assert (s0 == 25).all()
    for b, g in enumerate(gs):
        ref = O.doch(O.Problem(g, hs[b]), x0[off[b]:off[b + 1]], alphas[b], betas[b], 25)
        assert _rel(x0e[off[b]:off[b + 1]], ref).max() <= 1e-10
    # a huge eps: every pair stops after one step
    x1, s1 = _run(J, x0, alphas, betas, 25, 1e9, h=h, instances=off)
    assert (s1 == 1).all()
    for b, g in enumerate(gs):
        ref = O.doch(O.Problem(g, hs[b]), x0[off[b]:off[b + 1]], alphas[b], betas[b], 1)
        assert _rel(x1[off[b]:off[b + 1]], ref).max() <= 1e-12


def test_stop_batched_fp32_in_resident_kernel():
    """Batched FP32 instances apply the rule inside the shared-memory resident kernel
    (replica groups of 16, 8 and 2 here); eps = 0 and one-step runs reproduce
    ising_iterate bit for bit (the same kernel with the rule off)."""
    sizes, degrees = [500, 3000, 9000], [4, 7, 5]
    gs = [I.regular_gauss(n, d, seed=340 + b) for b, (n, d) in enumerate(zip(sizes, degrees))]
    hs = [I.field_gauss(g.n, 0.1, seed=350 + b).astype(np.float32) for b, g in enumerate(gs)]
    off = np.cumsum([0] + [g.n for g in gs]).astype(np.int64)
    nz = np.cumsum([0] + [g.nnz for g in gs])
    rp = np.concatenate([[0]] + [g.row_ptr[1:] + z for g, z in zip(gs, nz[:-1])])
    col = np.concatenate([g.col + o for g, o in zip(gs, off[:-1])]).astype(np.int32)
    J = I.CSR(int(off[-1]), rp, col, np.concatenate([g.val for g in gs]).astype(np.float32))
    h = np.concatenate(hs)
    R = 16
    x0 = I.x0_uniform(J.n, R, seed=360)
    ab = [O.alpha_beta(g, eta=1.0, method="wigner") for g in gs]
    alphas, betas = [a for a, _ in ab], [b for _, b in ab]
    x, steps = _run(J, x0, alphas, betas, 300, 1e-4, h=h, instances=off)
    for b, g in enumerate(gs):
        compared, _ = _compare(O.Problem(g, hs[b]), x0[off[b]:off[b + 1]], alphas[b], betas[b], 300, 1e-4,
                               x[off[b]:off[b + 1]], steps[b * R:(b + 1) * R], 1e-3, 1e-5)
        assert compared >= R - 2
    hd = N.ising_create(N.Problem(J, h, off))
    try:
        for iters, eps in ((20, 0.0), (1, 1e9)):
            xa = torch.from_numpy(x0.copy()).cuda()
            N.ising_iterate(hd, xa, alphas, betas, iters, n_instances=len(gs))
            xb = torch.from_numpy(x0.copy()).cuda()
            sb = torch.zeros(len(gs) * R, dtype=torch.int32, device="cuda")
            N.ising_iterate_until(hd, xb, alphas, betas, 20, eps, steps=sb)
            assert torch.equal(xa, xb)
            assert (sb.cpu().numpy() == iters).all()
    finally:
        N.ising_destroy(hd)
