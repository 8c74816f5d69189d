"""Degenerate and boundary cases of the DOCH iteration and readout, against the
FP64 oracle (element by element) or against what the method fixes exactly.

* zero iterations leave x unchanged, bit for bit, on every storage form;
* x = 0 is a fixed point of T when h = 0 (cbrt(0) = 0), and its spins are all +1
  (sign(0) = +1), whose energy is -1/2 sum_ij J_ij exactly;
* rows without couplings (isolated spins, an empty CSR row) follow
  x' = cbrt(alpha x / beta) (or cbrt((alpha x + h) / beta) with a field);
* couplings all zero: the spins decouple, and the energy of any spin vector
  is -h^T s;
* the smallest problems: n = 1 and n = 2 (the two-spin example's size), one
  replica; a batch whose instances include one with a single spin;
* ragged sizes: n one above and one below a tile of 128 rows, R = 3.
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


def _run(J, x0, alpha, beta, iters, h=None, instances=None, flags=0):
    hd = N.ising_create(N.Problem(J, h, instances), flags)
    try:
        x = torch.from_numpy(np.ascontiguousarray(x0)).cuda()
        N.ising_iterate(hd, x, np.atleast_1d(alpha), np.atleast_1d(beta), iters,
                        n_instances=1 if instances is None else len(instances) - 1)
        return x.cpu().numpy()
    finally:
        N.ising_destroy(hd)


def _csr_with_empty_rows(n, seed):
    """An Erdos-Renyi graph with every third spin isolated (its row empty)."""
    g = I.erdos_renyi_pm1(n, 0.2, seed=seed)
    d = g.to_dense()
    iso = np.arange(0, n, 3)
    d[iso, :] = 0
    d[:, iso] = 0
    i, j = np.nonzero(np.triu(d, 1))
    return I.csr_from_upper(n, i, j, d[i, j].astype(np.int8)), iso


@pytest.mark.parametrize("form", ["torus", "csr", "dense_bf16", "dense_f32"])
def test_zero_iterations_leave_x_unchanged(form):
    if form == "torus":
        J = I.torus_pm1(8, 16, seed=1)
    elif form == "csr":
        J = I.erdos_renyi_pm1(100, 0.1, seed=2)
    else:
        J = I.dense_pm1(130, seed=3)
    x0 = I.x0_uniform(J.n if hasattr(J, "n") else J.shape[0], 4, seed=4)
    hd = N.ising_create(N.Problem(J))
    try:
        x = torch.from_numpy(x0).cuda()
        if form == "dense_bf16":
            x = x.to(torch.bfloat16)
        ref = x.clone()
        N.ising_iterate(hd, x, [1.0], [1.0], 0)
        assert torch.equal(x, ref)
    finally:
        N.ising_destroy(hd)


@pytest.mark.parametrize("form", ["torus", "csr"])
def test_zero_is_a_fixed_point_and_its_spins_are_plus_one(form):
    J = I.torus_pm1(16, 32, seed=5) if form == "torus" else I.erdos_renyi_pm1(300, 0.05, seed=6)
    alpha, beta = O.alpha_beta(J, eta=1.0, method="eig")
    n = J.n
    x = _run(J, np.zeros((n, 2), np.float32), alpha, beta, 7)
    assert np.all(x == 0.0)
    hd = N.ising_create(N.Problem(J))
    try:
        E = np.zeros(2, np.int64)
        sp = np.zeros((n, 2), np.int8)
        N.ising_energy(hd, torch.zeros((n, 2), dtype=torch.float32, device="cuda"), E_int=E, spins=sp)
    finally:
        N.ising_destroy(hd)
    assert np.all(sp == 1)
    Er, _ = O.energy_int(O.Problem(J), np.ones((n, 2), np.int8))
    assert np.array_equal(E, Er)
    jsum = int(J.to_csr().val.astype(np.int64).sum()) if form == "torus" else int(J.val.astype(np.int64).sum())
    assert E[0] == -(jsum // 2)


@pytest.mark.parametrize("with_field", [False, True])
def test_rows_without_couplings(with_field):
    J, iso = _csr_with_empty_rows(200, seed=7)
    h = I.field_gauss(200, 0.1, seed=8) if with_field else None
    alpha, beta = 3.0, 40.0
    x0 = I.x0_uniform(200, 3, seed=9, dtype=np.float64)
    got = _run(J, x0, alpha, beta, 5, h=h)
    ref = O.doch(O.Problem(J, h), x0, alpha, beta, 5)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-15)
    # the isolated spins follow the one-variable map exactly as written
    x = x0[iso].copy()
    hi = (h[iso] if with_field else np.zeros(len(iso)))[:, None]
    for _ in range(5):
        x = np.cbrt((alpha * x + hi) / beta)
    np.testing.assert_allclose(got[iso], x, rtol=1e-13)


def test_all_zero_couplings_and_field_energy():
    n = 50
    J = I.csr_from_upper(n, np.array([0, 3], np.int64), np.array([1, 7], np.int64), np.zeros(2, np.int8))
    h = np.round(3 * I.field_gauss(n, 1.0, seed=10)).astype(np.int8)
    s = np.where(I.x0_uniform(n, 4, seed=11) >= 0, 1, -1).astype(np.int8)
    hd = N.ising_create(N.Problem(J, h))
    try:
        E = np.zeros(4, np.int64)
        N.ising_energy(hd, torch.from_numpy(s).cuda(), E_int=E)
    finally:
        N.ising_destroy(hd)
    assert np.array_equal(E, -(h.astype(np.int64) @ s.astype(np.int64)))


@pytest.mark.parametrize("n", [1, 2])
def test_smallest_problems(n):
    if n == 1:
        J = I.csr_from_upper(1, np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0, np.int8))
    else:
        J = np.array([[0, -1], [-1, 0]], np.int8)   # the two-spin antiferromagnet of the worked example
    x0 = np.array([[0.3], [-0.8]], np.float32)[:n]
    alpha, beta = 1.0, 2.0
    got = _run(J if n == 1 else I.csr_from_upper(2, np.array([0]), np.array([1]), np.array([-1], np.int8)),
               x0, alpha, beta, 6)
    ref = O.doch(O.Problem(J), x0.astype(np.float64), alpha, beta, 6)
    np.testing.assert_allclose(got, ref, rtol=1e-6)


def test_batch_with_a_single_spin_instance():
    g = I.regular_gauss(300, 3, seed=12)
    single = I.csr_from_upper(1, np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0, np.float64))
    off = np.array([0, 300, 301], np.int64)
    rp = np.concatenate([g.row_ptr, [g.row_ptr[-1]]]).astype(np.int64)
    J = I.CSR(301, rp, g.col.astype(np.int32), g.val.astype(np.float32))
    x0 = I.x0_uniform(301, 4, seed=13)
    a0, b0 = O.alpha_beta(g, eta=1.0, method="eig")
    got = _run(J, x0, [a0, 1.5], [b0, 7.0], 9, instances=off)
    ref0 = O.doch(O.Problem(g), x0[:300], a0, b0, 9)
    np.testing.assert_allclose(got[:300], ref0, rtol=1e-5, atol=1e-6 * np.abs(ref0).max())
    ref1 = O.doch(O.Problem(single), x0[300:], 1.5, 7.0, 9)
    np.testing.assert_allclose(got[300:], ref1, rtol=1e-6)


@pytest.mark.parametrize("n", [127, 129])
def test_ragged_dense_sizes_three_replicas(n):
    J = I.dense_pm1(n, seed=14)
    alpha, beta = O.alpha_beta(J, eta=1.0, method="eig")
    x0 = I.x0_uniform(n, 3, seed=15)
    got = _run(J, x0, alpha, beta, 1)
    ref = O.doch(O.Problem(J), x0, alpha, beta, 1)
    rel = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert rel.max() <= 1e-5
