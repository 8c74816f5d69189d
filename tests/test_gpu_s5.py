"""Algorithm S5 generated on the device (ising_create_s5) against the
reference generator, bit for bit; the device parameter rule against the host
rule; and DOCH on a device-generated problem against the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2509_01928_gb300 import _native as N
from paper_2509_01928_gb300 import build as B
from oracle import matrices as M
from paper_2509_01928_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available()
    B.build_library()
    return N.load()


@pytest.mark.parametrize("n, p, seed", [(1000, 5.0, 1), (4097, 0.5, 2), (777, 100.0, 3), (50, 50.0, 4),
                                        (20000, 0.05, 5)])
def test_s5_device_equals_reference(n, p, seed):
    h = N.ising_create_s5(n, p, seed)
    try:
        rp, col, val = N.ising_csr_export(h)
    finally:
        N.ising_destroy(h)
    J = M.s5_csr(n, p, seed)
    assert np.array_equal(rp, J.row_ptr)
    assert np.array_equal(col, J.col)
    assert np.array_equal(val.astype(np.int64), J.val.astype(np.int64))


@pytest.mark.parametrize("method", [1, 2])
def test_device_params_match_host_rule(method):
    J = M.s5_csr(1500, 3.0, seed=6)
    ha, hb = N.ising_default_params(N.Problem(J), eta=1.0, method=method)
    h = N.ising_create_s5(1500, 3.0, 6)
    try:
        da, db = N.ising_params_device(h, eta=1.0, method=method)
    finally:
        N.ising_destroy(h)
    tol = 1e-12 if method == 2 else 1e-9
    assert abs(da[0] - ha[0]) <= tol * abs(ha[0])
    assert abs(db[0] - hb[0]) <= tol * abs(hb[0])
    t = I.torus_pm1(48, 64, seed=7)
    ha, hb = N.ising_default_params(N.Problem(t), eta=1.3, method=method)
    h = N.ising_create(N.Problem(t))
    try:
        da, db = N.ising_params_device(h, eta=1.3, method=method)
    finally:
        N.ising_destroy(h)
    assert abs(da[0] - ha[0]) <= tol * abs(ha[0])
    assert abs(db[0] - hb[0]) <= tol * abs(hb[0])


def test_doch_on_device_generated_problem():
    n, p = 600, 4.0
    J = M.s5_csr(n, p, seed=8)
    alpha, beta = O.alpha_beta(J, eta=1.0, method="eig")
    x0 = I.x0_uniform(n, 4, seed=9, dtype=np.float64)
    ref = O.doch(O.Problem(J), x0, alpha, beta, 60)
    h = N.ising_create_s5(n, p, 8)
    try:
        x = torch.from_numpy(x0.copy()).cuda()
        N.ising_iterate(h, x, [alpha], [beta], 60)
        got = x.cpu().numpy()
        E = np.zeros(4, np.int64)
        N.ising_energy(h, x, E_int=E)
    finally:
        N.ising_destroy(h)
    rel = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert rel.max() <= 1e-10
    Er, _ = O.energy_int(O.Problem(J), O.sign(ref))
    assert np.array_equal(E, Er)


@pytest.mark.parametrize("method, omethod, tol", [(1, "eig", 1e-6), (2, "wigner", 1e-12)])
def test_device_params_match_oracle(method, omethod, tol):
    """ising_params_device against the oracle's Eq. alphabeta: the power method
    on the device against a dense symmetric eigensolver (to the power method's
    convergence, 1e-6), the Wigner estimate of Eq. estimate_eig_J to 1e-12."""
    J = M.s5_csr(1500, 3.0, seed=6)
    ao, bo = O.alpha_beta(J, eta=1.0, method=omethod)
    h = N.ising_create_s5(1500, 3.0, 6)
    try:
        da, db = N.ising_params_device(h, eta=1.0, method=method)
    finally:
        N.ising_destroy(h)
    assert da[0] == pytest.approx(ao, rel=tol) and db[0] == pytest.approx(bo, rel=tol)
    t = I.torus_pm1(48, 64, seed=7)
    ao, bo = O.alpha_beta(t, eta=1.3, method=omethod)
    h = N.ising_create(N.Problem(t))
    try:
        da, db = N.ising_params_device(h, eta=1.3, method=method)
    finally:
        N.ising_destroy(h)
    assert da[0] == pytest.approx(ao, rel=tol) and db[0] == pytest.approx(bo, rel=tol)
