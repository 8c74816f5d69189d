"""eta chosen by probe iterations on the device (ising_tune_eta) against the
oracle's tune_eta (Supplementary Note 6: alpha = eta lambda_max(-J), eta tuned
by the Ising energy after a few iterations).

FP64 iterates agree with the oracle's to ~1e-12, so the spins after the
probes, their integer energies, the scores and the chosen candidate are the
oracle's exactly. FP32 iterates: the device's scores are the exact energies of
its own probe iterates (ising_iterate + ising_energy on the chosen candidate
give the same numbers), and the chosen alpha and beta follow Eq. alphabeta.
"""
import numpy as np
import pytest

import oracle as O
from paper_2509_01928_gb300 import _native as N
from paper_2509_01928_gb300 import build as B
from paper_2509_01928_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ETAS = [0.2, 0.5, 0.8, 1.0, 1.2, 1.5, 2.0]


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available()
    B.build_library()
    return N.load()


@pytest.mark.parametrize("kind, probe", [("er800", 5), ("er800", 1), ("torus", 3), ("regular", 8)])
def test_tune_eta_fp64_matches_oracle(kind, probe):
    if kind == "er800":
        J = I.erdos_renyi_pm1(800, 0.06, seed=1)
        method = "eig"
    elif kind == "torus":
        J = I.torus_pm1(48, 96, seed=11)
        method = "wigner"
    else:
        J = I.regular_gauss(2000, 4, seed=12)
        method = "eig"
    R = 8
    x0 = I.x0_uniform(J.n, R, seed=13, dtype=np.float64)
    a1, b1 = O.alpha_beta(J, eta=1.0, method=method)
    best_r, mean_r, k_r = O.tune_eta(O.Problem(J), x0, ETAS, probe, a1, b1)
    h = N.ising_create(N.Problem(J))
    try:
        a, b, k, best, mean = N.ising_tune_eta(h, torch.from_numpy(x0).cuda(), ETAS, probe, a1, b1)
    finally:
        N.ising_destroy(h)
    if O.Problem(J).integer:
        assert np.array_equal(best, best_r)
    else:
        np.testing.assert_allclose(best, best_r, rtol=1e-12)
    np.testing.assert_allclose(mean, mean_r, rtol=1e-12)
    assert k == k_r
    a_r, b_r = O.alpha_beta(J, eta=ETAS[k_r], method=method)
    assert a == pytest.approx(a_r, rel=1e-12) and b == pytest.approx(b_r, rel=1e-12)


def test_tune_eta_fp32_scores_are_the_probe_energies():
    t = I.torus_pm1(64, 256, seed=14)
    R = 4
    x0 = I.x0_uniform(t.n, R, seed=15)
    a1, b1 = O.alpha_beta(t, eta=1.0, method="wigner")
    h = N.ising_create(N.Problem(t))
    try:
        xd = torch.from_numpy(x0.copy()).cuda()
        a, b, k, best, mean = N.ising_tune_eta(h, xd, ETAS, 3, a1, b1)
        assert np.array_equal(xd.cpu().numpy(), x0)                   # the start is not modified
        for j, eta in enumerate(ETAS):
            x = torch.from_numpy(x0.copy()).cuda()
            N.ising_iterate(h, x, [eta * a1], [b1 + t.n ** 1.5 * (eta - 1.0) * a1], 3)
            E = np.zeros(R, np.int64)
            N.ising_energy(h, x, E_int=E)
            assert best[j] == E.min() and mean[j] == pytest.approx(E.mean(), rel=1e-15)
            s = O.sign(x.cpu().numpy().astype(np.float64))
            assert np.array_equal(E, O.energy_int(O.Problem(t), s)[0])  # exact energies of those spins
        assert best[k] == best.min()
        assert a == pytest.approx(ETAS[k] * a1, rel=1e-15)
        # a host array as the start gives the same table
        ah, bh, kh, besth, meanh = N.ising_tune_eta(h, x0.copy(), ETAS, 3, a1, b1)
        assert (ah, bh, kh) == (a, b, k) and np.array_equal(besth, best) and np.array_equal(meanh, mean)
    finally:
        N.ising_destroy(h)


def test_tune_eta_argument_errors():
    t = I.torus_pm1(8, 8, seed=16)
    h = N.ising_create(N.Problem(t))
    try:
        x0 = torch.zeros((t.n, 1), dtype=torch.float32, device="cuda")
        for args in (([], 3, 1.0, 1.0), ([1.0], -1, 1.0, 1.0), ([1.0], 3, 1.0, 0.0), ([float("nan")], 3, 1.0, 1.0)):
            with pytest.raises((N.IsingError, ValueError)):
                N.ising_tune_eta(h, x0, *args)
    finally:
        N.ising_destroy(h)
