"""Failure detection in the forms that fault, trap or hang no GPU.

* Bounded device waits: ising_selftest_wait runs the tensor-core kernel's
  bounded mbarrier wait in a one-thread kernel. With nothing arriving, the wait
  gives up after its limit (1 ms here), sets the handle's error word and
  returns; the call reports ISING_ERR_TIMEOUT, clears the word, and the same
  handle then iterates and reads out correctly. With an arrival the same call
  returns OK at once.
* Monotone monitor: with alpha = 0 (eta = 0, below lambda_max(-J)) the DC
  split of Eq. Hamilton loses its convex g and H(x^k) rises on an
  Erdos-Renyi graph; with ISING_FLAG_STRICT_MONOTONE and an H trace the call
  returns ISING_ERR_NOT_MONOTONE, the trace it still delivers matches the
  oracle's, and the handle stays usable.
"""
import time

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


def test_bounded_wait_times_out_and_the_handle_stays_usable():
    t = I.torus_pm1(16, 64, seed=90)
    x0 = I.x0_uniform(t.n, 1, seed=91)
    alpha, beta = O.alpha_beta(t, eta=1.0, method="eig")
    h = N.ising_create(N.Problem(t))
    try:
        N.ising_selftest_wait(h, True, 1_000_000)          # satisfied wait: OK
        w0 = time.perf_counter()
        with pytest.raises(N.IsingError) as e:
            N.ising_selftest_wait(h, False, 1_000_000)     # nothing arrives: 1 ms, then TIMEOUT
        assert e.value.name == "ISING_ERR_TIMEOUT"
        assert time.perf_counter() - w0 >= 1e-3
        N.ising_synchronize(h)                             # the error word was cleared
        N.ising_selftest_wait(h, True, 1_000_000)
        x = torch.from_numpy(x0.copy()).cuda()
        N.ising_iterate(h, x, [alpha], [beta], 9)
        E = np.zeros(1, np.int64)
        N.ising_energy(h, x, E_int=E)
        ref = O.doch(O.Problem(t), x0, alpha, beta, 9)
        got = x.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
        assert E[0] == O.energy_int(O.Problem(t), O.sign(got))[0][0]
    finally:
        N.ising_destroy(h)


def test_bounded_wait_rejects_limits_out_of_range():
    t = I.torus_pm1(4, 8, seed=92)
    h = N.ising_create(N.Problem(t))
    try:
        for lim in (0, 999, 2_000_000_000):
            with pytest.raises(N.IsingError) as e:
                N.ising_selftest_wait(h, False, lim)
            assert e.value.name == "ISING_ERR_INVALID_ARG"
    finally:
        N.ising_destroy(h)


def test_strict_monotone_reports_a_rising_hamiltonian():
    g = I.erdos_renyi_pm1(200, 0.1, seed=50)
    _, beta = O.alpha_beta(g, eta=1.0, method="eig")
    beta /= 4 * 200 ** 1.5
    alpha = 0.0                                            # eta = 0: g is not convex
    x0 = I.x0_uniform(g.n, 4, seed=52, dtype=np.float64)
    _, Href = O.doch(O.Problem(g), x0, alpha, beta, 15, trace=True)
    assert (np.diff(Href, axis=0) > 1e-6 * np.abs(Href[:-1])).any()   # the oracle's H rises
    h = N.ising_create(N.Problem(g), N.FLAG_STRICT_MONOTONE)
    try:
        x = torch.from_numpy(x0.copy()).cuda()
        H = np.zeros((16, 1, 4))
        with pytest.raises(N.IsingError) as e:
            N.ising_iterate(h, x, [alpha], [beta], 15, H_trace=H)
        assert e.value.name == "ISING_ERR_NOT_MONOTONE"
        np.testing.assert_allclose(H[:, 0, :], Href, rtol=1e-10, atol=1e-12 * np.abs(Href).max())
        # the handle stays usable: a convex split (eta = 1) passes the same check
        a1, b1 = O.alpha_beta(g, eta=1.0, method="eig")
        x = torch.from_numpy(x0.copy()).cuda()
        N.ising_iterate(h, x, [a1], [b1], 15, H_trace=np.zeros((16, 1, 4)))
    finally:
        N.ising_destroy(h)
    h = N.ising_create(N.Problem(g))                       # without the flag the rise is only recorded
    try:
        x = torch.from_numpy(x0.copy()).cuda()
        H = np.zeros((16, 1, 4))
        N.ising_iterate(h, x, [alpha], [beta], 15, H_trace=H)
        np.testing.assert_allclose(H[:, 0, :], Href, rtol=1e-10, atol=1e-12 * np.abs(Href).max())
    finally:
        N.ising_destroy(h)
