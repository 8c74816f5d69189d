"""Host-side checks of the C ABI that need no GPU: the library loads, it
exports every entry point include/ising.h declares, its validation rejects
bad problems before touching the device, and its parameter rule (Eq.
alphabeta) agrees with the oracle's."""
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2509_01928_gb300 import _native as N
from paper_2509_01928_gb300 import build as B
from paper_2509_01928_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build_library()
    return N.load()


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(ising_\w+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert {"ising_create", "ising_iterate", "ising_energy", "ising_backward", "ising_destroy"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    assert N.ising_status_string(0) == "ok"
    assert "symmetric" in N.ising_status_string(2)


def _csr(n, rows):
    """Tiny CSR from a dict row -> list of (col, val)."""
    rp, col, val = [0], [], []
    for i in range(n):
        for j, v in rows.get(i, []):
            col.append(j)
            val.append(v)
        rp.append(len(col))
    return I.CSR(n, np.array(rp), np.array(col, np.int32), np.array(val, np.int8))


@pytest.mark.parametrize("rows, status", [
    ({0: [(1, 1)], 1: [(0, -1)]}, "ISING_ERR_NOT_SYMMETRIC"),
    ({0: [(0, 1), (1, 1)], 1: [(0, 1)]}, "ISING_ERR_NONZERO_DIAG"),
    ({0: [(2, 1)], 2: [(0, 1)]}, "ISING_ERR_INDEX_RANGE"),
])
def test_validation_rejects(lib, rows, status):
    n = 2 if status != "ISING_ERR_INDEX_RANGE" else 2
    p = N.Problem(_csr(n, rows))
    with pytest.raises(N.IsingError) as e:
        N.ising_default_params(p)
    assert e.value.name == status


def test_validation_rejects_nonfinite_and_bad_torus(lib):
    J = I.CSR(2, np.array([0, 1, 2]), np.array([1, 0], np.int32), np.array([np.nan, np.nan]))
    with pytest.raises(N.IsingError) as e:
        N.ising_default_params(N.Problem(J))
    assert e.value.name == "ISING_ERR_NONFINITE"
    D = np.array([[0.0, 0.5], [0.5, 0.0]])     # real-valued dense J has no exact tensor-core form
    with pytest.raises(N.IsingError) as e:
        N.ising_default_params(N.Problem(D))
    assert e.value.name == "ISING_ERR_UNSUPPORTED"
    t = I.Torus2D(np.ones((1, 4), np.int8), np.ones((1, 4), np.int8))
    with pytest.raises(N.IsingError) as e:
        N.ising_default_params(N.Problem(t))
    assert e.value.name == "ISING_ERR_INVALID_ARG"


@pytest.mark.parametrize("kind", ["er", "torus", "dense", "regular"])
def test_default_params_match_oracle(lib, kind):
    if kind == "er":
        J = I.erdos_renyi_pm1(300, 0.06, seed=1)
    elif kind == "torus":
        J = I.torus_pm1(12, 16, seed=2)
    elif kind == "dense":
        J = I.dense_pm1(200, seed=3)
    else:
        J = I.regular_gauss(400, 5, seed=4)
    a, b = N.ising_default_params(N.Problem(J), eta=1.0, method=1)   # power iteration
    ao, bo = O.alpha_beta(J, eta=1.0, method="eig")                   # dense eigensolver
    assert a[0] == pytest.approx(ao, rel=1e-6)
    assert b[0] == pytest.approx(bo, rel=1e-6)
    aw, bw = N.ising_default_params(N.Problem(J), eta=0.7, method=2)  # Wigner estimate
    aow, bow = O.alpha_beta(J, eta=0.7, method="wigner")
    assert aw[0] == pytest.approx(aow, rel=1e-12)
    assert bw[0] == pytest.approx(bow, rel=1e-12)


def test_default_params_batched(lib):
    gs = [I.regular_gauss(60 + 10 * b, 3 + b, seed=10 + b) for b in range(3)]
    off = np.cumsum([0] + [g.n for g in gs])
    rp = np.concatenate([[0]] + [g.row_ptr[1:] + g0 for g, g0 in
                                 zip(gs, np.cumsum([0] + [g.nnz for g in gs])[:-1])])
    col = np.concatenate([g.col + o for g, o in zip(gs, off[:-1])]).astype(np.int32)
    val = np.concatenate([g.val for g in gs])
    p = N.Problem(I.CSR(off[-1], rp, col, val), instances=off)
    a, b = N.ising_default_params(p, eta=1.0, method=1)
    for k, g in enumerate(gs):
        ao, bo = O.alpha_beta(g, eta=1.0, method="eig")
        assert a[k] == pytest.approx(ao, rel=1e-6)
        assert b[k] == pytest.approx(bo, rel=1e-6)
