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


def test_problem_struct_layout_matches_the_header(tmp_path):
    """The ctypes ising_problem_t of the binding has the size and field offsets
    the C compiler gives the header's struct."""
    import ctypes
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    fields = [f for f, _ in N.IsingProblem._fields_]
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "ising.h"\nint main(void) {\n'
                   '  printf("%zu\\n", sizeof(ising_problem_t));\n'
                   + "".join(f'  printf("%zu\\n", offsetof(ising_problem_t, {f}));\n' for f in fields)
                   + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert out[0] == ctypes.sizeof(N.IsingProblem)
    assert out[1:] == [getattr(N.IsingProblem, f).offset for f in fields]


class _Ell:
    def __init__(self, csr, width, pad_first=False):
        n = csr.n
        self.ell_col = np.full((n, width), -1, np.int32)
        self.ell_val = np.zeros((n, width), np.asarray(csr.val).dtype)
        for i in range(n):
            e0, e1 = csr.row_ptr[i], csr.row_ptr[i + 1]
            k0 = width - (e1 - e0) if pad_first else 0
            self.ell_col[i, k0:k0 + e1 - e0] = csr.col[e0:e1]
            self.ell_val[i, k0:k0 + e1 - e0] = csr.val[e0:e1]


def test_ell_input_is_the_csr_problem(lib):
    """ELL rows (empty slots -1, anywhere in the row) load as the same CSR problem:
    the same parameters by the power method, batched too; bad columns are rejected."""
    g = I.regular_gauss(300, 5, seed=611)
    for pad_first in (False, True):
        a_csr, b_csr = N.ising_default_params(N.Problem(g), eta=1.0, method=1)
        a_ell, b_ell = N.ising_default_params(N.Problem(_Ell(g, 8, pad_first)), eta=1.0, method=1)
        assert np.array_equal(a_csr, a_ell) and np.array_equal(b_csr, b_ell)
    gs = [I.regular_pm1(120, 3, seed=612), I.regular_pm1(80, 4, seed=613)]
    off = np.array([0, 120, 200], np.int64)
    rp = np.concatenate([[0], gs[0].row_ptr[1:], gs[1].row_ptr[1:] + gs[0].row_ptr[-1]])
    col = np.concatenate([gs[0].col, gs[1].col + 120]).astype(np.int32)
    J = I.CSR(200, rp, col, np.concatenate([gs[0].val, gs[1].val]))
    a1, b1 = N.ising_default_params(N.Problem(J, instances=off), eta=1.0, method=1)
    a2, b2 = N.ising_default_params(N.Problem(_Ell(J, 6), instances=off), eta=1.0, method=1)
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2)
    bad = _Ell(g, 8)
    bad.ell_col[3, 7] = 300
    with pytest.raises(N.IsingError, match="INDEX_RANGE"):
        N.ising_default_params(N.Problem(bad), eta=1.0, method=1)


def test_dense_values_in_fp8_bf16_and_float_types(lib):
    """Dense couplings may come in any storage type as long as they are integers with
    |J| <= 256: FP8 E4M3 bytes (+1 = 0x38, -1 = 0xB8, 0 = 0x00, 2 = 0x40), BF16,
    F32 give the parameters of the int8 matrix; a non-integer is rejected."""
    Jd = I.dense_pm1(64, seed=614).astype(np.int8)
    Jd[3, 5] = Jd[5, 3] = 2
    ref = N.ising_default_params(N.Problem(Jd), eta=1.0, method=1)
    codes = {1: 0x38, -1: 0xB8, 0: 0x00, 2: 0x40}
    fp8 = np.vectorize(lambda v: codes[int(v)])(Jd).astype(np.uint8)
    got = N.ising_default_params(N.Problem(fp8, jtype=N.FP8E4M3), eta=1.0, method=1)
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])
    bf16 = (Jd.astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)
    got = N.ising_default_params(N.Problem(bf16, jtype=N.BF16), eta=1.0, method=1)
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])
    got = N.ising_default_params(N.Problem(Jd.astype(np.float32)), eta=1.0, method=1)
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])
    half = Jd.astype(np.float32)
    half[1, 2] = half[2, 1] = 0.5
    with pytest.raises(N.IsingError, match="UNSUPPORTED"):
        N.ising_default_params(N.Problem(half), eta=1.0, method=1)


def test_host_exceptions_become_statuses(lib):
    """A problem whose host copy cannot be allocated (a dense n = 2^31 matrix) returns
    ISING_ERR_OOM from the C ABI instead of letting a C++ exception leave it."""
    import ctypes
    small = np.zeros(16, np.int8)
    s = N.IsingProblem()
    s.n, s.format, s.jtype = 1 << 31, N.FMT_DENSE, N.I8
    s.dense = small.ctypes.data
    a = np.zeros(1)
    b = np.zeros(1)
    st = lib.ising_default_params(ctypes.byref(s), 1.0, 1, a.ctypes.data, b.ctypes.data)
    assert st == 6  # ISING_ERR_OOM
    assert "allocation" in lib.ising_last_error().decode()
