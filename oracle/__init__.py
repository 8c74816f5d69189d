"""FP64 oracle for the DOCH Ising solver -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package. The product path (the CUDA library and its
Python binding) never imports, links or runs it, and it shares no code with
that path: the arithmetic lives in ``doch_oracle.c`` (plain C99, FP64,
single-threaded, IEEE semantics with FMA contraction disabled) and in the
numpy parameter rule below.

What each part restates (arXiv 2509.01928):
  * ``doch``          -- Algorithm 1 with the operator T of Eq. FPE.
  * ``hamiltonian``   -- Eq. Hamilton (H = f - g), with -h^T x for a field.
  * ``energy``        -- Eq. IsingModel; ``cut`` per Supplementary Note 5 (W = -2J).
  * ``procedural_rows`` -- rows of J x for J_ij = sin(i j + c) (Supplementary
                         Note 9), 1-based indices, J_ii = 0.
  * ``backward``      -- adjoint of N steps of Eq. FPE (derived; the paper has none).
  * ``adjoint_along`` -- the same adjoint recursion along a given trajectory.
  * ``alpha_beta``    -- Eq. alphabeta; lambda_max by a dense symmetric
                         eigensolver, or by the Wigner estimate of Eq.
                         estimate_eig_J for n >= 1e4 (Supplementary Note 6).
  * ``adoch``         -- Algorithm 2 (ADOCH), Nesterov extrapolation with the
                         non-monotone acceptance test of Eq. BBscheme.
  * ``tune_eta``      -- the choice of eta by probe iterations (Supplementary Note 6).

Readings of the paper used here (where it is silent or ambiguous):
  * field h enters the convex part g, so T(x) = cbrt((Jx + alpha x + h)/beta);
  * sign(0) = +1;  cut weights W = -2J;
  * <J> in the Wigner estimate is the standard deviation of the n(n-1)
    off-diagonal entries (zeros included);
  * alpha_max uses lambda_max(-J) as in Eq. alphabeta;
  * the ADOCH window is H(x^(max(0,k-q))) .. H(x^(k));
  * the procedural matrix sin(i j + c) counts i and j from 1 and has J_ii = 0.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "doch_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORC_CSR, ORC_TORUS, ORC_DENSE = 0, 1, 2

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i8p = ctypes.POINTER(ctypes.c_int8)


class _Problem(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("form", ctypes.c_int32), ("pad_", ctypes.c_int32),
        ("row_ptr", _i64p), ("col", _i32p), ("val", _dp), ("ival", _i64p),
        ("l_rows", ctypes.c_int64), ("l_cols", ctypes.c_int64),
        ("right", _dp), ("down", _dp), ("iright", _i64p), ("idown", _i64p),
        ("dense", _dp), ("idense", _i64p),
        ("h", _dp), ("ih", _i64p),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle's C file into ``liboracle.so`` (gcc, -O2, no FMA contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or (
                os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            subprocess.check_call([
                "gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
                "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER(_Problem)
        lib.orc_coupling_product.argtypes = [P, ctypes.c_int, _dp, _dp]
        lib.orc_hamiltonian.argtypes = [P, ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double, _dp]
        lib.orc_doch.argtypes = [P, ctypes.c_int, _dp, _dp, ctypes.c_int, ctypes.c_double,
                                 ctypes.c_int, _dp]
        lib.orc_doch.restype = ctypes.c_int
        lib.orc_sign.argtypes = [ctypes.c_int64, _dp, _i8p]
        lib.orc_energy.argtypes = [P, ctypes.c_int, _i8p, _dp, _dp]
        lib.orc_energy_int.argtypes = [P, ctypes.c_int, _i8p, _i64p, _i64p]
        lib.orc_backward.argtypes = [P, ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_int,
                                     _dp, _dp, _dp, _i64p]
        lib.orc_backward.restype = ctypes.c_int
        lib.orc_adjoint_along.argtypes = [P, ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_int,
                                          _dp, _dp, _dp, _i64p]
        lib.orc_adjoint_along.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a, typ):
    return None if a is None else a.ctypes.data_as(typ)


class Problem:
    """Coupling matrix J (and optional field h) handed to the oracle in FP64.

    ``J`` is an object with ``row_ptr/col/val`` (CSR), one with ``right/down``
    (2-D torus), or a square ndarray (dense). Integer couplings are also
    kept as int64 for the exact integer energy.
    """

    def __init__(self, J, h=None):
        s = _Problem()
        self._keep = []
        if hasattr(J, "row_ptr"):
            s.form = ORC_CSR
            s.n = J.n
            rp = np.ascontiguousarray(J.row_ptr, dtype=np.int64)
            col = np.ascontiguousarray(J.col, dtype=np.int32)
            val = np.ascontiguousarray(J.val, dtype=np.float64)
            self._keep += [rp, col, val]
            s.row_ptr, s.col, s.val = _ptr(rp, _i64p), _ptr(col, _i32p), _ptr(val, _dp)
            self.integer = np.issubdtype(np.asarray(J.val).dtype, np.integer)
            if self.integer:
                iv = np.ascontiguousarray(J.val, dtype=np.int64)
                self._keep.append(iv)
                s.ival = _ptr(iv, _i64p)
        elif hasattr(J, "right"):
            s.form = ORC_TORUS
            lr, lc = J.right.shape
            s.n, s.l_rows, s.l_cols = lr * lc, lr, lc
            r = np.ascontiguousarray(J.right, dtype=np.float64)
            d = np.ascontiguousarray(J.down, dtype=np.float64)
            self._keep += [r, d]
            s.right, s.down = _ptr(r, _dp), _ptr(d, _dp)
            self.integer = np.issubdtype(J.right.dtype, np.integer)
            if self.integer:
                ir = np.ascontiguousarray(J.right, dtype=np.int64)
                idn = np.ascontiguousarray(J.down, dtype=np.int64)
                self._keep += [ir, idn]
                s.iright, s.idown = _ptr(ir, _i64p), _ptr(idn, _i64p)
        else:
            Jd = np.asarray(J)
            assert Jd.ndim == 2 and Jd.shape[0] == Jd.shape[1]
            s.form = ORC_DENSE
            s.n = Jd.shape[0]
            dd = np.ascontiguousarray(Jd, dtype=np.float64)
            self._keep.append(dd)
            s.dense = _ptr(dd, _dp)
            self.integer = np.issubdtype(Jd.dtype, np.integer)
            if self.integer:
                idd = np.ascontiguousarray(Jd, dtype=np.int64)
                self._keep.append(idd)
                s.idense = _ptr(idd, _i64p)
        if h is not None:
            hh = np.ascontiguousarray(h, dtype=np.float64)
            assert hh.shape == (s.n,)
            self._keep.append(hh)
            s.h = _ptr(hh, _dp)
            if np.issubdtype(np.asarray(h).dtype, np.integer):
                ih = np.ascontiguousarray(h, dtype=np.int64)
                self._keep.append(ih)
                s.ih = _ptr(ih, _i64p)
            else:
                self.integer = False
        self.n = int(s.n)
        self.has_h = h is not None
        self._s = s

    @property
    def ref(self):
        return ctypes.byref(self._s)


def _state(x, n):
    x = np.array(x, dtype=np.float64, order="C", copy=True)
    if x.ndim == 1:
        x = x.reshape(n, 1)
    assert x.shape[0] == n
    return x


def coupling_product(p: Problem, x) -> np.ndarray:
    """u = J x for every replica column of x ([n][R])."""
    x = _state(x, p.n)
    u = np.empty_like(x)
    _load().orc_coupling_product(p.ref, x.shape[1], _ptr(x, _dp), _ptr(u, _dp))
    return u


def procedural_rows(n: int, c: int, rows, x) -> np.ndarray:
    """u_i = sum_{j != i} sin(i j + c) x_j for the listed 0-based rows of the
    procedural matrix of Supplementary Note 9 (1-based i, j in the formula),
    one row at a time in FP64 (i j + c is an exact double below 2^53).
    x: [n][R]; returns [len(rows)][R]."""
    x = _state(x, n)
    cols = np.arange(1, n + 1, dtype=np.float64)
    out = np.empty((len(rows), x.shape[1]))
    for k, i in enumerate(rows):
        w = np.sin((i + 1) * cols + float(c))
        w[i] = 0.0
        out[k] = w @ x
    return out


def hamiltonian(p: Problem, x, alpha: float, beta: float) -> np.ndarray:
    """H(x) per replica (Eq. Hamilton, with -h^T x)."""
    x = _state(x, p.n)
    H = np.empty(x.shape[1])
    _load().orc_hamiltonian(p.ref, x.shape[1], _ptr(x, _dp), float(alpha), float(beta),
                            _ptr(H, _dp))
    return H


def doch(p: Problem, x0, alpha, beta: float, iters: int, trace: bool = False):
    """Algorithm 1: returns x^(N) ([n][R], FP64) and optionally H(x^(k)), k=0..N."""
    x = _state(x0, p.n)
    R = x.shape[1]
    a = np.atleast_1d(np.asarray(alpha, dtype=np.float64))
    H = np.empty((iters + 1, R)) if trace else None
    rc = _load().orc_doch(p.ref, R, _ptr(x, _dp), _ptr(a, _dp), a.size, float(beta), int(iters),
                          _ptr(H, _dp))
    if rc:
        raise ValueError(f"orc_doch failed ({rc})")
    return (x, H) if trace else x


def doch_until(p: Problem, x0, alpha: float, beta: float, max_iters: int, eps: float):
    """Algorithm 1 with the stopping rule of Remark S2, per replica: after each
    step, r^(k) = ||x^(k+1) - x^(k)||_2 / ||x^(k)||_2; the replica stops at the
    first k with r^(k) < eps, keeping x^(k+1). Returns x ([n][R], each replica's
    last iterate), the steps taken per replica ([R], <= max_iters) and the
    trace r ([max_iters][R], NaN after a replica stopped)."""
    x = _state(x0, p.n)
    R = x.shape[1]
    steps = np.full(R, max_iters, dtype=np.int32)
    rtr = np.full((max_iters, R), np.nan)
    for r in range(R):
        xk = x[:, r:r + 1].copy()
        for k in range(max_iters):
            xn = doch(p, xk, alpha, beta, 1)
            rtr[k, r] = np.linalg.norm(xn - xk) / np.linalg.norm(xk)
            xk = xn
            if rtr[k, r] < eps:
                steps[r] = k + 1
                break
        x[:, r] = xk[:, 0]
    return x, steps, rtr


def sign(x) -> np.ndarray:
    """s = sign(x) with sign(0) = +1, int8."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    s = np.empty(x.shape, dtype=np.int8)
    _load().orc_sign(x.size, _ptr(x, _dp), _ptr(s, _i8p))
    return s


def energy(p: Problem, s):
    """(E, cut) per replica in FP64 for a spin array s ([n][R] or [n], +-1)."""
    s = np.ascontiguousarray(s, dtype=np.int8)
    if s.ndim == 1:
        s = s.reshape(-1, 1)
    R = s.shape[1]
    E, cut = np.empty(R), np.empty(R)
    _load().orc_energy(p.ref, R, _ptr(s, _i8p), _ptr(E, _dp), _ptr(cut, _dp))
    return E, cut


def energy_int(p: Problem, s):
    """(E, cut) per replica in exact int64 arithmetic (integer J and h only)."""
    if not p.integer:
        raise ValueError("integer energy needs integer couplings and field")
    s = np.ascontiguousarray(s, dtype=np.int8)
    if s.ndim == 1:
        s = s.reshape(-1, 1)
    R = s.shape[1]
    E, cut = np.empty(R, dtype=np.int64), np.empty(R, dtype=np.int64)
    _load().orc_energy_int(p.ref, R, _ptr(s, _i8p), _ptr(E, _i64p), _ptr(cut, _i64p))
    return E, cut


def backward(p: Problem, x0, alpha, beta: float, iters: int):
    """Adjoint of N DOCH steps: (grad_alpha[N], grad_x0[n][R], loss, zero_events)."""
    x0 = _state(x0, p.n)
    R = x0.shape[1]
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(alpha, dtype=np.float64), (iters,)))
    ga = np.empty(iters)
    gx = np.empty_like(x0)
    loss = ctypes.c_double(0.0)
    zeros = ctypes.c_int64(0)
    rc = _load().orc_backward(p.ref, R, _ptr(x0, _dp), _ptr(a, _dp), float(beta), int(iters),
                              _ptr(ga, _dp), _ptr(gx, _dp), ctypes.byref(loss), ctypes.byref(zeros))
    if rc:
        raise ValueError(f"orc_backward failed ({rc})")
    return ga, gx, loss.value, zeros.value


def adjoint_along_replica(p: Problem, xs, alpha, beta: float, R: int):
    """The adjoint recursion of ``backward`` for ONE replica along a GIVEN
    trajectory xs = (x^(0), ..., x^(N)) ([N+1][n], used as it is, in FP64)
    instead of the oracle's own iterates. R is the replica count of the mean
    in L. Returns (this replica's dL/dalpha [N], dL/dx^(0) [n], its share of
    L, its count of components with x^(k+1) = 0)."""
    a = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64).ravel())
    iters = a.size
    xs = np.ascontiguousarray(xs, dtype=np.float64)
    assert xs.shape == (iters + 1, p.n)
    ga = np.zeros(iters)
    g1 = np.empty(p.n)
    loss = ctypes.c_double(0.0)
    zeros = ctypes.c_int64(0)
    rc = _load().orc_adjoint_along(p.ref, int(R), _ptr(xs, _dp), _ptr(a, _dp), float(beta), iters,
                                   _ptr(ga, _dp), _ptr(g1, _dp), ctypes.byref(loss), ctypes.byref(zeros))
    if rc:
        raise ValueError(f"orc_adjoint_along failed ({rc})")
    return ga, g1, loss.value, zeros.value


def adjoint_along(p: Problem, trajectory, alpha, beta: float, R: int | None = None):
    """adjoint_along_replica for every replica of a trajectory [N+1][n][Rs]
    (R defaults to Rs; a subset of a larger run passes the full count).
    Returns (grad_alpha[N] summed over the replicas in replica order,
    grad_x0[n][Rs], the replicas' share of L, zero_events)."""
    t = np.asarray(trajectory)
    Rs = t.shape[2]
    R = Rs if R is None else int(R)
    ga = np.zeros(t.shape[0] - 1)
    gx = np.empty((p.n, Rs))
    loss, zeros = 0.0, 0
    for r in range(Rs):
        g, gx[:, r], l, z = adjoint_along_replica(p, t[:, :, r], alpha, beta, R)
        ga += g
        loss += l
        zeros += z
    return ga, gx, loss, zeros


# ---------------------------------------------------------------------------
# parameter rule (Eq. alphabeta, Eq. estimate_eig_J, Supplementary Note 6)
# ---------------------------------------------------------------------------

def _stats(J):
    """(n, sum of off-diagonal entries, sum of squares, max_j sum_i |J_ij|)."""
    if hasattr(J, "row_ptr"):
        v = np.asarray(J.val, dtype=np.float64)
        rows = np.repeat(np.arange(J.n), np.diff(J.row_ptr))
        rowabs = np.bincount(rows, weights=np.abs(v), minlength=J.n)
        return J.n, v.sum(), (v * v).sum(), rowabs.max()
    if hasattr(J, "right"):
        r = np.asarray(J.right, dtype=np.float64)
        d = np.asarray(J.down, dtype=np.float64)
        # site (a,b) touches right[a,b], right[a,b-1], down[a,b], down[a-1,b]
        rowabs = (np.abs(r) + np.abs(np.roll(r, 1, axis=1))
                  + np.abs(d) + np.abs(np.roll(d, 1, axis=0)))
        return r.size, 2 * (r.sum() + d.sum()), 2 * ((r * r).sum() + (d * d).sum()), rowabs.max()
    Jd = np.asarray(J, dtype=np.float64)
    return Jd.shape[0], Jd.sum(), (Jd * Jd).sum(), np.abs(Jd).sum(axis=1).max()


def wigner_lambda(J) -> float:
    """Eq. estimate_eig_J: lambda_max ~ 2 <J> sqrt(n), <J> = std of off-diagonal entries."""
    n, s1, s2, _ = _stats(J)
    m = n * (n - 1.0)
    mean = s1 / m
    var = s2 / m - mean * mean
    return 2.0 * np.sqrt(max(var, 0.0)) * np.sqrt(n)


def lambda_max_neg(J) -> float:
    """lambda_max(-J) = -lambda_min(J), by a dense symmetric eigensolver."""
    if hasattr(J, "to_dense"):
        Jd = J.to_dense()
    elif hasattr(J, "right"):
        Jd = J.to_csr().to_dense()
    else:
        Jd = np.asarray(J, dtype=np.float64)
    return float(-np.linalg.eigvalsh(Jd)[0])


def alpha_beta(J, eta: float = 1.0, method: str = "auto"):
    """Eq. alphabeta: alpha = eta * lambda_max(-J), beta = n^1.5 * max_j (alpha + sum_i |J_ij|).

    method: "eig" (dense eigensolver), "wigner" (Eq. estimate_eig_J) or
    "auto" (eigensolver below n = 1e4, Wigner from there on, as the paper does).
    """
    n, _, _, rowabs = _stats(J)
    if method == "auto":
        method = "eig" if n < 10_000 else "wigner"
    lam = lambda_max_neg(J) if method == "eig" else wigner_lambda(J)
    alpha = eta * lam
    beta = float(n) ** 1.5 * (alpha + rowabs)
    return float(alpha), float(beta)


def tune_eta(p: Problem, x0, etas, probe_iters: int, alpha1: float, beta1: float):
    """Choice of eta in alpha = eta * lambda_max(-J) by a few probe iterations
    (Supplementary Note 6: eta in (0, 2] is tuned by examining the Ising energy
    over the first iterations, 5-10 for large graphs, 1-3 for ultra-large ones).

    alpha1, beta1 are Eq. alphabeta at eta = 1 (alpha1 = lambda_max(-J));
    since beta = n^1.5 (alpha + max_j sum_i |J_ij|) is affine in alpha, the
    candidate eta has alpha = eta alpha1 and beta = beta1 + n^1.5 (eta - 1) alpha1.
    For each candidate (in the given order): probe_iters DOCH steps from x0,
    then the Ising energy of sign(x) per replica (exact int64 for integer J,
    FP64 otherwise). Score = the best (lowest) energy over the replicas; the
    chosen candidate has the lowest score, ties broken by the lower mean energy
    and then by the earlier position. Returns (best[k], mean[k], index)."""
    etas = [float(e) for e in etas]
    n = float(p.n)
    best, mean = [], []
    for eta in etas:
        a = eta * alpha1
        b = beta1 + n ** 1.5 * (eta - 1.0) * alpha1
        x = doch(p, x0, a, b, probe_iters)
        s = sign(x)
        E = energy_int(p, s)[0] if p.integer else energy(p, s)[0]
        best.append(float(E.min()))
        mean.append(float(np.mean(E.astype(np.float64))))
    order = sorted(range(len(etas)), key=lambda k: (best[k], mean[k], k))
    return np.array(best), np.array(mean), order[0]


# ---------------------------------------------------------------------------
# ADOCH, Algorithm 2
# ---------------------------------------------------------------------------

def adoch(p: Problem, x0, alpha: float, beta: float, iters: int, q: int, decisions=None,
          margins: bool = False):
    """Algorithm 2 (ADOCH) per replica: returns x^(N) ([n][R]) and the
    per-iteration acceptance flags [N][R] (1 where the extrapolated point was used).

    t_0 = 1, t_(k+1) = (1 + sqrt(1 + 4 t_k^2)) / 2; for k >= 1,
    y^k = x^k + ((t_k - 1)/t_(k+1)) (x^k - x^(k-1)), y^0 = x^0;
    v^k = y^k if H(y^k) <= max(H(x^(max(0,k-q))), ..., H(x^k)) else x^k;
    x^(k+1) = T(v^k).

    decisions: optional [N][R] flags that replace the test (v^k = y^k where 1),
    to follow a trajectory whose near-tied decisions were taken elsewhere.
    margins: also return the signed margin (window max - H(y^k)) / |H(x^k)| of
    the test per step and replica (>= 0 where it accepts; inf at k = 0, where
    y^0 = x^0 and the test accepts exactly).
    """
    x = _state(x0, p.n)
    R = x.shape[1]
    out = np.empty_like(x)
    acc = np.zeros((iters, R), dtype=np.int8)
    marg = np.full((iters, R), np.inf)
    for r in range(R):
        xk = x[:, r:r + 1].copy()
        xprev = xk.copy()
        hist = [hamiltonian(p, xk, alpha, beta)[0]]
        t = 1.0
        for k in range(iters):
            t_next = (1.0 + np.sqrt(1.0 + 4.0 * t * t)) / 2.0
            if k >= 1:
                y = xk + ((t - 1.0) / t_next) * (xk - xprev)
            else:
                y = xk.copy()
            window = hist[max(0, k - q):k + 1]
            hy = hamiltonian(p, y, alpha, beta)[0]
            if k >= 1:
                marg[k, r] = (max(window) - hy) / abs(hist[-1])
            take = hy <= max(window) if decisions is None else bool(decisions[k][r])
            if take:
                v = y
                acc[k, r] = 1
            else:
                v = xk
            xnew = doch(p, v, alpha, beta, 1)
            xprev, xk = xk, xnew
            hist.append(hamiltonian(p, xk, alpha, beta)[0])
            t = t_next
        out[:, r] = xk[:, 0]
    if margins:
        return out, acc, marg
    return out, acc
