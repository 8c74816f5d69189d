"""ctypes binding of libising_doch.so: argument marshalling only.

Every function here has the name of the C entry point it calls (see
include/ising.h) and does nothing but turn numpy arrays / torch tensors into
pointers, sizes and enum values. All arithmetic of the method runs in the
CUDA library. If the library has not been built this module raises: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libising_doch.so")

# enums of include/ising.h
ISING_OK = 0
STATUS_NAMES = {
    0: "ISING_OK", 1: "ISING_ERR_INVALID_ARG", 2: "ISING_ERR_NOT_SYMMETRIC",
    3: "ISING_ERR_NONZERO_DIAG", 4: "ISING_ERR_INDEX_RANGE", 5: "ISING_ERR_NONFINITE",
    6: "ISING_ERR_OOM", 7: "ISING_ERR_CUDA", 8: "ISING_ERR_TIMEOUT", 9: "ISING_ERR_NOT_MONOTONE",
    10: "ISING_ERR_UNSUPPORTED",
}
FMT_CSR, FMT_TORUS2D, FMT_DENSE, FMT_PROCEDURAL, FMT_ELL = 0, 1, 2, 3, 4
I8, I16, I32, FP8E4M3, BF16, F32, F64 = range(7)
FLAG_ASYNC, FLAG_SKIP_VALIDATION, FLAG_STRICT_MONOTONE, FLAG_SINGLE_STEP = 1, 2, 4, 8

_vp = ctypes.c_void_p


class IsingProblem(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("format", ctypes.c_int32), ("jtype", ctypes.c_int32),
        ("row_ptr", _vp), ("col", _vp), ("val", _vp),
        ("l_rows", ctypes.c_int64), ("l_cols", ctypes.c_int64), ("right", _vp), ("down", _vp),
        ("dense", _vp), ("h", _vp), ("htype", ctypes.c_int32), ("n_instances", ctypes.c_int32),
        ("inst_offset", _vp), ("ell_width", ctypes.c_int64),
    ]


class IsingError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        self.name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{where}: {self.name}: {message}")


_lib = None


def load():
    """Load libising_doch.so (built in-tree by paper_2509_01928_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            "libising_doch.so is not built; run paper_2509_01928_gb300.build.build() "
            "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    st = ctypes.c_int
    P = ctypes.POINTER(IsingProblem)
    lib.ising_default_params.argtypes = [P, ctypes.c_double, ctypes.c_int32, _vp, _vp]
    lib.ising_create.argtypes = [P, ctypes.c_int32, ctypes.POINTER(_vp)]
    lib.ising_destroy.argtypes = [_vp]
    lib.ising_destroy.restype = None
    lib.ising_iterate.argtypes = [_vp, _vp, ctypes.c_int32, ctypes.c_int32, _vp, ctypes.c_int32, _vp,
                                  ctypes.c_int32, _vp, _vp]
    lib.ising_iterate_adoch.argtypes = [_vp, _vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp, ctypes.c_int32,
                                        ctypes.c_int32, _vp, _vp, _vp]
    lib.ising_iterate_until.argtypes = [_vp, _vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp, ctypes.c_int32,
                                        ctypes.c_double, _vp, _vp]
    lib.ising_create_s5.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_uint64, ctypes.c_int32,
                                    ctypes.POINTER(_vp)]
    lib.ising_create_procedural.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(_vp)]
    lib.ising_params_device.argtypes = [_vp, ctypes.c_double, ctypes.c_int32, _vp, _vp]
    lib.ising_csr_export.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
    lib.ising_energy.argtypes = [_vp, _vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
    lib.ising_backward.argtypes = [_vp, _vp, ctypes.c_int32, ctypes.c_int32, _vp, ctypes.c_int32,
                                   ctypes.c_double, ctypes.c_int32, _vp, _vp, _vp, _vp, _vp]
    lib.ising_synchronize.argtypes = [_vp, _vp]
    lib.ising_get_size.argtypes = [_vp, _vp, _vp]
    lib.ising_energy_torus_noalloc.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_int64, _vp,
                                               ctypes.c_int32, _vp, _vp, _vp]
    lib.ising_energy_torus_noalloc.restype = ctypes.c_int
    lib.ising_selftest_cbrt.argtypes = [_vp, _vp, _vp, ctypes.c_int64, ctypes.c_int32, _vp]
    lib.ising_selftest_cbrt.restype = ctypes.c_int
    lib.ising_selftest_cbrt_log.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_float, _vp]
    lib.ising_selftest_cbrt_log.restype = ctypes.c_int
    lib.ising_selftest_procedural.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                              ctypes.c_int64, _vp, _vp]
    lib.ising_selftest_procedural.restype = ctypes.c_int
    lib.ising_tune_eta.argtypes = [_vp, _vp, ctypes.c_int32, ctypes.c_int32, _vp, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_double, ctypes.c_double, _vp, _vp, _vp, _vp, _vp, _vp]
    lib.ising_tune_eta.restype = ctypes.c_int
    lib.ising_selftest_wait.argtypes = [_vp, ctypes.c_int32, ctypes.c_int64, _vp]
    lib.ising_selftest_wait.restype = ctypes.c_int
    lib.ising_status_string.argtypes = [ctypes.c_int]
    lib.ising_status_string.restype = ctypes.c_char_p
    lib.ising_last_error.argtypes = []
    lib.ising_last_error.restype = ctypes.c_char_p
    for name in ("ising_default_params", "ising_create", "ising_iterate", "ising_iterate_adoch", "ising_iterate_until",
                 "ising_energy", "ising_create_s5", "ising_create_procedural", "ising_params_device", "ising_csr_export",
                 "ising_backward", "ising_synchronize", "ising_get_size"):
        getattr(lib, name).restype = st
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != ISING_OK:
        msg = _lib.ising_last_error().decode(errors="replace")
        raise IsingError(status, where, msg)


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _dtype_code(a) -> int:
    if _is_torch(a):
        import torch
        table = {torch.int8: I8, torch.int16: I16, torch.int32: I32, torch.bfloat16: BF16,
                 torch.float32: F32, torch.float64: F64}
        if hasattr(torch, "float8_e4m3fn"):
            table[torch.float8_e4m3fn] = FP8E4M3
        return table[a.dtype]
    table = {np.dtype(np.int8): I8, np.dtype(np.int16): I16, np.dtype(np.int32): I32,
             np.dtype(np.float32): F32, np.dtype(np.float64): F64}
    return table[np.asarray(a).dtype]


def _ptr(a):
    """Address of a contiguous numpy array or torch tensor (host or device)."""
    if a is None:
        return None
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if not (isinstance(a, np.ndarray) and a.flags.c_contiguous):
        raise ValueError("array must be a C-contiguous numpy array")
    return a.ctypes.data


def _stream(stream, *tensors):
    if stream is not None:
        return int(stream)
    for t in tensors:
        if t is not None and _is_torch(t) and t.is_cuda:
            import torch
            return torch.cuda.current_stream(t.device).cuda_stream
    return 0


def _f64(a, count=None):
    if a is None:
        return None
    out = np.ascontiguousarray(np.asarray(a, dtype=np.float64)).reshape(-1)
    if count is not None and out.size != count:
        raise ValueError(f"expected {count} values, got {out.size}")
    return out


class Problem:
    """Marshals a coupling matrix into an ising_problem_t (keeps the arrays alive).

    J: an object with row_ptr/col/val (CSR), one with ell_col/ell_val ([n][w]
    ELL rows, column -1 for an empty slot), one with right/down (2-D torus), or
    a square array (dense). instances: optional spin offsets [B + 1] for a
    batch of CSR/ELL instances concatenated along n. jtype overrides the type
    code of J's values (e.g. FP8E4M3 for raw E4M3 bytes held in a uint8 array).
    """

    def __init__(self, J, h=None, instances=None, jtype=None):
        s = IsingProblem()
        keep = []

        def code(a):
            return _dtype_code(a) if jtype is None else int(jtype)

        def arr(a, dtype=None):
            if _is_torch(a):
                a = a.contiguous()
            else:
                a = np.ascontiguousarray(a if dtype is None else np.asarray(a, dtype=dtype))
            keep.append(a)
            return a

        if hasattr(J, "row_ptr"):
            rp = arr(J.row_ptr, np.int64)
            col = arr(J.col, np.int32)
            val = arr(J.val)
            s.n = int(rp.shape[0]) - 1
            s.format, s.jtype = FMT_CSR, code(val)
            s.row_ptr, s.col, s.val = _ptr(rp), _ptr(col), _ptr(val)
        elif hasattr(J, "ell_col"):
            col = arr(J.ell_col, np.int32)
            val = arr(J.ell_val)
            s.n, s.ell_width = int(col.shape[0]), int(col.shape[1])
            s.format, s.jtype = FMT_ELL, code(val)
            s.col, s.val = _ptr(col), _ptr(val)
        elif hasattr(J, "right"):
            r = arr(J.right)
            d = arr(J.down)
            lr, lc = r.shape
            s.n, s.l_rows, s.l_cols = lr * lc, lr, lc
            s.format, s.jtype = FMT_TORUS2D, code(r)
            s.right, s.down = _ptr(r), _ptr(d)
        else:
            D = arr(J)
            s.n = int(D.shape[0])
            s.format, s.jtype = FMT_DENSE, code(D)
            s.dense = _ptr(D)
        if h is not None:
            hh = arr(h)
            s.h, s.htype = _ptr(hh), _dtype_code(hh)
        if instances is not None:
            off = arr(instances, np.int64)
            s.n_instances = int(off.shape[0]) - 1
            s.inst_offset = _ptr(off)
        self.struct = s
        self._keep = keep
        self.n = int(s.n)
        self.n_instances = max(1, int(s.n_instances))


# ---------------------------------------------------------------------------
# entry points
# ---------------------------------------------------------------------------

def ising_default_params(problem: Problem, eta: float = 1.0, method: int = 0):
    """Eq. alphabeta per instance: returns (alpha[B], beta[B]) as float64 arrays."""
    lib = load()
    a = np.zeros(problem.n_instances)
    b = np.zeros(problem.n_instances)
    _check(lib.ising_default_params(ctypes.byref(problem.struct), float(eta), int(method),
                                    a.ctypes.data, b.ctypes.data), "ising_default_params")
    return a, b


def ising_create(problem: Problem, flags: int = 0) -> int:
    lib = load()
    h = _vp()
    _check(lib.ising_create(ctypes.byref(problem.struct), int(flags), ctypes.byref(h)), "ising_create")
    return h.value


def ising_destroy(handle: int) -> None:
    load().ising_destroy(handle)


def ising_get_size(handle: int):
    n = ctypes.c_int64()
    b = ctypes.c_int32()
    _check(load().ising_get_size(handle, ctypes.byref(n), ctypes.byref(b)), "ising_get_size")
    return n.value, b.value


def ising_iterate(handle: int, x, alpha, beta, iters: int, H_trace=None, stream=None,
                  n_instances: int = 1):
    """In-place DOCH iterations on x ([n][R] or [n]); alpha [B][len] and beta [B] host values."""
    R = 1 if x.ndim == 1 else int(x.shape[1])
    a = _f64(alpha)
    b = _f64(beta)
    alpha_len = a.size // max(1, n_instances)
    _check(load().ising_iterate(handle, _ptr(x), _dtype_code(x), R, a.ctypes.data, alpha_len,
                                b.ctypes.data, int(iters), _ptr(H_trace), _stream(stream, x)),
           "ising_iterate")
    return x


def ising_iterate_adoch(handle: int, x, alpha, beta, iters: int, q: int, accepted=None, H_trace=None,
                        stream=None):
    """In-place ADOCH iterations (Algorithm 2) on x ([n][R] or [n]); alpha [B] and beta [B] host values;
    optional accepted [iters][B R] int8 and H_trace [iters + 1][B R] FP64 outputs."""
    R = 1 if x.ndim == 1 else int(x.shape[1])
    a = _f64(alpha)
    b = _f64(beta)
    _check(load().ising_iterate_adoch(handle, _ptr(x), _dtype_code(x), R, a.ctypes.data, b.ctypes.data,
                                      int(iters), int(q), _ptr(accepted), _ptr(H_trace),
                                      _stream(stream, x, accepted, H_trace)),
           "ising_iterate_adoch")
    return x


def ising_iterate_until(handle: int, x, alpha, beta, max_iters: int, eps: float, steps=None, stream=None):
    """DOCH with the stopping rule of Remark S2 per (instance, replica), in place on x;
    alpha [B] and beta [B] host values; optional steps [B R] int32 output."""
    R = 1 if x.ndim == 1 else int(x.shape[1])
    a = _f64(alpha)
    b = _f64(beta)
    _check(load().ising_iterate_until(handle, _ptr(x), _dtype_code(x), R, a.ctypes.data, b.ctypes.data,
                                      int(max_iters), float(eps), _ptr(steps), _stream(stream, x, steps)),
           "ising_iterate_until")
    return x


def ising_create_s5(n: int, p: float, seed: int, flags: int = 0) -> int:
    """Handle of the Algorithm S5 matrix (n spins, p percent), generated on the device."""
    out = ctypes.c_void_p()
    _check(load().ising_create_s5(int(n), float(p), int(seed) & 0xFFFFFFFFFFFFFFFF, int(flags), ctypes.byref(out)),
           "ising_create_s5")
    return out.value


def ising_create_procedural(n: int, c: int = 100, flags: int = 0) -> int:
    """Handle of the procedural dense couplings J_ij = sin(i j + c) (1-based, J_ii = 0)."""
    out = ctypes.c_void_p()
    _check(load().ising_create_procedural(int(n), int(c), int(flags), ctypes.byref(out)), "ising_create_procedural")
    return out.value


def ising_selftest_procedural(row0: int, rows: int, col0: int, cols: int, c: int, out, stream=None):
    """Device couplings sin(i j + c) of a block of rows and columns, generated as the product kernels
    generate them, into out ([rows][cols] FP32 on the device)."""
    _check(load().ising_selftest_procedural(int(row0), int(rows), int(col0), int(cols), int(c), _ptr(out),
                                            _stream(stream, out)), "ising_selftest_procedural")


def ising_params_device(handle: int, eta: float = 1.0, method: int = 0):
    """(alpha, beta) of Eq. alphabeta computed on the device for a one-instance handle."""
    a = np.zeros(1)
    b = np.zeros(1)
    _check(load().ising_params_device(handle, float(eta), int(method), a.ctypes.data, b.ctypes.data),
           "ising_params_device")
    return a, b


def ising_csr_export(handle: int):
    """(row_ptr, col, val) of a CSR handle, copied to host numpy arrays."""
    lib = load()
    nnz = ctypes.c_int64()
    jt = ctypes.c_int32()
    _check(lib.ising_csr_export(handle, None, None, None, ctypes.byref(nnz), ctypes.byref(jt)), "ising_csr_export")
    n = ctypes.c_int64()
    _check(lib.ising_get_size(handle, ctypes.byref(n), None), "ising_get_size")
    rp = np.zeros(n.value + 1, np.int64)
    col = np.zeros(max(1, nnz.value), np.int32)
    vdt = {I8: np.int8, I32: np.int32, F32: np.float32, F64: np.float64}[jt.value]
    val = np.zeros(max(1, nnz.value), vdt)
    _check(lib.ising_csr_export(handle, rp.ctypes.data, col.ctypes.data, val.ctypes.data, None, None),
           "ising_csr_export")
    return rp, col[:nnz.value], val[:nnz.value]


def ising_energy(handle: int, x, E_int=None, cut_int=None, E_f64=None, cut_f64=None, best=None,
                 spins=None, stream=None):
    """Sign rounding + energy/cut per (instance, replica) into the given output arrays."""
    R = 1 if x.ndim == 1 else int(x.shape[1])
    _check(load().ising_energy(handle, _ptr(x), _dtype_code(x), R, _ptr(E_int), _ptr(cut_int),
                               _ptr(E_f64), _ptr(cut_f64), _ptr(best), _ptr(spins),
                               _stream(stream, x, E_int, E_f64)), "ising_energy")


def ising_tune_eta(handle: int, x0, etas, probe_iters: int, alpha1: float, beta1: float, stream=None):
    """eta by probe iterations (Supplementary Note 6): returns (alpha, beta, index, score_best[k],
    score_mean[k]) of the chosen candidate among etas, all starts in x0 ([n][R] or [n])."""
    R = 1 if x0.ndim == 1 else int(x0.shape[1])
    e = _f64(etas)
    k = e.size
    best, mean = np.zeros(k), np.zeros(k)
    idx = np.zeros(1, np.int32)
    a, b = np.zeros(1), np.zeros(1)
    _check(load().ising_tune_eta(handle, _ptr(x0), _dtype_code(x0), R, e.ctypes.data, k, int(probe_iters),
                                 float(alpha1), float(beta1), best.ctypes.data, mean.ctypes.data, idx.ctypes.data,
                                 a.ctypes.data, b.ctypes.data, _stream(stream, x0)), "ising_tune_eta")
    return float(a[0]), float(b[0]), int(idx[0]), best, mean


def ising_backward(handle: int, x0, alpha, beta: float, iters: int, ckpt_every: int,
                   grad_alpha=None, grad_x0=None, loss=None, zero_events=None, stream=None):
    """Adjoint of `iters` DOCH steps into the given output arrays."""
    R = 1 if x0.ndim == 1 else int(x0.shape[1])
    a = _f64(alpha, iters)
    _check(load().ising_backward(handle, _ptr(x0), _dtype_code(x0), R, a.ctypes.data, int(iters),
                                 float(beta), int(ckpt_every), _ptr(grad_alpha), _ptr(grad_x0),
                                 _ptr(loss), _ptr(zero_events), _stream(stream, x0, grad_x0)),
           "ising_backward")


def ising_energy_torus_noalloc(right, down, x, E_out=None, cut_out=None, stream=None):
    """Lattice energy/cut from device arrays, with no device allocation (see include/ising.h).

    The C entry point cannot see array lengths, so the arguments are checked here before
    the call: right and down int8 torch tensors of one 2-D shape [l_rows][l_cols]; x a
    float32 tensor [n] or [n][R] with n = l_rows * l_cols; E_out and cut_out int64 tensors
    of at least R elements; all contiguous CUDA tensors on x's device (the call runs with
    that device current). ValueError otherwise."""
    import torch

    def need(cond, msg):
        if not cond:
            raise ValueError(f"ising_energy_torus_noalloc: {msg}")

    for name, t in (("right", right), ("down", down), ("x", x), ("E_out", E_out), ("cut_out", cut_out)):
        need(t is None or isinstance(t, torch.Tensor), f"{name} must be a torch tensor")
    need(E_out is not None or cut_out is not None, "give E_out, cut_out or both")
    need(right.dtype == torch.int8 and down.dtype == torch.int8, "right and down must be int8")
    need(right.dim() == 2 and tuple(down.shape) == tuple(right.shape), "right and down must share one 2-D shape")
    lr, lc = int(right.shape[0]), int(right.shape[1])
    need(x.dtype == torch.float32, "x must be float32")
    need(x.dim() in (1, 2) and int(x.shape[0]) == lr * lc, "x must be [l_rows * l_cols] or [l_rows * l_cols][R]")
    R = 1 if x.dim() == 1 else int(x.shape[1])
    for name, t in (("E_out", E_out), ("cut_out", cut_out)):
        if t is not None:
            need(t.dtype == torch.int64 and t.numel() >= R, f"{name} must be int64 with at least R = {R} elements")
    tensors = [t for t in (right, down, x, E_out, cut_out) if t is not None]
    need(all(t.is_contiguous() for t in tensors), "every tensor must be contiguous")
    need(all(t.is_cuda for t in tensors), "every tensor must be a CUDA tensor")
    need(all(t.device == x.device for t in tensors), "every tensor must be on x's device")
    with torch.cuda.device(x.device):
        _check(load().ising_energy_torus_noalloc(_ptr(right), _ptr(down), lr, lc, _ptr(x), R,
                                                 _ptr(E_out), _ptr(cut_out), _stream(stream, x)),
               "ising_energy_torus_noalloc")


def ising_selftest_wait(handle: int, arrive: bool, limit_ns: int, stream=None):
    """One bounded mbarrier wait of limit_ns on the device (see include/ising.h): raises
    IsingError(ISING_ERR_TIMEOUT) when nothing arrives."""
    _check(load().ising_selftest_wait(handle, 1 if arrive else 0, int(limit_ns), _stream(stream)),
           "ising_selftest_wait")


def ising_synchronize(handle: int, stream=None):
    _check(load().ising_synchronize(handle, _stream(stream)), "ising_synchronize")


def ising_status_string(status: int) -> str:
    return load().ising_status_string(int(status)).decode()
