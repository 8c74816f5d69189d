"""GPU parity of the DOCH iteration and readout against the FP64 oracle.

Every case feeds the same seeded inputs to the CUDA library (through the C
ABI) and to the oracle, and compares element by element:
  * FP32 iterates: max_r ||x_gpu - x_ref|| / ||x_ref|| <= 1e-5 (the FP32
    tolerance of the accuracy bar, a vector criterion), and every element
    within 10x that of max|x_ref|: a wrong neighbour or a missed tile seam
    shows up as an O(1) error in one element. The element bound is looser
    because a component whose sum u_i + alpha x_i nearly cancels is small,
    and the cube root multiplies the FP32 rounding of that sum by
    1 / (3 x_i^2);
  * FP64 iterates: the same with 1e-10 (summation order only);
  * FP32 iterates on graphs with weakly stable fixed points (random
    regular graphs): some replicas drift from the FP64 trajectory by more
    than 1e-5 under FP32 rounding alone, because the iteration contracts
    slowly there. For those tests each replica r must satisfy
    rel_r <= max(1e-5, 16 delta_r), where delta_r is the drift of the oracle
    trajectory when every step's output is perturbed by one FP32 rounding
    (relative 2^-24, seeded signs), and the median replica must be within
    1e-5;
  * integer energies and cuts of a given spin vector: bit-exact;
  * FP64 energies: 1e-12 relative.
"""
import numpy as np
import pytest

import oracle as O
from paper_2509_01928_gb300 import _native as N
from paper_2509_01928_gb300 import build as B
from paper_2509_01928_gb300 import inputs as I
from fp32_bounds import close32_conditioned, fp32_drift
from short_rows import short_rows_mixed

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-10


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build_library()
    return N.load()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _close(x_gpu, x_ref, tol):
    x_gpu = np.asarray(x_gpu, dtype=np.float64).reshape(x_ref.shape)
    if x_ref.ndim == 1:
        x_ref = x_ref[:, None]
        x_gpu = x_gpu[:, None]
    rel = np.linalg.norm(x_gpu - x_ref, axis=0) / np.linalg.norm(x_ref, axis=0)
    assert rel.max() <= tol, f"relative L2 error {rel.max():.3e} > {tol}"
    el = np.abs(x_gpu - x_ref).max() / np.abs(x_ref).max()
    assert el <= 10 * tol, f"element error {el:.3e} > {10 * tol}"


_fp32_drift = fp32_drift
_close32_conditioned = close32_conditioned


class Handle:
    def __init__(self, J, h=None, instances=None, flags=0):
        self.p = N.Problem(J, h, instances)
        self.h = N.ising_create(self.p, flags)

    def __enter__(self):
        return self.h

    def __exit__(self, *a):
        N.ising_destroy(self.h)


# ---------------------------------------------------------------------------
# 2-D torus (stencil) path
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(37, 1028), (16, 2048), (5, 8), (2, 4), (9, 4)])
@pytest.mark.parametrize("iters", [1, 7, 60])
def test_torus_fp32_r1(shape, iters):
    t = I.torus_pm1(*shape, seed=101)
    x0 = I.x0_uniform(t.n, 1, seed=102)
    alpha, beta = O.alpha_beta(t, eta=1.0, method="wigner")
    ref = O.doch(O.Problem(t), x0, alpha, beta, iters)
    with Handle(t) as h:
        x = _dev(x0)
        N.ising_iterate(h, x, [alpha], [beta], iters)
        _close(x.cpu().numpy(), ref, TOL32)


@pytest.mark.parametrize("shape, R, dtype", [((13, 11), 3, np.float32), ((6, 10), 4, np.float64),
                                             ((7, 9), 1, np.float64), ((3, 6), 1, np.float32)])
def test_torus_generic(shape, R, dtype):
    t = I.torus_pm1(*shape, seed=103)
    x0 = I.x0_uniform(t.n, R, seed=104, dtype=dtype)
    alpha, beta = O.alpha_beta(t, eta=1.0, method="eig")
    ref = O.doch(O.Problem(t), x0, alpha, beta, 25)
    with Handle(t) as h:
        x = _dev(x0)
        N.ising_iterate(h, x, [alpha], [beta], 25)
        _close(x.cpu().numpy(), ref, TOL32 if dtype == np.float32 else TOL64)


@pytest.mark.parametrize("shape", [(37, 1028), (16, 2048), (9, 4), (5, 8), (64, 1024), (100, 3000),
                                   (4, 120), (7, 124), (300, 968), (6, 16), (8, 16)])
@pytest.mark.parametrize("iters", [2, 3, 4, 8, 41])
def test_torus_fused_passes_match_single_steps(shape, iters, monkeypatch):
    """The two- and three-step passes compute every site with the single-step arithmetic:
    bit-identical iterates for at most 2 and 3 steps per pass (remainders of one and two
    steps included) and an alpha schedule; lattices with fewer than 6 rows take pairs."""
    t = I.torus_pm1(*shape, seed=107)
    x0 = I.x0_uniform(t.n, 1, seed=108)
    alpha, beta = O.alpha_beta(t, eta=1.0, method="wigner")
    sched = alpha * (1.0 + 0.05 * np.sin(np.arange(iters)))
    out = []
    for flags, per_pass in ((0, "3"), (0, "2"), (N.FLAG_SINGLE_STEP, "3")):
        monkeypatch.setenv("ISING_LATTICE_PASS", per_pass)
        with Handle(t, flags=flags) as h:
            x = _dev(x0)
            N.ising_iterate(h, x, sched, [beta], iters)
            out.append(x.cpu().numpy())
    assert np.array_equal(out[0], out[2]) and np.array_equal(out[1], out[2])


def test_torus_host_buffers_match_device():
    t = I.torus_pm1(20, 64, seed=105)
    x0 = I.x0_uniform(t.n, 1, seed=106)
    alpha, beta = O.alpha_beta(t, method="wigner")
    with Handle(t) as h:
        xd = _dev(x0)
        N.ising_iterate(h, xd, [alpha], [beta], 9)
        xh = x0.copy()
        N.ising_iterate(h, xh, [alpha], [beta], 9)
        assert np.array_equal(xh, xd.cpu().numpy())


# ---------------------------------------------------------------------------
# CSR path
# ---------------------------------------------------------------------------

def test_csr_fp64_er800_plain_method():
    """Erdos-Renyi n = 800, p = 0.06, +-1, FP64, R = 8, 1000 iterations."""
    g = I.erdos_renyi_pm1(800, 0.06, seed=1)
    x0 = I.x0_uniform(g.n, 8, seed=2, dtype=np.float64)
    alpha, beta = O.alpha_beta(g, eta=1.0, method="eig")
    ref = O.doch(O.Problem(g), x0, alpha, beta, 1000)
    with Handle(g) as h:
        x = _dev(x0)
        N.ising_iterate(h, x, [alpha], [beta], 1000)
        _close(x.cpu().numpy(), ref, TOL64)
        E = torch.zeros(8, dtype=torch.int64, device="cuda")
        cut = torch.zeros(8, dtype=torch.int64, device="cuda")
        best = torch.zeros(1, dtype=torch.int32, device="cuda")
        N.ising_energy(h, x, E_int=E, cut_int=cut, best=best)
        s_ref = O.sign(ref)
        s_gpu = O.sign(x.cpu().numpy())
        # FP64 iterates within 1e-10 of the oracle's: the final spins are the oracle's
        assert np.array_equal(s_ref, s_gpu), f"{int((s_ref != s_gpu).sum())} spins differ"
        Er, cr = O.energy_int(O.Problem(g), s_ref)
        assert np.array_equal(E.cpu().numpy(), Er)
        assert np.array_equal(cut.cpu().numpy(), cr)
        assert best.item() == int(np.argmin(Er))


@pytest.mark.parametrize("R", [64, 6, 1])
def test_csr_fp32_regular(R):
    g = I.regular_pm1(3000, 3, seed=3)
    x0 = I.x0_uniform(g.n, R, seed=4)
    alpha, beta = O.alpha_beta(g, eta=1.0, method="eig")
    ref, drift = _fp32_drift(O.Problem(g), x0, alpha, beta, 30)
    with Handle(g) as h:
        x = _dev(x0)
        N.ising_iterate(h, x, [alpha], [beta], 30)
        _close32_conditioned(x.cpu().numpy(), ref, drift)


def test_csr_fp32_large_uses_step_kernel():
    """An instance too large for shared memory runs one launch per step."""
    g = I.regular_pm1(70000, 3, seed=5)
    x0 = I.x0_uniform(g.n, 4, seed=6)
    alpha, beta = O.alpha_beta(g, eta=1.0, method="wigner")
    ref, drift = _fp32_drift(O.Problem(g), x0, alpha, beta, 12)
    with Handle(g) as h:
        x = _dev(x0)
        N.ising_iterate(h, x, [alpha], [beta], 12)
        _close32_conditioned(x.cpu().numpy(), ref, drift)


@pytest.mark.parametrize("R,dtype", [(64, np.float32), (6, np.float32), (1, np.float32), (2, np.float64),
                                     (3, np.float64)])
def test_csr_short_rows_pipelined_step(R, dtype):
    """The CSR step for short rows (loads pipelined across a thread's rows, one resident wave)
    on 40,010 spins, too many for shared memory: empty rows, hub rows longer than the first
    batch and a hub as the last row. Its iterates are bit-identical to the row-at-a-time step
    kernel's (the kernel a traced run uses, same sums in the same order) and match the oracle."""
    g = short_rows_mixed(40010, seed=71)
    deg = np.diff(g.row_ptr)
    assert deg.min() == 0 and deg.max() > 4 and deg[-1] > 4 and g.nnz <= 8 * g.n
    x0 = I.x0_uniform(g.n, R, seed=72, dtype=dtype)
    alpha, beta = O.alpha_beta(g, eta=1.0, method="wigner")
    iters = 10
    with Handle(g) as h:
        x = _dev(x0)
        N.ising_iterate(h, x, [alpha], [beta], iters)
        plain = x.cpu().numpy()
        x = _dev(x0)
        H = np.zeros((iters + 1, 1, R))
        N.ising_iterate(h, x, [alpha], [beta], iters, H_trace=H)
        traced = x.cpu().numpy()
    assert np.array_equal(plain, traced)
    if dtype == np.float64:
        _close(plain, O.doch(O.Problem(g), x0, alpha, beta, iters), TOL64)
    else:
        ref, drift = _fp32_drift(O.Problem(g), x0, alpha, beta, iters)
        _close32_conditioned(plain, ref, drift)


def test_csr_alpha_schedule():
    g = I.regular_pm1(500, 4, seed=7)
    x0 = I.x0_uniform(g.n, 8, seed=8)
    a0, beta = O.alpha_beta(g, eta=1.0, method="eig")
    sched = a0 * (1.0 + 0.3 * np.sin(np.arange(40) / 5.0))
    ref, drift = _fp32_drift(O.Problem(g), x0, sched, beta, 40)
    with Handle(g) as h:
        x = _dev(x0)
        N.ising_iterate(h, x, sched, [beta], 40)
        _close32_conditioned(x.cpu().numpy(), ref, drift)


def _batch(sizes, degrees, seed, with_h=True):
    gs = [I.regular_gauss(int(n), int(d), seed=seed + b) for b, (n, d) in enumerate(zip(sizes, degrees))]
    hs = [I.field_gauss(g.n, 0.1, seed=seed + 1000 + b) for b, g in enumerate(gs)]
    off = np.cumsum([0] + [g.n for g in gs]).astype(np.int64)
    nz = np.cumsum([0] + [g.nnz for g in gs])
    rp = np.concatenate([[0]] + [g.row_ptr[1:] + z for g, z in zip(gs, nz[:-1])])
    col = np.concatenate([g.col + o for g, o in zip(gs, off[:-1])]).astype(np.int32)
    val = np.concatenate([g.val for g in gs])
    h = np.concatenate(hs) if with_h else None
    return gs, hs, I.CSR(off[-1], rp, col, val), h, off


@pytest.mark.parametrize("xdtype, jdtype", [(np.float32, np.float32), (np.float64, np.float64)])
def test_csr_batched_uneven_with_field(xdtype, jdtype):
    sizes, degrees = [500, 1733, 64, 900], [3, 10, 5, 8]
    gs, hs, J, h, off = _batch(sizes, degrees, seed=20)
    J.val = J.val.astype(jdtype)
    h = h.astype(jdtype)
    R = 16
    x0 = I.x0_uniform(int(off[-1]), R, seed=21, dtype=xdtype)
    alphas, betas = zip(*[O.alpha_beta(g, eta=1.0, method="eig") for g in gs])
    iters = 40
    with Handle(J, h, off) as hd:
        x = _dev(x0)
        N.ising_iterate(hd, x, list(alphas), list(betas), iters, n_instances=len(gs))
        xg = x.cpu().numpy()
    for b, g in enumerate(gs):
        ref = O.doch(O.Problem(g, hs[b].astype(jdtype)), x0[off[b]:off[b + 1]], alphas[b], betas[b], iters)
        _close(xg[off[b]:off[b + 1]], ref, TOL32 if xdtype == np.float32 else TOL64)


@pytest.mark.parametrize("R", [16, 6])
def test_csr_batched_resident_group_widths(R):
    """Instance sizes that take every replica-group width of the shared-memory
    resident kernel (R = 16: G = 16, 8, 4, 2, 1; R = 6: G = 2, 1)."""
    sizes, degrees = [400, 3000, 6000, 12000, 20000], [4, 9, 3, 10, 6]
    gs, hs, J, h, off = _batch(sizes, degrees, seed=60)
    J.val = J.val.astype(np.float32)
    h = h.astype(np.float32)
    x0 = I.x0_uniform(int(off[-1]), R, seed=61)
    alphas, betas = zip(*[O.alpha_beta(g, eta=1.0, method="wigner") for g in gs])
    iters = 12
    with Handle(J, h, off) as hd:
        x = _dev(x0)
        N.ising_iterate(hd, x, list(alphas), list(betas), iters, n_instances=len(gs))
        xg = x.cpu().numpy()
    for b, g in enumerate(gs):
        ref = O.doch(O.Problem(g, hs[b].astype(np.float32)), x0[off[b]:off[b + 1]], alphas[b], betas[b], iters)
        _close(xg[off[b]:off[b + 1]], ref, TOL32)


def test_csr_batched_large_instance_global_kernel():
    """An instance whose two iterate copies exceed shared memory (n = 30000) runs
    the global-memory persistent kernel, in the same call as a small one."""
    sizes, degrees = [30000, 700], [3, 5]
    gs, hs, J, h, off = _batch(sizes, degrees, seed=62)
    J.val = J.val.astype(np.float32)
    h = h.astype(np.float32)
    R = 4
    x0 = I.x0_uniform(int(off[-1]), R, seed=63)
    alphas, betas = zip(*[O.alpha_beta(g, eta=1.0, method="wigner") for g in gs])
    iters = 15
    with Handle(J, h, off) as hd:
        x = _dev(x0)
        N.ising_iterate(hd, x, list(alphas), list(betas), iters, n_instances=len(gs))
        xg = x.cpu().numpy()
    for b, g in enumerate(gs):
        ref = O.doch(O.Problem(g, hs[b].astype(np.float32)), x0[off[b]:off[b + 1]], alphas[b], betas[b], iters)
        _close(xg[off[b]:off[b + 1]], ref, TOL32)


# ---------------------------------------------------------------------------
# energies and cuts of given (seeded) spin vectors
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["torus", "torus_vec", "er"])
def test_energy_integer_exact(kind):
    if kind == "torus":
        J = I.torus_pm1(33, 17, seed=30)
    elif kind == "torus_vec":
        J = I.torus_pm1(64, 1024, seed=31)
    else:
        J = I.erdos_renyi_pm1(800, 0.06, seed=32)
    n = J.n
    R = 5
    x = I.x0_uniform(n, R, seed=33)      # seeded reals: the sign is taken on both sides
    x[::97] = 0.0                        # exact zeros: sign(0) = +1
    s = O.sign(x.astype(np.float64))
    Er, cr = O.energy_int(O.Problem(J), s)
    with Handle(J) as h:
        for xin in (_dev(x), _dev(s), x):  # F32 device, I8 spins, F32 host
            E = np.zeros(R, np.int64)
            cut = np.zeros(R, np.int64)
            best = np.zeros(1, np.int32)
            sp = np.zeros((n, R), np.int8)
            N.ising_energy(h, xin, E_int=E, cut_int=cut, best=best, spins=sp)
            assert np.array_equal(E, Er)
            assert np.array_equal(cut, cr)
            assert best[0] == int(np.argmin(Er))
            assert np.array_equal(sp, s)


def test_energy_f64_batched_gaussian():
    sizes, degrees = [700, 1200, 300], [3, 9, 6]
    gs, hs, J, h, off = _batch(sizes, degrees, seed=40)
    R = 16
    x = I.x0_uniform(int(off[-1]), R, seed=41)
    with Handle(J, h, off) as hd:
        E1 = np.zeros((3, R))
        c1 = np.zeros((3, R))
        best = np.zeros(3, np.int32)
        N.ising_energy(hd, _dev(x), E_f64=E1, cut_f64=c1, best=best)
        E2 = np.zeros((3, R))
        N.ising_energy(hd, _dev(x), E_f64=E2)
        assert np.array_equal(E1, E2)     # fixed reduction order: identical run to run
        with pytest.raises(N.IsingError):  # no exact energy for real couplings
            N.ising_energy(hd, _dev(x), E_int=np.zeros((3, R), np.int64))
    for b, g in enumerate(gs):
        s = O.sign(x[off[b]:off[b + 1]].astype(np.float64))
        Er, cr = O.energy(O.Problem(g, hs[b]), s)
        np.testing.assert_allclose(E1[b], Er, rtol=1e-12)
        np.testing.assert_allclose(c1[b], cr, rtol=1e-12, atol=1e-9)
        assert best[b] == int(np.argmin(Er))


# ---------------------------------------------------------------------------
# FP64 Hamiltonian monitor
# ---------------------------------------------------------------------------

def test_hamiltonian_trace_fp64():
    g = I.erdos_renyi_pm1(200, 0.1, seed=50)
    h = np.round(2 * I.field_gauss(200, 0.1, seed=51)).astype(np.int8)
    alpha, beta = O.alpha_beta(g, eta=1.1, method="eig")
    beta /= 200 ** 1.5
    x0 = I.x0_uniform(g.n, 4, seed=52, dtype=np.float64)
    ref, Href = O.doch(O.Problem(g, h), x0, alpha, beta, 15, trace=True)
    with Handle(g, h, flags=N.FLAG_STRICT_MONOTONE) as hd:
        x = _dev(x0)
        H = np.zeros((16, 1, 4))
        N.ising_iterate(hd, x, [alpha], [beta], 15, H_trace=H)
        _close(x.cpu().numpy(), ref, TOL64)
        np.testing.assert_allclose(H[:, 0, :], Href, rtol=1e-10, atol=1e-12 * np.abs(Href).max())


def test_hamiltonian_trace_torus_fp32_monotone():
    t = I.torus_pm1(32, 64, seed=53)
    alpha, beta = O.alpha_beta(t, eta=1.05, method="eig")
    x0 = I.x0_uniform(t.n, 1, seed=54)
    with Handle(t) as hd:
        x = _dev(x0)
        H = torch.zeros((21, 1, 1), dtype=torch.float64, device="cuda")
        N.ising_iterate(hd, x, [alpha], [beta], 20, H_trace=H)
        Hh = H.cpu().numpy().ravel()
    _, Href = O.doch(O.Problem(t), x0, alpha, beta, 20, trace=True)
    np.testing.assert_allclose(Hh, Href.ravel(), rtol=1e-4)
    assert np.all(np.diff(Hh) <= 1e-6 * np.abs(Hh).max())


# ---------------------------------------------------------------------------
# argument errors reach the caller as statuses
# ---------------------------------------------------------------------------

def test_iterate_argument_errors():
    t = I.torus_pm1(8, 8, seed=60)
    with Handle(t) as h:
        x = _dev(I.x0_uniform(t.n, 1, seed=61))
        with pytest.raises(N.IsingError) as e:
            N.ising_iterate(h, x, [1.0], [0.0], 3)
        assert e.value.name == "ISING_ERR_INVALID_ARG"
        with pytest.raises(N.IsingError) as e:
            N.ising_iterate(h, x, [np.inf], [1.0], 3)
        assert e.value.name == "ISING_ERR_NONFINITE"
        with pytest.raises(N.IsingError):
            N.ising_iterate(h, x, [1.0, 2.0], [1.0], 3)   # alpha_len neither 1 nor iters


# ---------------------------------------------------------------------------
# device cube root of the stencil kernel against CUDA's cbrtf
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("k", [0, 21, -7])
def test_stencil_cube_root_accuracy(k):
    """Relative error of the stencil's cube root against cbrtf over prescaled
    arguments z' = z 2^(-3k) in [2^-60, 2^60]; odd; cbrt(0) = 0.

    Bound derived from the arithmetic: the FP32 value l = log2|z'| carries an
    absolute rounding of |l| 2^-24, which exp2(l / 3) turns into a relative
    error of (ln 2 / 3) |l| 2^-24 < 0.25 |l| 2^-24; the hardware log2/exp2
    approximations and the final products add about 2^-21. In the iteration
    |l| stays small (z' ~ 1 at the attractor scale)."""
    u = I.uniform01(I.stream_seed(9, k + 50), 0, 1 << 20)
    e = -60.0 + 120.0 * u                              # log2 of the prescaled magnitude
    sg = I.signs(I.stream_seed(9, k + 51), 0, 1 << 20)
    z = (sg * np.exp2(e + 3 * k)).astype(np.float32)
    z = np.concatenate([z, -z[:1000], np.zeros(4, np.float32)])
    zd = _dev(z)
    ours = torch.empty_like(zd)
    ref = torch.empty_like(zd)
    st = N.load().ising_selftest_cbrt(N._ptr(zd), N._ptr(ours), N._ptr(ref), z.size, k, None)
    assert st == 0
    o, r = ours.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
    nz = r != 0
    rel = np.abs(o[nz] - r[nz]) / np.abs(r[nz])
    lz = np.abs(np.log2(np.abs(z[nz].astype(np.float64))) - 3 * k)
    bound = 2.0 ** -21 + 0.25 * lz * 2.0 ** -24
    assert np.all(rel <= bound), (rel / bound).max()
    assert np.array_equal(np.sign(o), np.sign(r))
    assert np.all(o[-4:] == 0.0)


@pytest.mark.parametrize("c3", [-7.3, -1.1, 0.0, 0.5, 3.7])
def test_lattice_cube_root_accuracy(c3):
    """Relative error of the lattice kernels' cube root sign(z) 2^(log2|z|/3 + c3) (cbrt_log)
    against the FP64 value cbrt(z) 2^c3, for |z| in [2^-60, 2^60]; odd; 0 -> 0.

    Bound derived from the arithmetic: the FP32 value L = log2|z| carries an absolute rounding
    of |L| 2^-24, and l = L/3 + c3 (one FMA) one of |l| 2^-24; exp2 turns an absolute error e
    of l into a relative error of ln 2 e, so the two give at most (ln 2 / 3 |L| + ln 2 |l|) 2^-24
    < (0.25 |L| + 0.75 |l|) 2^-24; the hardware log2/exp2 approximations add about 2^-21."""
    u = I.uniform01(I.stream_seed(19, int(10 * c3) + 100), 0, 1 << 20)
    e = -60.0 + 120.0 * u
    sg = I.signs(I.stream_seed(19, int(10 * c3) + 200), 0, 1 << 20)
    z = (sg * np.exp2(e)).astype(np.float32)
    z = np.concatenate([z, -z[:1000], np.zeros(4, np.float32)])
    zd = _dev(z)
    out = torch.empty_like(zd)
    st = N.load().ising_selftest_cbrt_log(N._ptr(zd), N._ptr(out), z.size, float(np.float32(c3)), None)
    assert st == 0
    o = out.cpu().numpy().astype(np.float64)
    z64 = z.astype(np.float64)
    c3f = float(np.float32(c3))
    ref = np.cbrt(z64) * 2.0 ** c3f
    nz = z64 != 0
    rel = np.abs(o[nz] - ref[nz]) / np.abs(ref[nz])
    L = np.log2(np.abs(z64[nz]))
    l = L / 3.0 + c3f
    bound = 2.0 ** -21 + (0.25 * np.abs(L) + 0.75 * np.abs(l)) * 2.0 ** -24
    assert np.all(rel <= bound), (rel / bound).max()
    assert np.array_equal(np.sign(o), np.sign(z64))
    assert np.all(o[-4:] == 0.0)


def test_ell_input_runs_as_csr():
    """ELL rows (empty slots -1) create the CSR problem: the iterates of the two handles agree
    bit for bit (FP32 and FP64)."""
    g = I.regular_gauss(500, 6, seed=621)
    w = 9
    col = np.full((g.n, w), -1, np.int32)
    val = np.zeros((g.n, w), np.asarray(g.val).dtype)
    for i in range(g.n):
        e0, e1 = g.row_ptr[i], g.row_ptr[i + 1]
        col[i, w - (e1 - e0):] = g.col[e0:e1]
        val[i, w - (e1 - e0):] = g.val[e0:e1]

    class Ell:
        ell_col, ell_val = col, val

    alpha, beta = O.alpha_beta(g, eta=1.0, method="eig")
    for dtype in (np.float32, np.float64):
        x0 = I.x0_uniform(g.n, 4, seed=622, dtype=dtype)
        outs = []
        for prob in (N.Problem(g), N.Problem(Ell())):
            hd = N.ising_create(prob)
            try:
                x = torch.from_numpy(x0.copy()).cuda()
                N.ising_iterate(hd, x, [alpha], [beta], 30)
                outs.append(x.cpu().numpy())
            finally:
                N.ising_destroy(hd)
        assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("eps", [0.0, 1e-4])
def test_batched_resident_variants_agree(eps, monkeypatch):
    """Every variant of the shared-memory resident kernel the autotuner chooses from (512 or
    1024 threads; both Jacobi copies in shared memory, or one copy with the new iterate through
    global scratch, which doubles the replicas per item) computes the same arithmetic in the same
    order: bit-identical iterates (and step counts under the stopping rule), and the oracle's
    iterates within the FP32 bar. The second call of ising_iterate replays the captured graph."""
    sizes, degrees = [400, 3000, 6000, 12000, 20000], [4, 9, 3, 10, 6]
    gs, hs, J, h, off = _batch(sizes, degrees, seed=64)
    J.val = J.val.astype(np.float32)
    h = h.astype(np.float32)
    R = 16
    x0 = I.x0_uniform(int(off[-1]), R, seed=65)
    alphas, betas = zip(*[O.alpha_beta(g, eta=1.0, method="wigner") for g in gs])
    iters = 14
    outs = []
    for variant in ("1024:2", "1024:1", "512:2", "512:1"):
        monkeypatch.setenv("ISING_RESIDENT_VARIANT", variant)
        with Handle(J, h, off) as hd:
            x = _dev(x0)
            if eps > 0:
                steps = np.zeros((len(gs), R), np.int32)
                N.ising_iterate_until(hd, x, list(alphas), list(betas), iters, eps, steps=steps)
                outs.append((x.cpu().numpy(), steps))
            else:
                N.ising_iterate(hd, x, list(alphas), list(betas), iters, n_instances=len(gs))
                x2 = _dev(x0)
                N.ising_iterate(hd, x2, list(alphas), list(betas), iters, n_instances=len(gs))  # graph replay
                assert np.array_equal(x.cpu().numpy(), x2.cpu().numpy())
                outs.append((x.cpu().numpy(), None))
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0])
        if eps > 0:
            assert np.array_equal(o[1], outs[0][1])
    if eps == 0:
        xg = outs[0][0]
        for b, g in enumerate(gs):
            ref = O.doch(O.Problem(g, hs[b].astype(np.float32)), x0[off[b]:off[b + 1]], alphas[b], betas[b], iters)
            _close(xg[off[b]:off[b + 1]], ref, TOL32)


@pytest.mark.parametrize("kind", ["csr_step", "lattice"])
def test_fused_hamiltonian_monitor(kind):
    """The H monitor fused into the step kernel (the default for a trace) against the exact
    separate FP64 reduction (taken for FP32 iterates under ISING_FLAG_STRICT_MONOTONE) on the
    same iterates: the fused form sums FP32 terms with compensated FP32 sums per thread, so
    the two traces agree to ~1e-7 of the terms' scale (asserted: 1e-5 of the largest |H|);
    the iterates of a traced run are bit-identical to an untraced run's, and both traces
    match the oracle's H of the same starting point to the FP32 bar."""
    if kind == "csr_step":
        J = I.regular_pm1(70000, 3, seed=66)        # too large for shared memory: the step kernel
        R, method = 8, "wigner"
    else:
        J = I.torus_pm1(96, 512, seed=67)
        R, method = 1, "wigner"
    alpha, beta = O.alpha_beta(J, eta=1.0, method=method)
    x0 = I.x0_uniform(J.n, R, seed=68)
    iters = 12
    traces, outs = [], []
    for flags in (0, N.FLAG_STRICT_MONOTONE):
        with Handle(J, flags=flags) as h:
            x = _dev(x0)
            H = np.zeros((iters + 1, 1, R))
            N.ising_iterate(h, x, [alpha], [beta], iters, H_trace=H)
            traces.append(H[:, 0, :])
            outs.append(x.cpu().numpy())
    with Handle(J) as h:
        x = _dev(x0)
        N.ising_iterate(h, x, [alpha], [beta], iters)
        plain = x.cpu().numpy()
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], plain)
    fused, exact = traces
    assert np.all(np.abs(fused - exact) <= 1e-5 * np.abs(exact).max()), np.abs(fused - exact).max()
    _, Href = O.doch(O.Problem(J), x0, alpha, beta, 1, trace=True)
    np.testing.assert_allclose(fused[0], Href[0], rtol=1e-5)
