"""The lattice path at the benchmark's own shape: a 10^4 x 10^4 periodic
lattice with +-1 couplings (seed 2, x0 seed 2, Wigner parameters, eta = 1),
FP32, R = 1 -- the configuration bench.py times.

At this width the multi-step passes run 84 column segments with row strips of
hundreds of rows, so their shared-memory row rings wrap many times per strip;
the smaller lattices of test_gpu_doch.py never reach that regime. Checks:

  * the fused passes are bit-identical to single steps at 2, 3, 4 and 5
    iterations (one pair; one triple; a triple and a single step; a triple
    and a pair), on the full lattice;
  * one step against the oracle, element by element in z-space: the cube of
    the device's x^(1) must equal z = (J x + alpha x)/beta of the oracle
    within 40 * 2^-24 of the step's own scale (sum_j |J_ij x_j| + alpha |x_i|)
    / beta -- an FP32 sum of five terms and a product (8 units) plus three times
    the cube root's relative error of 2^-21 (25.6 units). A wrong neighbour or a
    missed seam moves z by O(scale); cancellation, which makes x-space element
    errors large where z is near zero, does not matter there;
  * 2 and 3 steps against the oracle on the full lattice: relative vector
    error <= 1e-5;
  * 500 steps (the timed count) on sampled 16 x 16 blocks: x^(500) of a site
    depends only on sites within 500 lattice steps, so the oracle runs on the
    open-boundary patch that extends each block by 500 sites in every
    direction (1016 x 1016 sites; the couplings of the patch are the
    lattice's own); relative vector error per block <= 1e-5 and every element
    within 1e-4 of the block's largest value. One block straddles the lattice's
    wrap in both directions, one a column-segment boundary of the kernel.
"""
import numpy as np
import pytest

import oracle as O
from paper_2509_01928_gb300 import _native as N
from paper_2509_01928_gb300 import build as B
from paper_2509_01928_gb300 import inputs as I
from oracle.lattice import light_cone_patch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

L = 10_000
TOL32 = 1e-5


@pytest.fixture(scope="module")
def lattice():
    assert torch.cuda.is_available()
    B.build_library()
    t = I.torus_pm1(L, L, seed=2)
    x0 = I.x0_uniform(t.n, 1, seed=2)
    alpha, beta = O.alpha_beta(t, eta=1.0, method="wigner")
    return t, x0, alpha, beta


def _run(t, x0, alpha, beta, iters, flags=0):
    h = N.ising_create(N.Problem(t), flags)
    try:
        x = torch.from_numpy(x0.copy()).cuda()
        N.ising_iterate(h, x, [alpha], [beta], iters)
        return x.cpu().numpy()
    finally:
        N.ising_destroy(h)


@pytest.mark.parametrize("iters", [2, 3, 4, 5])
def test_full_lattice_fused_equals_single_steps(lattice, iters):
    t, x0, alpha, beta = lattice
    assert np.array_equal(_run(t, x0, alpha, beta, iters), _run(t, x0, alpha, beta, iters, N.FLAG_SINGLE_STEP))


@pytest.mark.parametrize("iters", [3, 5])
def test_full_lattice_three_step_pass_equals_single_steps(lattice, iters, monkeypatch):
    """The opt-in three-step pass (ISING_LATTICE_PASS=3) on the full lattice: a triple, and a
    triple followed by a pair, bit-identical to single steps."""
    t, x0, alpha, beta = lattice
    monkeypatch.setenv("ISING_LATTICE_PASS", "3")
    assert np.array_equal(_run(t, x0, alpha, beta, iters), _run(t, x0, alpha, beta, iters, N.FLAG_SINGLE_STEP))


def test_full_lattice_one_step_elementwise(lattice):
    t, x0, alpha, beta = lattice
    x1 = _run(t, x0, alpha, beta, 1).astype(np.float64).ravel()
    xd = x0.astype(np.float64)
    z = (O.coupling_product(O.Problem(t), xd) + alpha * xd).ravel() / beta
    ones = I.Torus2D(np.ones_like(t.right), np.ones_like(t.down))       # |J| of +-1 couplings
    scale = (O.coupling_product(O.Problem(ones), np.abs(xd)) + alpha * np.abs(xd)).ravel() / beta
    err = np.abs(x1 ** 3 - z)
    bound = 40.0 * 2.0 ** -24 * scale
    worst = int(np.argmax(err / bound))
    assert np.all(err <= bound), f"site {worst}: {err[worst]:.3e} > {bound[worst]:.3e}"


@pytest.mark.parametrize("iters", [2, 3])
def test_full_lattice_against_oracle(lattice, iters):
    t, x0, alpha, beta = lattice
    got = _run(t, x0, alpha, beta, iters).astype(np.float64)
    ref = O.doch(O.Problem(t), x0, alpha, beta, iters)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= TOL32, rel


def test_full_lattice_500_steps_on_light_cone_blocks(lattice):
    t, x0, alpha, beta = lattice
    iters, size = 500, 16
    got = _run(t, x0, alpha, beta, iters).ravel()
    for r0, c0 in [(L - 8, L - 8), (4321, 7 * 120 - 8)]:
        J, G = light_cone_patch(t, r0, c0, size, iters)
        P = size + 2 * iters
        ref = O.doch(O.Problem(J), x0.ravel()[G].astype(np.float64), alpha, beta, iters).reshape(P, P)
        blk = ref[iters:iters + size, iters:iters + size].ravel()
        gblk = got[G.reshape(P, P)[iters:iters + size, iters:iters + size].ravel()].astype(np.float64)
        rel = np.linalg.norm(gblk - blk) / np.linalg.norm(blk)
        el = np.abs(gblk - blk).max() / np.abs(blk).max()
        assert rel <= TOL32 and el <= 10 * TOL32, (r0, c0, rel, el)
