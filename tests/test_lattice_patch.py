"""The light-cone patch helper against the full periodic lattice (CPU, oracle
on both sides): x^(N) on a block equals the oracle run on the block's patch
of margin N (to the rounding of the summation order, which differs between
the lattice and CSR forms), including blocks that wrap around the lattice;
with a margin one short of N the block's values change (the construction is
tight)."""
import numpy as np
import pytest

import oracle as O
from paper_2509_01928_gb300 import inputs as I
from oracle.lattice import light_cone_patch


@pytest.mark.parametrize("r0, c0", [(0, 0), (57, 61), (20, 33)])
def test_light_cone_patch_reproduces_the_lattice(r0, c0):
    t = I.torus_pm1(60, 64, seed=41)
    x0 = I.x0_uniform(t.n, 2, seed=42, dtype=np.float64)
    alpha, beta = O.alpha_beta(t, eta=1.0, method="eig")
    N_, size = 9, 5
    full = O.doch(O.Problem(t), x0, alpha, beta, N_)
    J, G = light_cone_patch(t, r0, c0, size, N_)
    P = size + 2 * N_
    ref = O.doch(O.Problem(J), x0[G], alpha, beta, N_).reshape(P, P, 2)
    blk = ref[N_:N_ + size, N_:N_ + size].reshape(-1, 2)
    gidx = G.reshape(P, P)[N_:N_ + size, N_:N_ + size].ravel()
    np.testing.assert_allclose(blk, full[gidx], rtol=1e-12, atol=1e-15)
    J2, G2 = light_cone_patch(t, r0, c0, size, N_ - 1)
    P2 = size + 2 * (N_ - 1)
    short = O.doch(O.Problem(J2), x0[G2], alpha, beta, N_).reshape(P2, P2, 2)
    assert np.abs(short[N_ - 1:N_ - 1 + size, N_ - 1:N_ - 1 + size].reshape(-1, 2) - full[gidx]).max() > 1e-10 * np.abs(full).max()
