"""Pins of the oracle's rows of the procedural product (Supplementary Note 9,
J_ij = sin(i j + c), 1-based, J_ii = 0) against facts fixed by mathematics."""
import numpy as np

import oracle as O
from oracle import matrices as M
from paper_2509_01928_gb300 import inputs as I


def test_rows_of_all_ones_are_the_geometric_series():
    # sum_{j=1..n} sin(c + j i) = sin(c + (n+1) i / 2) sin(n i / 2) / sin(i / 2)
    n, c = 5000, 100
    rows = [0, 1, 354, 709, 2047, n - 1]  # i = 710 has sin(i/2) ~ 3e-5
    u = O.procedural_rows(n, c, rows, np.ones((n, 1)))[:, 0]
    for k, r in enumerate(rows):
        i = r + 1
        closed = np.sin(c + (n + 1) * i / 2) * np.sin(n * i / 2) / np.sin(i / 2) - np.sin(i * i + c)
        assert abs(u[k] - closed) <= 1e-9 * max(1.0, abs(closed))


def test_rows_of_unit_vectors_pick_single_couplings():
    n, c = 300, 7
    x = np.zeros((n, 3))
    x[0, 0] = 1.0        # column j = 1
    x[41, 1] = 1.0       # column j = 42
    x[n - 1, 2] = -2.0   # column j = n
    rows = [0, 41, 120, n - 1]
    u = O.procedural_rows(n, c, rows, x)
    for k, r in enumerate(rows):
        i = r + 1
        assert u[k, 0] == (0.0 if i == 1 else np.sin(i * 1 + c))
        assert u[k, 1] == (0.0 if i == 42 else np.sin(i * 42 + c))
        assert u[k, 2] == (0.0 if i == n else -2.0 * np.sin(i * n + c))


def test_rows_agree_with_the_dense_product():
    n, c = 700, 100
    x = I.x0_uniform(n, 4, seed=71, dtype=np.float64)
    full = O.coupling_product(O.Problem(M.procedural_sin(n, c)), x)
    rows = [0, 5, 255, 256, 511, n - 1]
    np.testing.assert_allclose(O.procedural_rows(n, c, rows, x), full[rows], rtol=0, atol=1e-12)
