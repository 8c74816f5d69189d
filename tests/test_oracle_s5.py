"""Algorithm S5 (Supplementary Note 9) reference generator (oracle/matrices.py): the
vectorised generator against a literal pair-by-pair loop in Python integers,
the exact threshold form of the test z < 1023, and the distribution the
algorithm implies (density 1022 / N_p, values uniform on -510 .. 511)."""
import numpy as np

from oracle import matrices as M
from paper_2509_01928_gb300 import inputs as I


def _literal(n, p, seed):
    n_p = int(np.floor(102300.0 / p))
    sd = int(I.stream_seed(seed, I.TAG_S5))
    gamma, m1, m2, mask = 0x9E3779B97F4A7C15, 0xBF58476D1CE4E5B9, 0x94D049BB133111EB, (1 << 64) - 1

    def mix(z):
        z = ((z ^ (z >> 30)) * m1) & mask
        z = ((z ^ (z >> 27)) * m2) & mask
        return z ^ (z >> 31)

    d = np.zeros((n, n), dtype=np.int64)
    present = np.zeros((n, n), dtype=bool)
    t = 0
    for i in range(1, n):          # the algorithm's loops, 0-based: j < i
        for j in range(i):
            u = mix((sd + (t + 1) * gamma) & mask)
            z = 1 + (u * n_p >> 64)
            if z < 1023:
                d[i, j] = d[j, i] = z - 511
                present[i, j] = present[j, i] = True
            t += 1
    return d, present


def test_s5_matches_literal_loop():
    for n, p, seed in ((40, 30.0, 11), (64, 100.0, 3), (90, 7.5, 5)):
        J = M.s5_csr(n, p, seed)
        d, present = _literal(n, p, seed)
        got = np.zeros((n, n), dtype=bool)
        rows = np.repeat(np.arange(n), np.diff(J.row_ptr))
        got[rows, J.col] = True
        assert np.array_equal(got, present)               # explicit zeros included
        assert np.array_equal(J.to_dense(), d)
        assert np.all(np.diff(J.col[J.row_ptr[0]:J.row_ptr[1]]) > 0)


def test_s5_n_p_is_the_rounded_quotient():
    """N_p of p = 0.05 is 2046000 (102300 / 0.05 in decimal): the rounded double
    quotient, whose floor Python's float floor division would put at 2045999."""
    assert M.s5_params(0.05)[0] == 2046000
    assert M.s5_params(100.0)[0] == 1023 and M.s5_params(0.5)[0] == 204600


def test_s5_threshold_is_exact():
    rng = np.random.default_rng(0)
    for p in (100.0, 50.0, 3.3, 0.01, 1e-6):
        n_p, thr = M.s5_params(p)
        us = [int(v) for v in rng.integers(0, 2**63, 2000, dtype=np.int64)] + [thr - 1, thr, thr + 1, 0, 2**64 - 1]
        for u in us:
            u %= 1 << 64
            assert (u < thr) == (1 + (u * n_p >> 64) < 1023)
        assert int(M._mulhi64(np.array([thr - 1], np.uint64), n_p)[0]) == ((thr - 1) * n_p) >> 64


def test_s5_distribution():
    n, p = 3000, 2.0
    J = M.s5_csr(n, p, seed=21)
    n_p, _ = M.s5_params(p)
    pairs = n * (n - 1) // 2
    kept = J.nnz // 2
    mean = pairs * 1022 / n_p
    sd = np.sqrt(pairs * (1022 / n_p) * (1 - 1022 / n_p))
    assert abs(kept - mean) < 5 * sd
    upper = J.val[np.repeat(np.arange(n), np.diff(J.row_ptr)) < J.col].astype(np.int64)
    counts = np.bincount(upper + 510, minlength=1022)
    assert counts.size == 1022 and upper.min() >= -510 and upper.max() <= 511
    exp = kept / 1022.0
    chi2 = np.sum((counts - exp) ** 2 / exp)
    assert chi2 < 1021 + 6 * np.sqrt(2 * 1021)           # chi-square, 1021 dof, ~6 sigma
    d = J.to_dense()
    assert np.array_equal(d, d.T) and np.all(np.diag(d) == 0)
