"""The seeded input generators against their definitions: SplitMix64 against the published
sequence of its reference implementation (state 0), and the structure of every synthetic
workload (regular graphs, Erdos-Renyi graphs, lattices, starts, fields, batch sizes)."""
import numpy as np

from paper_2509_01928_gb300 import inputs as I


def test_splitmix64_reference_sequence():
    # the first outputs of SplitMix64 from state 0 (Vigna's reference generator)
    v = I.splitmix64(0, 0, 4)
    assert [int(x) for x in v] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F,
                                   0xF88BB8A8724C81EC]
    # counter-based: any window of the stream is the same values
    assert np.array_equal(I.splitmix64(7, 10, 5), I.splitmix64(7, 0, 15)[10:])


def _dense_of(g):
    D = np.zeros((g.n, g.n))
    for i in range(g.n):
        for e in range(g.row_ptr[i], g.row_ptr[i + 1]):
            D[i, g.col[e]] += g.val[e]
    return D


def test_random_regular_is_simple_and_regular():
    for n, d, seed in ((100, 3, 1), (64, 10, 2), (501, 4, 3)):
        g = I.regular_pm1(n, d, seed=seed)
        deg = np.diff(g.row_ptr)
        assert np.all(deg == d)
        for i in range(n):
            cols = g.col[g.row_ptr[i]:g.row_ptr[i + 1]]
            assert i not in cols and len(set(cols.tolist())) == d  # no self-loop, no repeated edge
        D = _dense_of(g)
        assert np.array_equal(D, D.T) and set(np.unique(D)) <= {-1.0, 0.0, 1.0}


def test_erdos_renyi_density_and_symmetry():
    n, p = 800, 0.06
    g = I.erdos_renyi_pm1(n, p, seed=1)
    D = _dense_of(g)
    assert np.array_equal(D, D.T) and np.all(np.diag(D) == 0)
    edges = g.row_ptr[-1] / 2
    expect = p * n * (n - 1) / 2
    assert abs(edges - expect) < 4 * np.sqrt(expect)  # binomial: within 4 standard deviations
    vals = np.asarray(g.val)
    assert set(np.unique(vals)) == {-1, 1} and abs(np.mean(vals)) < 0.05


def test_lattice_starts_fields_and_sizes():
    t = I.torus_pm1(37, 200, seed=4)
    assert t.right.shape == (37, 200) and t.down.shape == (37, 200) and t.right.dtype == np.int8
    assert set(np.unique(t.right)) == {-1, 1} and set(np.unique(t.down)) == {-1, 1}
    x = I.x0_uniform(1000, 8, seed=5)
    assert x.shape == (1000, 8) and x.dtype == np.float32 and x.min() >= -1.0 and x.max() < 1.0
    assert abs(x.mean()) < 0.02 and abs(x.var() - 1.0 / 3.0) < 0.02
    h = I.field_gauss(200000, 0.1, seed=6)
    assert abs(h.mean()) < 0.005 and abs(h.var() - 0.1) < 0.003  # "N(0, 0.1)": variance 0.1
    sizes, degs = I.batched_sizes(512, 500, 20000, 3, 10, seed=7)
    assert len(sizes) == len(degs) == 512
    assert np.all((np.asarray(sizes) >= 500) & (np.asarray(sizes) <= 20001))
    assert np.all((np.asarray(degs) >= 3) & (np.asarray(degs) <= 10))
    assert np.all(np.asarray(sizes) * np.asarray(degs) % 2 == 0)  # a d-regular graph exists
