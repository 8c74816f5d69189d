"""Seeded synthetic inputs for the DOCH Ising solver.

This module only draws random numbers and lays them out as coupling
structures and starting points. It holds none of the method's arithmetic
(no coupling product, no cube root, no energy), so the FP64 oracle and the
CUDA path can both be fed from it without sharing any computation.

Random source: SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used counter-style: value
``t`` of stream ``s`` is ``mix(s + (t + 1) * 0x9E3779B97F4A7C15)`` with the
published ``mix`` finaliser. Uniform doubles are ``(u >> 11) * 2**-53``.

Workload shapes follow the paper's benchmark families (supplementary
Note 8 and Note 9): Erdos-Renyi graphs with +-1 weights (a G-set-G10-like
800-node graph), two-dimensional toroidal lattices, dense +-1 matrices
(K2000-like), random d-regular graphs with Gaussian weights, and uniform
starting points x0 in [-1, 1).
"""
from __future__ import annotations

import collections

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22

# stream tags, so that each purpose gets an independent sub-stream of a seed
TAG_EDGE = 1
TAG_SIGN = 2
TAG_RIGHT = 3
TAG_DOWN = 4
TAG_X0 = 5
TAG_PAIR = 6
TAG_REPAIR = 7
TAG_GAUSS_A = 8
TAG_GAUSS_B = 9
TAG_FIELD_A = 10
TAG_FIELD_B = 11
TAG_SIZE = 12
TAG_S5 = 13


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_seed(seed: int, tag: int) -> np.uint64:
    """Seed of the sub-stream ``tag`` of ``seed`` (one SplitMix64 output)."""
    with np.errstate(over="ignore"):
        s = np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF)], dtype=np.uint64)
        s = _mix(s * _GAMMA + np.uint64(tag) * _M2)
    return s[0]


def splitmix64(seed, start: int, count: int) -> np.ndarray:
    """Values ``start .. start+count-1`` of the counter-based stream ``seed``."""
    s = np.uint64(seed)
    out = np.empty(count, dtype=np.uint64)
    for c0 in range(0, count, _CHUNK):
        c1 = min(count, c0 + _CHUNK)
        t = np.arange(start + c0 + 1, start + c1 + 1, dtype=np.uint64)
        out[c0:c1] = _mix(s + t * _GAMMA)
    return out


def uniform01(seed, start: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    u = splitmix64(seed, start, count)
    return (u >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def signs(seed, start: int, count: int) -> np.ndarray:
    """+1 / -1 (int8) from the top bit of each stream value."""
    u = splitmix64(seed, start, count)
    return np.where((u >> np.uint64(63)) == 1, 1, -1).astype(np.int8)


def gaussian(seed_a, seed_b, start: int, count: int) -> np.ndarray:
    """Standard normal draws by the Box-Muller transform of two streams."""
    u1 = uniform01(seed_a, start, count)
    u2 = uniform01(seed_b, start, count)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


# ---------------------------------------------------------------------------
# coupling structures
# ---------------------------------------------------------------------------

class CSR:
    """Symmetric coupling matrix in CSR form, zero diagonal, columns sorted."""

    def __init__(self, n, row_ptr, col, val):
        self.n = int(n)
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = np.ascontiguousarray(val)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n), dtype=np.float64)
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        d[rows, self.col] = self.val
        return d


def csr_from_upper(n: int, i: np.ndarray, j: np.ndarray, v: np.ndarray) -> CSR:
    """Mirror upper-triangle entries (i < j) into a symmetric CSR matrix."""
    rows = np.concatenate([i, j]).astype(np.int64)
    cols = np.concatenate([j, i]).astype(np.int64)
    vals = np.concatenate([v, v])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return CSR(n, row_ptr, cols.astype(np.int32), vals)


def _upper_pairs(n: int):
    """All pairs i < j in row-major order of the upper triangle."""
    i, j = np.triu_indices(n, k=1)
    return i.astype(np.int64), j.astype(np.int64)


def erdos_renyi_pm1(n: int, p: float, seed: int) -> CSR:
    """Erdos-Renyi graph G(n, p) with couplings uniform in {-1, +1}, int8.

    Pair t of the upper triangle (row-major) is an edge when draw t of the
    edge stream is below p; its sign is draw t of the sign stream.
    """
    i, j = _upper_pairs(n)
    m = i.size
    keep = uniform01(stream_seed(seed, TAG_EDGE), 0, m) < p
    s = signs(stream_seed(seed, TAG_SIGN), 0, m)
    return csr_from_upper(n, i[keep], j[keep], s[keep])


class Torus2D:
    """L_rows x L_cols periodic lattice with nearest-neighbour couplings.

    ``right[r, c]`` couples site (r, c) with (r, (c+1) mod L_cols) and
    ``down[r, c]`` couples (r, c) with ((r+1) mod L_rows, c). Site (r, c)
    is spin index ``r * L_cols + c``.
    """

    def __init__(self, right: np.ndarray, down: np.ndarray):
        assert right.shape == down.shape
        self.right = np.ascontiguousarray(right)
        self.down = np.ascontiguousarray(down)

    @property
    def shape(self):
        return self.right.shape

    @property
    def n(self) -> int:
        return int(self.right.size)

    def to_csr(self) -> CSR:
        lr, lc = self.shape
        r, c = np.meshgrid(np.arange(lr), np.arange(lc), indexing="ij")
        a = (r * lc + c).ravel()
        b_right = (r * lc + (c + 1) % lc).ravel()
        b_down = (((r + 1) % lr) * lc + c).ravel()
        i = np.concatenate([a, a])
        j = np.concatenate([b_right, b_down])
        v = np.concatenate([self.right.ravel(), self.down.ravel()])
        # an edge may be listed twice on tiny lattices (L = 2); merge those
        lo, hi = np.minimum(i, j), np.maximum(i, j)
        key = lo * self.n + hi
        uk, inv = np.unique(key, return_inverse=True)
        acc = np.zeros(uk.size, dtype=np.int64)
        np.add.at(acc, inv, v.astype(np.int64))
        return csr_from_upper(self.n, uk // self.n, uk % self.n, acc.astype(self.right.dtype))


def torus_pm1(l_rows: int, l_cols: int, seed: int) -> Torus2D:
    """Toroidal lattice with +-1 couplings stored as int8 per edge."""
    m = l_rows * l_cols
    right = signs(stream_seed(seed, TAG_RIGHT), 0, m).reshape(l_rows, l_cols)
    down = signs(stream_seed(seed, TAG_DOWN), 0, m).reshape(l_rows, l_cols)
    return Torus2D(right, down)


def dense_pm1(n: int, seed: int) -> np.ndarray:
    """Dense symmetric n x n int8 matrix, off-diagonal entries uniform in {-1, +1}.

    Entry (i, j), i < j, is draw t of the sign stream with t the row-major
    index of the pair in the upper triangle; the lower triangle mirrors it.
    """
    out = np.zeros((n, n), dtype=np.int8)
    sd = stream_seed(seed, TAG_SIGN)
    t0 = 0
    for i in range(n - 1):
        k = n - 1 - i
        row = signs(sd, t0, k)
        out[i, i + 1:] = row
        t0 += k
    return out + out.T


def random_regular(n: int, d: int, seed: int):
    """Random simple d-regular graph on n vertices as upper-triangle edges.

    Configuration (pairing) model: the n*d stubs are put in the order of
    their stream keys and paired consecutively; self-loops and repeated
    pairs are then removed one at a time by random double-edge switches
    drawn from a second stream, which keeps every degree equal to d.
    Requires n*d even and d < n.
    """
    if (n * d) % 2 or d >= n:
        raise ValueError("need n*d even and d < n")
    stubs = np.repeat(np.arange(n, dtype=np.int64), d)
    keys = splitmix64(stream_seed(seed, TAG_PAIR), 0, stubs.size)
    order = np.argsort(keys, kind="stable")
    e = stubs[order].reshape(-1, 2)
    a = np.minimum(e[:, 0], e[:, 1])
    b = np.maximum(e[:, 0], e[:, 1])
    m = a.size
    key = a * n + b
    counts = collections.Counter(key.tolist())

    def bad(idx):
        return a[idx] == b[idx] or counts[int(a[idx] * n + b[idx])] > 1

    rs = stream_seed(seed, TAG_REPAIR)
    draw = 0
    _, inv, cnt = np.unique(key, return_inverse=True, return_counts=True)
    todo = np.nonzero((a == b) | (cnt[inv] > 1))[0].tolist()
    guard = 0
    while todo:
        t = todo.pop()
        if not bad(t):
            continue
        while True:
            guard += 1
            if guard > 1000 * (m + 10):
                raise RuntimeError("regular-graph repair did not terminate")
            f = int(splitmix64(rs, draw, 1)[0] % np.uint64(m))
            flip = int(splitmix64(rs, draw + 1, 1)[0] & np.uint64(1))
            draw += 2
            if f == t:
                continue
            u, v = int(a[t]), int(b[t])
            x, y = int(a[f]), int(b[f])
            if flip:
                x, y = y, x
            n1 = (min(u, x), max(u, x))
            n2 = (min(v, y), max(v, y))
            if n1[0] == n1[1] or n2[0] == n2[1] or n1 == n2:
                continue
            if counts.get(n1[0] * n + n1[1], 0) or counts.get(n2[0] * n + n2[1], 0):
                continue
            for k in (int(a[t] * n + b[t]), int(a[f] * n + b[f])):
                counts[k] -= 1
                if counts[k] == 0:
                    del counts[k]
            a[t], b[t] = n1
            a[f], b[f] = n2
            for k in (n1[0] * n + n1[1], n2[0] * n + n2[1]):
                counts[k] = counts.get(k, 0) + 1
            break
    return a, b


def regular_pm1(n: int, d: int, seed: int) -> CSR:
    """Random d-regular graph with couplings uniform in {-1, +1} (int8)."""
    a, b = random_regular(n, d, seed)
    s = signs(stream_seed(seed, TAG_SIGN), 0, a.size)
    return csr_from_upper(n, a, b, s)


def regular_gauss(n: int, d: int, seed: int) -> CSR:
    """Random d-regular graph with couplings N(0, 1) (float64 draws)."""
    a, b = random_regular(n, d, seed)
    g = gaussian(stream_seed(seed, TAG_GAUSS_A), stream_seed(seed, TAG_GAUSS_B), 0, a.size)
    return csr_from_upper(n, a, b, g)


def field_gauss(n: int, variance: float, seed: int) -> np.ndarray:
    """External field h_i ~ N(0, variance) (float64 draws)."""
    g = gaussian(stream_seed(seed, TAG_FIELD_A), stream_seed(seed, TAG_FIELD_B), 0, n)
    return np.sqrt(variance) * g


def x0_uniform(n: int, replicas: int, seed: int, dtype=np.float32) -> np.ndarray:
    """Starting points x0 uniform in [-1, 1), layout [n][R], rounded to ``dtype``.

    Draw t = r * n + i of the stream is component i of replica r.
    """
    u = uniform01(stream_seed(seed, TAG_X0), 0, n * replicas)
    x = (2.0 * u - 1.0).reshape(replicas, n).T
    return np.ascontiguousarray(x.astype(dtype))


def batched_sizes(count: int, lo: int, hi: int, dlo: int, dhi: int, seed: int):
    """Instance sizes n_b uniform in [lo, hi] and degrees d_b uniform in [dlo, dhi].

    When n_b * d_b is odd, n_b is raised by one so a d_b-regular graph exists.
    """
    u = splitmix64(stream_seed(seed, TAG_SIZE), 0, 2 * count)
    ns = lo + (u[:count] % np.uint64(hi - lo + 1)).astype(np.int64)
    ds = dlo + (u[count:] % np.uint64(dhi - dlo + 1)).astype(np.int64)
    ns = np.where((ns * ds) % 2 == 1, ns + 1, ns)
    return ns, ds
