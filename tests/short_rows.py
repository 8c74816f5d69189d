"""Test graph for the CSR kernels that pipeline their loads across rows."""
import numpy as np

from paper_2509_01928_gb300 import inputs as I


def short_rows_mixed(n, seed):
    """A graph with short rows on average (about 3 entries) but every row shape the pipelined
    step meets: empty rows (every 97th vertex isolated), rows longer than the first batch (two
    hubs with 60 and 33 neighbours, one of them the last row) and 3-regular rows between."""
    g = I.regular_pm1(n, 3, seed=seed)
    rows = np.repeat(np.arange(n), np.diff(g.row_ptr))
    up = rows < g.col
    i, j, v = rows[up], g.col[up].astype(np.int64), g.val[up]
    iso = (i % 97 == 0) | (j % 97 == 0)
    i, j, v = i[~iso], j[~iso], v[~iso]
    rng = np.random.default_rng(seed)
    hubs = []
    for hub, deg in ((5, 60), (n - 1, 33)):
        nb = rng.choice(np.setdiff1d(np.arange(1, n - 1), [5]), size=deg, replace=False)
        nb = nb[nb % 97 != 0]
        hubs.append((np.minimum(hub, nb), np.maximum(hub, nb), rng.choice([-1, 1], size=nb.size)))
    ii = np.concatenate([i] + [h[0] for h in hubs])
    jj = np.concatenate([j] + [h[1] for h in hubs])
    vv = np.concatenate([v] + [h[2].astype(v.dtype) for h in hubs])
    key = ii * n + jj
    _, first = np.unique(key, return_index=True)
    return I.csr_from_upper(n, ii[first], jj[first], vv[first])
