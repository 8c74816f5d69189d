"""Light-cone patches of a periodic lattice -- oracle inputs, TEST INFRASTRUCTURE ONLY
(no method arithmetic; only the tests and the benchmark's CPU legs use it).

After N Jacobi steps of Eq. FPE the iterate of a lattice site depends only on
the sites within N lattice steps of it. So x^(N) on a block of sites can be
computed from the open-boundary sub-lattice that extends the block by N sites
in every direction: every site within N - 1 steps of the block has all of its
neighbours inside that patch. This module lays out such a patch as CSR with
the lattice's own couplings; the oracle run on that patch gives x^(N) of the
block's sites of the full lattice (checked against the full lattice on the
CPU by the test suite).
"""
import numpy as np

from paper_2509_01928_gb300 import inputs as I


def light_cone_patch(t, r0, c0, size, margin):
    """Open-boundary CSR of the lattice sites (r0 - margin .. r0 + size + margin - 1)
    x (c0 - margin .. c0 + size + margin - 1), indices taken modulo the lattice
    (which must be wider than the patch); the coupling between two patch sites is
    the lattice's own. Returns the CSR and the lattice index of every patch site
    (patch row-major)."""
    Lr, Lc = t.right.shape
    P = size + 2 * margin
    assert P <= Lr and P <= Lc
    gr = (r0 - margin + np.arange(P)) % Lr
    gc = (c0 - margin + np.arange(P)) % Lc
    G = gr[:, None] * Lc + gc[None, :]
    pid = np.arange(P * P).reshape(P, P)
    rows, cols, vals = [], [], []
    w = t.right[np.ix_(gr, gc)][:, :-1].ravel()      # (pr, pc) - (pr, pc + 1): right[gr, gc]
    a, b = pid[:, :-1].ravel(), pid[:, 1:].ravel()
    rows += [a, b]
    cols += [b, a]
    vals += [w, w]
    w = t.down[np.ix_(gr, gc)][:-1, :].ravel()       # (pr, pc) - (pr + 1, pc): down[gr, gc]
    a, b = pid[:-1, :].ravel(), pid[1:, :].ravel()
    rows += [a, b]
    cols += [b, a]
    vals += [w, w]
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rp = np.zeros(P * P + 1, np.int64)
    np.add.at(rp, r + 1, 1)
    return I.CSR(P * P, np.cumsum(rp), c.astype(np.int32), v), G.ravel()
