"""Reference forms of the generated coupling matrices -- TEST INFRASTRUCTURE ONLY.

Part of the oracle: only the tests, the smoke check and the benchmark's CPU
legs may import it. Each function restates a matrix the paper defines, as the
checker of the library's on-device generation:
  * ``s5_csr``          -- Algorithm S5 (Supplementary Note 9), the p-sparse
                           9-bit couplings, drawn from the counter-based
                           SplitMix64 stream of the inputs module;
  * ``procedural_sin``  -- the procedural dense couplings J_ij = sin(i j + c)
                           of Supplementary Note 9 (1-based, J_ii = 0), FP64.
"""
from __future__ import annotations

import numpy as np

from paper_2509_01928_gb300.inputs import CSR, TAG_S5, _CHUNK, csr_from_upper, splitmix64, stream_seed


def s5_params(p: float):
    """N_p = floor(102300 / p) for p in percent (the IEEE double quotient, then the
    floor, so that p = 0.05 gives 2046000), and the keep threshold of a draw:
    with z = 1 + floor(u N_p / 2^64) (u a 64-bit stream value), z < 1023 exactly
    when u < T = ceil(1022 * 2^64 / N_p)."""
    if not (0.0 < p <= 100.0):
        raise ValueError("p must be in (0, 100]")
    n_p = int(np.floor(np.float64(102300.0) / np.float64(p)))
    thr = -((-1022 << 64) // n_p)  # ceil
    return n_p, min(thr, 1 << 64)


def _mulhi64(u: np.ndarray, m: int) -> np.ndarray:
    """floor(u m / 2^64) for uint64 u and an integer 0 < m < 2^64, exactly."""
    m_lo, m_hi = np.uint64(m & 0xFFFFFFFF), np.uint64(m >> 32)
    mask = np.uint64(0xFFFFFFFF)
    u_lo, u_hi = u & mask, u >> np.uint64(32)
    with np.errstate(over="ignore"):
        ll = u_lo * m_lo
        lh = u_lo * m_hi
        hl = u_hi * m_lo
        hh = u_hi * m_hi
        mid = (ll >> np.uint64(32)) + (lh & mask) + (hl & mask)
        return hh + (lh >> np.uint64(32)) + (hl >> np.uint64(32)) + (mid >> np.uint64(32))


def s5_csr(n: int, p: float, seed: int) -> CSR:
    """Algorithm S5 (Supplementary Note 9): for every pair i > j (0-based), draw
    z in {1, ..., N_p}; if z < 1023 then J_ij = J_ji = z - 511 (a 9-bit signed
    value, stored even when it is 0). The draw of pair (i, j) is value
    t = i (i - 1) / 2 + j of the stream stream_seed(seed, TAG_S5) (the order of
    the algorithm's loops), mapped by z = 1 + floor(u N_p / 2^64). Returns the
    symmetric CSR matrix with int16 values."""
    n_p, thr = s5_params(p)
    sd = stream_seed(seed, TAG_S5)
    ii, jj, vv = [], [], []
    t0 = 0
    block = max(1, _CHUNK // max(1, n))
    for i0 in range(1, n, block):
        i1 = min(n, i0 + block)
        count = (i1 * (i1 - 1)) // 2 - t0
        u = splitmix64(sd, t0, count)
        keep = np.nonzero(u < np.uint64(thr))[0] if thr < (1 << 64) else np.arange(count)
        if keep.size:
            t = keep + t0
            i = np.floor((1.0 + np.sqrt(1.0 + 8.0 * t.astype(np.float64))) / 2.0).astype(np.int64)
            i -= (i * (i - 1) // 2 > t).astype(np.int64)      # exact row of the triangle index
            i += ((i + 1) * i // 2 <= t).astype(np.int64)
            j = t - i * (i - 1) // 2
            z = 1 + _mulhi64(u[keep], n_p).astype(np.int64)
            ii.append(i)
            jj.append(j)
            vv.append((z - 511).astype(np.int16))
        t0 += count
    if ii:
        i, j, v = np.concatenate(ii), np.concatenate(jj), np.concatenate(vv)
    else:
        i = j = np.zeros(0, np.int64)
        v = np.zeros(0, np.int16)
    return csr_from_upper(n, j, i, v)


def procedural_sin(n: int, offset: float = 100.0) -> np.ndarray:
    """Dense J_ij = sin(i j + offset) for 1-based i != j, J_ii = 0 (FP64; the
    argument i j + offset is an exact double for i j < 2^53)."""
    idx = np.arange(1, n + 1, dtype=np.float64)
    J = np.sin(np.outer(idx, idx) + offset)
    np.fill_diagonal(J, 0.0)
    return J
