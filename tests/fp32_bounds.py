"""FP32 parity bound for iterations with weakly stable fixed points (test helper).

On random graphs and dense couplings some replicas approach fixed points where
the iteration contracts slowly, and FP32 rounding alone moves them away from
the FP64 trajectory by more than the 1e-5 FP32 bar after a few steps. The
bound used there: each replica r must satisfy rel_r <= max(1e-5, 16 delta_r),
with delta_r the drift of the oracle's own trajectory when every step's output
is perturbed by the step's FP32 rounding (relative eps_step, seeded signs),
and the median replica must be within max(1e-5, 4 median_r delta_r).

eps_step is 2^-24 (one rounding) where a step sums a handful of terms (the
lattice stencil, sparse rows). A dense step sums n products in FP32, whose
accumulated rounding grows like sqrt(n) 2^-24 relative to the sum of the
absolute terms (the random-walk model of rounding errors); there
eps_step = sqrt(n) 2^-24.
"""
import numpy as np

import oracle as O
from paper_2509_01928_gb300 import inputs as I

TOL32 = 1e-5


def fp32_drift(P, x0, alpha, beta, iters, eps_step=2.0 ** -24):
    """The oracle trajectory x^(iters) and, per replica, its relative drift when every
    component is perturbed by a relative eps_step after each step (max over two seeded sign
    patterns)."""
    ref = O.doch(P, x0, alpha, beta, iters)
    a = np.broadcast_to(np.asarray(alpha, dtype=np.float64), (iters,))
    out = np.zeros(ref.shape[1])
    for seed in (1, 2):
        x = np.asarray(x0, dtype=np.float64)
        for j in range(iters):
            x = O.doch(P, x, a[j], beta, 1)
            sg = I.signs(I.stream_seed(seed, 200 + j), 0, x.size).reshape(x.shape)
            x = x * (1.0 + sg * eps_step)
        out = np.maximum(out, np.linalg.norm(x - ref, axis=0) / np.linalg.norm(ref, axis=0))
    return ref, out


def close32_conditioned(x_gpu, ref, drift):
    x_gpu = np.asarray(x_gpu, dtype=np.float64).reshape(ref.shape)
    rel = np.linalg.norm(x_gpu - ref, axis=0) / np.linalg.norm(ref, axis=0)
    bound = np.maximum(TOL32, 16.0 * drift)
    assert np.all(rel <= bound), f"replica error {rel.max():.3e} above its bound {bound[np.argmax(rel)]:.3e}"
    med = max(TOL32, 4.0 * float(np.median(drift)))
    assert np.median(rel) <= med, f"median replica error {np.median(rel):.3e} > {med:.3e}"
