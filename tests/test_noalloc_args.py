"""Argument checks of the allocation-free lattice energy binding, on the CPU:
wrong types and shapes are rejected with ValueError before the C entry point
(which cannot see array lengths) is reached."""
import numpy as np
import pytest

from paper_2509_01928_gb300 import _native as N

torch = pytest.importorskip("torch")


def _args(lr=4, lc=6, R=3):
    right = torch.ones((lr, lc), dtype=torch.int8)
    down = torch.ones((lr, lc), dtype=torch.int8)
    x = torch.zeros((lr * lc, R), dtype=torch.float32)
    E = torch.zeros(R, dtype=torch.int64)
    cut = torch.zeros(R, dtype=torch.int64)
    return right, down, x, E, cut


@pytest.mark.parametrize("case", ["right_dtype", "down_shape", "x_dtype", "x_rows", "x_3d", "E_short",
                                  "E_dtype", "cut_short", "no_output", "numpy", "not_contiguous", "cpu"])
def test_noalloc_rejects_before_the_call(case):
    right, down, x, E, cut = _args()
    kw = {"E_out": E, "cut_out": cut}
    if case == "right_dtype":
        right = right.to(torch.int16)
    elif case == "down_shape":
        down = torch.ones((4, 5), dtype=torch.int8)
    elif case == "x_dtype":
        x = x.double()
    elif case == "x_rows":
        x = torch.zeros((23, 3), dtype=torch.float32)
    elif case == "x_3d":
        x = torch.zeros((24, 3, 1), dtype=torch.float32)
    elif case == "E_short":
        kw["E_out"] = torch.zeros(2, dtype=torch.int64)
    elif case == "E_dtype":
        kw["E_out"] = torch.zeros(3, dtype=torch.int32)
    elif case == "cut_short":
        kw["cut_out"] = torch.zeros(1, dtype=torch.int64)
    elif case == "no_output":
        kw = {}
    elif case == "numpy":
        right = np.ones((4, 6), np.int8)
    elif case == "not_contiguous":
        x = torch.zeros((3, 24), dtype=torch.float32).t()
    # "cpu": every check but the device one passes
    with pytest.raises(ValueError):
        N.ising_energy_torus_noalloc(right, down, x, **kw)
