"""The allocation-free lattice energy entry point against ising_energy.

ising_energy_torus_noalloc serves callers that cannot allocate device memory
(another allocator owns the device, or an allocation's possible device
synchronisation is not acceptable in their loop). Its reduction partials sit
in a fixed device array shared by every call, so these tests make calls in a
row with different replica counts, lattices and iterates, and check each
against the handle-based ising_energy, bit-exact (integer energies and
cuts). The shapes cover the launch clamps: a lattice with both sides 2 (both
wrap edges of a pair join the same two sites), few sites per replica, and
R = 8192, the documented limit (one chunk of sites per replica).
"""
import ctypes

import numpy as np
import pytest

from paper_2509_01928_gb300 import _native as N
from paper_2509_01928_gb300 import build as B
from paper_2509_01928_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _handle_energy(t, x):
    h = N.ising_create(N.Problem(t))
    try:
        R = x.shape[1]
        E = np.zeros(R, np.int64)
        cut = np.zeros(R, np.int64)
        N.ising_energy(h, torch.from_numpy(x).cuda(), E_int=E, cut_int=cut)
        return E, cut
    finally:
        N.ising_destroy(h)


@pytest.mark.parametrize("cases", [
    [((48, 1000), 5, 72), ((48, 1000), 2, 73)],          # the original pair of calls
    [((2, 4), 3, 75), ((2, 2), 1, 76), ((3, 2), 40, 77)],  # tiny lattices, 2-wide sides
    [((8, 16), 8192, 78), ((64, 96), 33, 79)],           # the replica limit, then a ragged tile
])
def test_noalloc_energy_matches_ising_energy_in_a_row(cases):
    assert torch.cuda.is_available()
    B.build_library()
    for call, ((lr, lc), R, seed) in enumerate(cases):
        t = I.torus_pm1(lr, lc, seed=seed)
        right = torch.from_numpy(t.right).cuda()
        down = torch.from_numpy(t.down).cuda()
        x = I.x0_uniform(t.n, R, seed=seed)
        x[::53] = 0.0                                   # sign(0) = +1 on both paths
        E_ref, cut_ref = _handle_energy(t, x)
        xd = torch.from_numpy(x).cuda()
        E = torch.full((R,), -7, dtype=torch.int64, device="cuda")
        cut = torch.full((R,), -7, dtype=torch.int64, device="cuda")
        N.ising_energy_torus_noalloc(right, down, xd, E_out=E, cut_out=cut)
        torch.cuda.synchronize()
        assert np.array_equal(E.cpu().numpy(), E_ref), f"call {call}"
        assert np.array_equal(cut.cpu().numpy(), cut_ref), f"call {call}"


def test_noalloc_energy_rejects_oversize_and_host_arrays():
    B.build_library()
    t = I.torus_pm1(4, 8, seed=74)
    right = torch.from_numpy(t.right).cuda()
    down = torch.from_numpy(t.down).cuda()
    x = torch.zeros((t.n, 8193), dtype=torch.float32, device="cuda")
    E = torch.zeros(8193, dtype=torch.int64, device="cuda")
    with pytest.raises(N.IsingError) as e:
        N.ising_energy_torus_noalloc(right, down, x, E_out=E)
    assert e.value.name == "ISING_ERR_INVALID_ARG"
    # host arrays reach the C entry point only through a direct call: rejected there
    lib = N.load()
    xh = np.zeros((t.n, 1), np.float32)
    Eh = np.zeros(1, np.int64)
    st = lib.ising_energy_torus_noalloc(t.right.ctypes.data, t.down.ctypes.data, 4, 8, xh.ctypes.data, 1,
                                        Eh.ctypes.data, None, None)
    assert N.STATUS_NAMES[st] == "ISING_ERR_INVALID_ARG"
