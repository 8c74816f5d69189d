"""Procedural dense couplings J_ij = sin(i j + 100) (Supplementary Note 9): the
reference matrix, and the fixed-point constant the device uses for the
argument reduction, floor(2^96 / (2 pi)), against a high-precision value."""
import numpy as np
import pytest

from oracle import matrices as M


def test_procedural_reference_matrix():
    J = M.procedural_sin(50)
    assert J.shape == (50, 50) and np.array_equal(J, J.T) and np.all(np.diag(J) == 0)
    assert J[0, 1] == np.sin(1 * 2 + 100.0) and J[9, 3] == np.sin(10 * 4 + 100.0)


def test_phase_constant():
    sympy = pytest.importorskip("sympy")
    F = 0x28BE60DB9391054A7F09D5F4          # the value the device code uses
    exact = sympy.Integer(2) ** 96 / (2 * sympy.pi)
    assert sympy.floor(exact) == F
    # the phase of a = i j + 100 modulo 2^96 gives frac(a / (2 pi)) within a 2^-96 per unit of a
    a = 99999 * 99998 + 100
    frac_fixed = ((a * F) % (1 << 96)) / sympy.Integer(2) ** 96
    frac_exact = sympy.Rational(a, 1) / (2 * sympy.pi) - sympy.floor(sympy.Rational(a, 1) / (2 * sympy.pi))
    assert abs(sympy.N(frac_fixed - frac_exact, 50)) < sympy.Float(a) * sympy.Integer(2) ** -96 * 2
