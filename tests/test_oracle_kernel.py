"""Pins of the oracle's smoothing kernel against closed forms (no GPU).

The kernel must integrate to one in its own dimension (normalisation of the convolution in
Eq. 12), vanish with zero slope at the support radius, and its derivative must be the
derivative of the kernel (checked by finite differences, not by retyping the formula).
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O

SHELL = {1: lambda r: 2.0, 2: lambda r: 2.0 * math.pi * r, 3: lambda r: 4.0 * math.pi * r * r}


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("h", [0.0037, 1.0, 4.88])
def test_kernel_normalised(d, h):
    R = 2.0 * h
    val, err = integrate.quad(lambda r: SHELL[d](r) * O.W(d, r, h), 0.0, R, epsabs=0, epsrel=1e-13, limit=200)
    assert abs(val - 1.0) < 1e-11


@pytest.mark.parametrize("d", [1, 2, 3])
def test_kernel_support_and_slope(d):
    h = 0.3
    R = 2.0 * h
    assert O.W(d, R, h) == 0.0 and O.W(d, 1.5 * R, h) == 0.0
    assert O.dW(d, R, h) == 0.0 and O.dW(d, 0.0, h) == 0.0
    assert O.W(d, 0.0, h) > 0
    r = np.linspace(0, R, 101)
    w = np.array([O.W(d, x, h) for x in r])
    assert np.all(np.diff(w) <= 0)          # monotone decreasing
    assert abs(O.W(d, R * (1 - 1e-3), h)) < 1e-9 * O.W(d, 0, h)   # C2 contact at the support edge


@pytest.mark.parametrize("d", [1, 2, 3])
def test_kernel_derivative_matches_finite_difference(d):
    h = 0.7
    for q in [0.05, 0.2, 0.5, 0.77, 0.95]:
        r = q * 2.0 * h
        e = 1e-6 * h
        fd = (O.W(d, r + e, h) - O.W(d, r - e, h)) / (2 * e)
        assert abs(O.dW(d, r, h) - fd) <= 1e-7 * abs(fd) + 1e-12


def test_lattice_shepard_sum_converges_to_one():
    # Riemann sum of W over a fine square lattice -> integral = 1 (pins the 2D normalisation
    # as used inside the oracle's density sum, Eq. 20).
    h = 1.0
    for s, tol in [(0.25, 2e-3), (0.125, 2e-4)]:
        m = int(math.ceil(2 * h / s)) + 1
        tot = 0.0
        for i in range(-m, m + 1):
            for j in range(-m, m + 1):
                tot += O.W(2, math.hypot(i * s, j * s), h) * s * s
        assert abs(tot - 1.0) < tol
