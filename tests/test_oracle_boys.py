"""Pins for the oracle's Boys function F_m(x) = int_0^1 t^{2m} exp(-x t^2) dt.

The Boys function is the auxiliary of the analytic Gaussian ERIs (Sec. 2,
full-range and short-range ERI definitions).  Pinned against: F_m(0) =
1/(2m+1); the closed form F_0(x) = sqrt(pi/(4x)) erf(sqrt x); the regularised
lower incomplete gamma function F_m(x) = Gamma(m+1/2) P(m+1/2, x) / (2 x^{m+1/2});
and the defining integral evaluated by mpmath at 30 digits.
"""
import math

import mpmath
import numpy as np
import pytest
from scipy.special import erf, gamma, gammainc

import oracle

XS = np.concatenate([[1e-12, 1e-6, 1e-3, 0.05, 0.5, 1.0, 2.5, 7.0, 12.0, 20.0, 30.0],
                     [34.999, 35.0, 35.001, 40.0, 60.0, 100.0, 500.0, 3000.0]])


@pytest.mark.parametrize("m", range(0, 17))
def test_boys_at_zero(m):
    assert oracle.boys(m, 0.0)[m] == pytest.approx(1.0 / (2 * m + 1), rel=1e-15)


def test_boys_f0_closed_form():
    for x in XS:
        if x < 1e-6:
            continue
        ref = 0.5 * math.sqrt(math.pi / x) * erf(math.sqrt(x))
        assert oracle.boys(0, x)[0] == pytest.approx(ref, rel=2e-15)


@pytest.mark.parametrize("mmax", [4, 8, 16])
def test_boys_incomplete_gamma(mmax):
    for x in XS:
        F = oracle.boys(mmax, x)
        for m in range(mmax + 1):
            a = m + 0.5
            ref = gamma(a) * gammainc(a, x) / (2.0 * x ** a)
            assert F[m] == pytest.approx(ref, rel=5e-14), (m, x)


def test_boys_definition_mpmath():
    mpmath.mp.dps = 30
    for m in (0, 3, 8):
        for x in (0.3, 9.0, 34.5, 35.5, 80.0):
            ref = mpmath.quad(lambda t: t ** (2 * m) * mpmath.exp(-x * t * t), [0, 1])
            assert oracle.boys(8, x)[m] == pytest.approx(float(ref), rel=1e-14), (m, x)
