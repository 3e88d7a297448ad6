"""The device Boys-function evaluators (used by every ERI kernel) against the
oracle's long-double series: the FP64 Taylor/downward evaluator to 5e-14
relative, the double-single one of the mixed path to 2e-12 relative, over
arguments spanning grid points, grid mid-points, the 60 switch to the
asymptotic form and large values.  Double-single numbers carry an FP32
exponent: values below 1e-30 (F_8 beyond T ~ 3e4, irrelevant to any
integral) are compared in absolute terms, to 1e-37."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _args():
    rng = np.random.default_rng(5)
    T = np.concatenate([[0.0, 1e-9, 1e-4, 1.0 / 32, 1.0 / 16, 0.5, 1.0, 7.03125, 29.96875, 35.0, 59.96875,
                         59.999, 60.0, 60.001, 75.0, 300.0, 5e3, 7e4],
                        rng.uniform(0, 60, 400), np.exp(rng.uniform(np.log(60), np.log(1e5), 100))])
    return T


@pytest.mark.parametrize("prec,tol", [(0, 5e-14), (1, 2e-12)])
@pytest.mark.parametrize("mmax", [0, 1, 4, 8])
def test_device_boys(prec, tol, mmax):
    from paper_2009_03555_gb300 import hfx
    b = hfx.Basis(synth.water_dimer(0))
    T = _args()
    F = b.boys(T, mmax, precision=prec)
    ref = np.array([oracle.boys(mmax, t) for t in T])
    big = np.abs(ref) > (1e-30 if prec == 1 else 0.0)
    rel = np.where(big, np.abs(F - ref) / np.where(big, np.abs(ref), 1.0), 0.0)
    assert rel.max() <= tol, (rel.max(), T[np.unravel_index(rel.argmax(), rel.shape)[0]])
    assert np.all(np.abs(F - ref)[~big] <= 1e-37)
