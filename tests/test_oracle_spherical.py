"""Pins of the spherical-harmonic transform the tests use (spherical_helpers):

  * orthonormality: with the Cartesian normalisation of the axial component,
    the analytic overlap of the six Cartesian d components of one Gaussian
    (moments int x^2k exp(-2a x^2) = (2k-1)!! / (4a)^k sqrt(pi / 2a)) becomes
    the identity under T;
  * rotational symmetry, through the oracle's integrals: for an s and a d
    shell on the same centre, (d_m s | d_m' s) is diagonal with equal diagonal
    elements for the Coulomb and erfc kernels (a spherically symmetric
    kernel and s functions cannot couple different m), which the Cartesian
    components are not.
"""
import numpy as np
import pytest

import oracle
import synth
from spherical_helpers import T_D


def _moment(k, a):
    # int x^(2k) exp(-2 a x^2) dx
    df = 1.0
    for j in range(1, 2 * k, 2):
        df *= j
    return df / (4.0 * a) ** k * np.sqrt(np.pi / (2.0 * a))


def test_d_harmonics_orthonormal():
    a = 0.7
    comps = [(2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)]
    S = np.zeros((6, 6))
    for i, ci in enumerate(comps):
        for j, cj in enumerate(comps):
            e = [ci[k] + cj[k] for k in range(3)]
            if any(x % 2 for x in e):
                continue
            S[i, j] = np.prod([_moment(x // 2, a) for x in e])
    S /= S[0, 0]  # the axial component has unit norm
    np.testing.assert_allclose(T_D @ S @ T_D.T, np.eye(5), rtol=0, atol=1e-14)
    assert abs(S[1, 1] - 1.0 / 3.0) < 1e-14  # xy itself is not unit-normalised


@pytest.mark.parametrize("kernel", [oracle.KERNEL_COULOMB, oracle.KERNEL_ERFC])
def test_d_harmonics_do_not_couple_through_s(kernel):
    rng = np.random.default_rng(5)
    s = synth.System(name="sd", atom_Z=np.array([6], dtype=np.int32), atom_xyz=np.zeros((1, 3)),
                     shell_atom=np.array([0, 0], dtype=np.int32), shell_l=np.array([0, 2], dtype=np.int32),
                     prim_off=np.array([0, 2, 5], dtype=np.int32),
                     alpha=np.array([3.0, 0.4, 5.0, 1.1, 0.3]), coef=rng.uniform(0.2, 1.0, size=5))
    b = oracle.Basis(s)
    (g,) = oracle.quartets(b, [(1, 0, 1, 0)], kernel=kernel, omega=0.11)
    M = g[:, 0, :, 0]
    Ms = T_D @ M @ T_D.T
    d = np.diag(Ms)
    assert np.abs(Ms - np.diag(d)).max() <= 1e-13 * d.max()
    assert np.ptp(d) <= 1e-13 * d.max()
    assert abs(M[0, 3]) > 1e-3 * M[0, 0]  # Cartesian xx and yy do couple
