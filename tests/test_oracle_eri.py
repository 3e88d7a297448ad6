"""Pins for the oracle's contracted shell-quartet ERIs.

ERIs follow Sec. 2 (full-range ERI definition for 1/r; Eq. ERI-SR for
erfc(w r)/r with w = 0.11 bohr^-1; erf is its complement).  Pinned against:
  * brute-force numerical quadrature of the six-dimensional integral
    (tests/quadrature.py: Gaussian transform of the kernel, Gauss-Hermite per
    axis, adaptive quadrature in t) for every angular-momentum combination of
    s, p, d, all three kernels;
  * the textbook interaction of two unit Gaussian charge clouds,
    erf(sqrt(mu) R)/R (Coulomb) and erf(sqrt(mu') R)/R with
    1/mu' = 1/mu + 1/w^2 (erf kernel);
  * the 8-fold permutation symmetry (Sec. 2), erf + erfc = Coulomb, the
    limits w -> 0 and w -> infinity, translation invariance and the cyclic
    relabelling of Cartesian axes;
  * numerically computed normalisation.
"""
import itertools
import math

import numpy as np
import pytest
from scipy.special import erf

import oracle
import synth
from quadrature import cart_components, eri_quadrature, normalized_coefs

K_NAMES = {"coulomb": oracle.KERNEL_COULOMB, "erfc": oracle.KERNEL_ERFC, "erf": oracle.KERNEL_ERF}


@pytest.fixture(scope="module")
def small():
    s = synth.ch_cluster(3, 99, nprim=2)
    return s, oracle.Basis(s)


def _shell_tuple(s, b, S):
    p0, p1 = s.prim_off[S], s.prim_off[S + 1]
    return (s.atom_xyz[s.shell_atom[S]], int(s.shell_l[S]), s.alpha[p0:p1], b.coef[p0:p1])


def test_normalisation_matches_quadrature(small):
    s, b = small
    sw = synth.water_dimer(0)
    for sysobj in (s, sw):
        bb = oracle.Basis(sysobj)
        for S in range(sysobj.n_shells):
            p0, p1 = sysobj.prim_off[S], sysobj.prim_off[S + 1]
            ref = normalized_coefs(int(sysobj.shell_l[S]), sysobj.alpha[p0:p1], sysobj.coef[p0:p1])
            np.testing.assert_allclose(bb.coef[p0:p1], ref, rtol=1e-13)


def _shells_by_l(s):
    by = {0: [], 1: [], 2: []}
    for S in range(s.n_shells):
        by[int(s.shell_l[S])].append(S)
    return by


# one quartet per (la, lb, lc, ld) pattern, shells on different atoms where possible
L_PATTERNS = [(0, 0, 0, 0), (1, 0, 0, 0), (0, 1, 1, 0), (1, 1, 1, 1), (2, 0, 0, 0), (2, 1, 0, 1),
              (0, 2, 2, 0), (2, 2, 1, 0), (1, 2, 2, 1), (2, 2, 2, 2)]


@pytest.mark.parametrize("pattern", L_PATTERNS)
@pytest.mark.parametrize("kname", ["coulomb", "erfc", "erf"])
def test_quartet_vs_quadrature(small, pattern, kname):
    s, b = small
    by = _shells_by_l(s)
    rng = np.random.default_rng(hash(pattern) % 1000)
    quad = [int(rng.choice(by[l])) for l in pattern]
    ref = eri_quadrature([_shell_tuple(s, b, S) for S in quad], kname)
    got = oracle.quartets(b, [quad], K_NAMES[kname])[0]
    scale = max(1.0, np.abs(ref).max())
    np.testing.assert_allclose(got, ref, rtol=0, atol=2e-13 * scale)


def _one_prim_system(xyz, alphas):
    n = len(alphas)
    return synth.System(name="s_prims", atom_Z=np.ones(n, dtype=np.int32),
                        atom_xyz=np.asarray(xyz, dtype=np.float64),
                        shell_atom=np.arange(n, dtype=np.int32), shell_l=np.zeros(n, dtype=np.int32),
                        prim_off=np.arange(n + 1, dtype=np.int32),
                        alpha=np.asarray(alphas, dtype=np.float64), coef=np.ones(n))


@pytest.mark.parametrize("R", [0.0, 0.7, 3.0, 11.0])
def test_gaussian_charge_interaction(R):
    """(aa|cc) for unit-normalised s Gaussians is the interaction of two unit
    Gaussian charges with exponents 2a and 2c: erf(sqrt(mu) R)/R."""
    a, c, w = 0.8, 2.3, 0.11
    s = _one_prim_system([[0.0, 0.0, 0.0], [R, 0.0, 0.0]], [a, c])
    b = oracle.Basis(s)
    mu = (2 * a) * (2 * c) / (2 * a + 2 * c)
    mu_w = 1.0 / (1.0 / mu + 1.0 / (w * w))

    def f(m):
        return 2.0 * math.sqrt(m / math.pi) if R == 0.0 else erf(math.sqrt(m) * R) / R

    coul = oracle.quartets(b, [(0, 0, 1, 1)], oracle.KERNEL_COULOMB, w)[0].item()
    erfk = oracle.quartets(b, [(0, 0, 1, 1)], oracle.KERNEL_ERF, w)[0].item()
    erfck = oracle.quartets(b, [(0, 0, 1, 1)], oracle.KERNEL_ERFC, w)[0].item()
    assert coul == pytest.approx(f(mu), rel=1e-14)
    assert erfk == pytest.approx(f(mu_w), rel=1e-13)
    assert erfck == pytest.approx(f(mu) - f(mu_w), rel=1e-12, abs=1e-15)


def _random_quartets(s, n, rng):
    return [tuple(int(x) for x in rng.integers(0, s.n_shells, size=4)) for _ in range(n)]


def test_eightfold_symmetry(small):
    s, b = small
    rng = np.random.default_rng(7)
    for q in _random_quartets(s, 25, rng):
        I, J, K, L = q
        base = oracle.quartets(b, [q], oracle.KERNEL_ERFC)[0]
        perms = {(J, I, K, L): (1, 0, 2, 3), (I, J, L, K): (0, 1, 3, 2), (J, I, L, K): (1, 0, 3, 2),
                 (K, L, I, J): (2, 3, 0, 1), (L, K, I, J): (3, 2, 0, 1), (K, L, J, I): (2, 3, 1, 0),
                 (L, K, J, I): (3, 2, 1, 0)}
        for pq, axes in perms.items():
            other = oracle.quartets(b, [pq], oracle.KERNEL_ERFC)[0]
            np.testing.assert_allclose(np.transpose(base, axes), other, rtol=1e-12, atol=1e-15)


def test_erf_plus_erfc_is_coulomb(small):
    s, b = small
    rng = np.random.default_rng(8)
    qs = _random_quartets(s, 20, rng)
    c = oracle.quartets(b, qs, oracle.KERNEL_COULOMB)
    e = oracle.quartets(b, qs, oracle.KERNEL_ERF)
    ec = oracle.quartets(b, qs, oracle.KERNEL_ERFC)
    for x, y, z in zip(c, e, ec):
        np.testing.assert_allclose(y + z, x, rtol=0, atol=1e-14 * max(1.0, np.abs(x).max()))


def test_omega_limits(small):
    s, b = small
    rng = np.random.default_rng(9)
    qs = _random_quartets(s, 10, rng)
    c = oracle.quartets(b, qs, oracle.KERNEL_COULOMB)
    big = oracle.quartets(b, qs, oracle.KERNEL_ERFC, 1e4)
    tiny = oracle.quartets(b, qs, oracle.KERNEL_ERFC, 1e-9)
    for x, y, z in zip(c, big, tiny):
        m = max(1.0, np.abs(x).max())
        assert np.abs(y).max() < 1e-5 * m  # erfc(w r)/r -> 0 (Gaussian tails ~ 1/w^2)
        np.testing.assert_allclose(z, x, rtol=0, atol=1e-8 * m)


def test_translation_invariance(small):
    s, b = small
    rng = np.random.default_rng(10)
    qs = _random_quartets(s, 10, rng)
    b2 = oracle.Basis(s.translated([3.7, -1.2, 0.4]))
    for k in (oracle.KERNEL_COULOMB, oracle.KERNEL_ERFC):
        for x, y in zip(oracle.quartets(b, qs, k), oracle.quartets(b2, qs, k)):
            np.testing.assert_allclose(y, x, rtol=0, atol=1e-12 * max(1.0, np.abs(x).max()))


def test_cyclic_axis_relabelling(small):
    """Moving every centre (x, y, z) -> (z, x, y) maps component (ex, ey, ez) to
    (ez, ex, ey); catches any mix-up of axes or component order."""
    s, b = small
    rot = s.translated([0, 0, 0])
    rot.atom_xyz = np.ascontiguousarray(s.atom_xyz[:, [2, 0, 1]])
    br = oracle.Basis(rot)
    rng = np.random.default_rng(11)
    qs = _random_quartets(s, 12, rng)
    for q, x, y in zip(qs, oracle.quartets(b, qs, 1), oracle.quartets(br, qs, 1)):
        maps = []
        for S in q:
            comps = cart_components(int(s.shell_l[S]))
            idx = {c: i for i, c in enumerate(comps)}
            maps.append([idx[(c[2], c[0], c[1])] for c in comps])
        expect = x
        moved = np.zeros_like(y)
        for a, bb, c, d in itertools.product(*(range(len(m)) for m in maps)):
            moved[maps[0][a], maps[1][bb], maps[2][c], maps[3][d]] = expect[a, bb, c, d]
        np.testing.assert_allclose(y, moved, rtol=0, atol=1e-12 * max(1.0, np.abs(x).max()))


def test_schwarz_inequality(small):
    s, b = small
    Q = oracle.schwarz(b, oracle.KERNEL_ERFC)
    rng = np.random.default_rng(12)
    qs = _random_quartets(s, 40, rng)
    for q, x in zip(qs, oracle.quartets(b, qs, oracle.KERNEL_ERFC)):
        I, J, K, L = q
        assert np.abs(x).max() <= Q[I, J] * Q[K, L] * (1 + 1e-12) + 1e-300
    assert np.allclose(Q, Q.T)
