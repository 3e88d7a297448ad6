"""The seeded input generators (CPU): the workload recipe the tests and the
benchmark rely on -- sizes, geometry rules, exponent and coefficient laws,
determinism -- and the properties of the synthetic density matrices.
"""
import numpy as np
import pytest

import synth


def test_water_dimer_recipe():
    s, P = synth.config0()
    assert s.n_atoms == 6 and s.n_shells == 22 and s.n_bf == 38
    assert list(s.atom_Z) == [8, 1, 1, 8, 1, 1]
    d = synth.atom_distances(s)
    for o, hs in ((0, (1, 2)), (3, (4, 5))):
        for h in hs:
            assert abs(d[o, h] - 1.81) < 0.35          # O-H 1.81 bohr, +-0.1 jitter per coordinate
    assert abs(d[0, 3] - 5.5) < 0.35                     # O-O 5.5 bohr
    assert np.all(np.diff(s.prim_off) == 3)              # 3 primitives per shell
    assert s.n_occ == 10
    np.testing.assert_allclose(P, P.T, atol=0)
    np.testing.assert_allclose(P @ P, P, atol=1e-12)     # P = C C^T with orthonormal C
    assert abs(np.trace(P) - 10) < 1e-12


def test_cluster_recipe_400():
    s = synth.ch_cluster(400, 2)
    assert s.n_atoms == 400 and s.n_shells == 2000 and s.n_bf == 5600
    d = synth.atom_distances(s)
    np.fill_diagonal(d, np.inf)
    assert d.min() >= 2.2                                # minimum spacing
    assert s.atom_xyz.min() >= 0.0 and s.atom_xyz.max() <= 30.0   # 30 bohr box
    assert list(s.atom_Z[:4]) == [6, 1, 6, 1]            # C/H alternating
    assert np.all(np.diff(s.prim_off) == 4)              # 4 primitives per shell
    per_atom = np.bincount(s.shell_atom, minlength=400)
    assert np.all(per_atom == 5)                         # 2s + 2p + 1d
    assert list(np.bincount(s.shell_l)) == [800, 800, 400]   # s, p, d shells
    assert s.alpha.min() >= 0.1 and s.alpha.max() <= 50.0          # log-uniform in [0.1, 50]
    for S in range(0, s.n_shells, 97):                   # sorted descending within a shell
        a = s.alpha[s.prim_off[S]:s.prim_off[S + 1]]
        assert np.all(np.diff(a) <= 0)
    assert s.coef.min() > 0.1 - 1e-12 and s.coef.max() <= 1.0     # U(0.1, 1]


def test_generators_are_deterministic_and_seeded():
    a, b = synth.ch_cluster(40, 3, sub=5), synth.ch_cluster(40, 3, sub=5)
    np.testing.assert_array_equal(a.atom_xyz, b.atom_xyz)
    np.testing.assert_array_equal(a.alpha, b.alpha)
    c = synth.ch_cluster(40, 3, sub=6)
    assert not np.array_equal(a.atom_xyz, c.atom_xyz)
    P1 = synth.density_matrix(a, 3, sub=5)
    P2 = synth.density_matrix(b, 3, sub=5)
    np.testing.assert_array_equal(P1, P2)


@pytest.mark.parametrize("make,spacing,dim", [(lambda: synth.ch_chain(30, sub=1), 2.8, 1),
                                              (lambda: synth.ch_slab(25, sub=2), 4.0, 2)])
def test_chain_and_slab_geometry(make, spacing, dim):
    s = make()
    d = synth.atom_distances(s)
    np.fill_diagonal(d, np.inf)
    nearest = d.min(axis=1)
    assert np.all(np.abs(nearest - spacing) < 0.5)        # lattice spacing, 0.1 bohr jitter
    extent = np.ptp(s.atom_xyz, axis=0)
    assert np.sum(extent > 1.0) == dim                    # a chain spans one axis, a slab two


def test_density_cutoff_and_perturbation():
    s = synth.ch_cluster(30, 4, sub=1)
    P = synth.density_matrix(s, 4, cutoff=6.0, sub=1)
    mask = synth.atom_pair_mask(s, 6.0)
    dense_mask = synth.expand_atom_mask(s, mask)
    assert np.all(P[dense_mask == 0] == 0)               # blocks beyond the cutoff are zero
    np.testing.assert_allclose(P, P.T, atol=0)
    Q = synth.perturb_density(P, np.random.default_rng(1), rel=1e-3)
    np.testing.assert_allclose(Q, Q.T, atol=0)           # symmetric noise
    assert np.all(Q[P == 0] == 0)                        # pattern kept
    nz = P != 0
    rel = np.abs(Q[nz] / P[nz] - 1)
    assert 0 < rel.max() < 1e-2 and rel.mean() < 2e-3    # relative noise of order 1e-3
