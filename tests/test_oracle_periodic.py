"""Pins of the oracle's periodic exchange (CPU).

The periodic form of Eq. H-HFX (Sec. 2): K^G_{mu lambda} = sum_{N,H} sum_{nu sigma}
P^{H-N}_{nu sigma} (mu^0 nu^N | lambda^G sigma^H), mu in the home cell, the cells
N, G, H over the extended set, the Gamma-point real-space density of Eq. dm
(P^L = the home density where the atoms are at most r_P apart).  The oracle
sums it by brute force over home rows.  Pinned here by:
  * the image list against a plain enumeration of a large block of shifts;
  * the molecular oracle (pinned to quadrature elsewhere) run on an extended
    atom set built here independently, whose rows of the home atoms must
    equal the periodic rows: the lattice sum is a molecular exchange over the
    extended set;
  * a lattice too large for any image: the molecular exchange of the cell;
  * a unimodular change of lattice vectors (the same crystal): same images,
    same rows;
  * the same crystal described by a doubled supercell: with short-ranged
    shells and a generous extended set, the rows of the cell's atoms agree.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth

SKEW = np.array([[6.0, 0.0, 0.0], [1.0, 6.0, 0.0], [0.0, 1.0, 6.0]])
FCC = 7.0 * np.array([[0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
D_RECIPE = {"C": [0, 1, 2], "H": [0, 1]}


def enumerate_images(xyz, A, r_ext, m=8):
    """(a, n1, n2, n3) with n != 0 and R_a + n.A within r_ext of a home atom, by
    testing every shift of a (2m+1)^3 block."""
    out = set()
    for n in itertools.product(range(-m, m + 1), repeat=3):
        if n == (0, 0, 0):
            continue
        pos = xyz + np.array(n, dtype=np.float64) @ A
        d = np.linalg.norm(pos[:, None, :] - xyz[None, :, :], axis=-1)
        for a in np.flatnonzero(d.min(axis=1) <= r_ext):
            out.add((int(a),) + n)
    return out


def extended_system(s, A, images):
    """The extended atom set as a molecule: home atoms, then the images in the
    given order, each with its home atom's shells."""
    atoms = [(a, (0, 0, 0)) for a in range(s.n_atoms)] + [(r[0], tuple(r[1:])) for r in images]
    xyz, Z, sa, sl, off, al, co = [], [], [], [], [0], [], []
    for X, (a, n) in enumerate(atoms):
        xyz.append(s.atom_xyz[a] + np.array(n, dtype=np.float64) @ A)
        Z.append(s.atom_Z[a])
        for S in np.flatnonzero(s.shell_atom == a):
            p0, p1 = s.prim_off[S], s.prim_off[S + 1]
            sa.append(X)
            sl.append(s.shell_l[S])
            al.extend(s.alpha[p0:p1])
            co.extend(s.coef[p0:p1])
            off.append(off[-1] + p1 - p0)
    e = synth.System(name="ext", atom_Z=np.array(Z, dtype=np.int32), atom_xyz=np.array(xyz),
                     shell_atom=np.array(sa, dtype=np.int32), shell_l=np.array(sl, dtype=np.int32),
                     prim_off=np.array(off, dtype=np.int32), alpha=np.array(al), coef=np.array(co))
    return e, atoms


def extended_density(s, e, atoms, P, r_P):
    """P over the extended set: block (X, Y) = home block (home(X), home(Y))
    where the two atoms are at most r_P apart."""
    hf, ef = s.atom_func_off, e.atom_func_off
    Pe = np.zeros((e.n_bf, e.n_bf))
    d = synth.atom_distances(e)
    for X, (a, _) in enumerate(atoms):
        for Y, (b, _) in enumerate(atoms):
            if d[X, Y] <= r_P:
                Pe[ef[X]:ef[X + 1], ef[Y]:ef[Y + 1]] = P[hf[a]:hf[a + 1], hf[b]:hf[b + 1]]
    return Pe


def rows_by_key(s, K_rows, ext):
    """{(home atom, shift): the (home nbf x nf) column block of that extended atom}."""
    nf = np.diff(s.atom_func_off)
    out, c = {}, 0
    for a, n1, n2, n3 in ext:
        out[(int(a), (int(n1), int(n2), int(n3)))] = K_rows[:, c:c + nf[a]]
        c += nf[a]
    assert c == K_rows.shape[1]
    return out


@pytest.mark.parametrize("A,n_atoms,r_ext", [(SKEW, 3, 5.0), (FCC, 2, 6.5), (np.diag([5.0, 7.0, 9.0]), 2, 8.0)])
def test_images_against_enumeration(A, n_atoms, r_ext):
    s = synth.periodic_cell(n_atoms, A, sub=11)
    got = oracle.periodic_images(s.atom_xyz, A, r_ext)
    assert len({tuple(map(int, r)) for r in got}) == len(got)  # no duplicates
    assert {tuple(map(int, r)) for r in got} == enumerate_images(s.atom_xyz, A, r_ext)
    assert [tuple(r) for r in got] == sorted(tuple(r) for r in got)  # atom by atom, shifts lexicographic
    assert len(got) > 0


CASES = [
    dict(kernel=oracle.KERNEL_COULOMB, screen=False, density_screen=False),
    dict(kernel=oracle.KERNEL_ERFC, screen=True, density_screen=True, tau=1e-8, eps=1e-8),
]


@pytest.mark.parametrize("opts", CASES, ids=["coulomb", "erfc-screened"])
@pytest.mark.parametrize("A,n_atoms,r_ext,r_P", [(SKEW, 2, 5.0, 4.0), (FCC, 2, 4.6, 4.5)], ids=["skew", "fcc"])
def test_lattice_sum_is_molecular_exchange_over_extended_set(opts, A, n_atoms, r_ext, r_P):
    s = synth.periodic_cell(n_atoms, A, sub=12, recipe=D_RECIPE)
    P = synth.periodic_density_matrix(s, cutoff=r_P, sub=12)
    K_rows, ext, n = oracle.K_periodic(s, P, A, r_ext, r_P, **opts)
    assert n > 0
    # independent extended set, images in shift-major order (the oracle's is atom-major)
    imgs = sorted(enumerate_images(s.atom_xyz, A, r_ext), key=lambda r: (r[1:], r[0]))
    e, atoms = extended_system(s, A, imgs)
    Pe = extended_density(s, e, atoms, P, r_P)
    Km, _ = oracle.build_K(e, Pe, **opts)
    nb = s.n_bf
    ef = e.atom_func_off
    got = rows_by_key(s, K_rows, ext)
    assert set(got) == {(a, n) for a, n in atoms}
    scale = np.abs(Km[:nb]).max()
    assert scale > 0
    for X, key in enumerate(atoms):
        np.testing.assert_allclose(got[key], Km[:nb, ef[X]:ef[X + 1]], rtol=0, atol=1e-12 * scale)


def test_no_images_reduces_to_molecular_exchange():
    s = synth.periodic_cell(3, np.eye(3) * 8.0, sub=13, recipe=D_RECIPE)
    far = np.eye(3) * 1000.0  # the same atoms in a huge cell: no image within reach
    P = synth.density_matrix(s, 4, cutoff=14.0, sub=13)
    K_rows, ext, _ = oracle.K_periodic(s, P, far, 10.0, 14.0, kernel=oracle.KERNEL_ERFC, screen=True,
                                       density_screen=True)
    assert ext.shape[0] == s.n_atoms and not ext[:, 1:].any()
    Km, _ = oracle.build_K(s, P, kernel=oracle.KERNEL_ERFC, screen=True, density_screen=True)
    np.testing.assert_allclose(K_rows, Km, rtol=0, atol=1e-13 * np.abs(Km).max())


def test_unimodular_change_of_lattice_vectors():
    s = synth.periodic_cell(2, SKEW, sub=14)
    B = np.array([[1, 0, 0], [1, 1, 0], [0, -1, 1]], dtype=np.float64) @ SKEW  # det 1: the same lattice
    P = synth.periodic_density_matrix(s, cutoff=4.0, sub=14)
    opts = dict(kernel=oracle.KERNEL_ERFC, screen=True, density_screen=True)
    Ka, ea, _ = oracle.K_periodic(s, P, SKEW, 5.0, 4.0, **opts)
    Kb, eb, _ = oracle.K_periodic(s, P, B, 5.0, 4.0, **opts)

    def by_position(K, ext, A):
        blocks = rows_by_key(s, K, ext)
        return {(a, tuple(np.round(s.atom_xyz[a] + np.array(n, dtype=np.float64) @ A, 9))): v
                for (a, n), v in blocks.items()}

    ga, gb = by_position(Ka, ea, SKEW), by_position(Kb, eb, B)
    assert set(ga) == set(gb)
    for k in ga:
        np.testing.assert_allclose(ga[k], gb[k], rtol=0, atol=1e-14 * np.abs(Ka).max())


def test_supercell_describes_the_same_crystal():
    """A cell and its doubled supercell (a1 -> 2 a1) with the density repeated
    in the same way: the cell's rows K^G_{mu lambda} for lambda near mu equal
    the supercell's rows of the same atoms, once both extended sets reach
    past the range of the (compact) shells."""
    A = np.diag([6.0, 6.5, 7.0])
    r_P, r_ext = 2.9, 8.0  # r_P below half the shortest vector: one image per pair
    s = synth.periodic_cell(2, A, sub=15, alpha_range=(3.0, 20.0))
    P = synth.periodic_density_matrix(s, cutoff=r_P, sub=15)
    # supercell: the two cells' atoms, lattice (2 a1, a2, a3)
    sup_atoms = [(a, (0, 0, 0)) for a in range(s.n_atoms)] + [(a, (1, 0, 0)) for a in range(s.n_atoms)]
    S2, _ = extended_system(s, A, [(a,) + n for a, n in sup_atoms[s.n_atoms:]])
    A2 = A.copy()
    A2[0] *= 2.0
    S2.lattice = A2
    # supercell home density: cell blocks where the supercell's minimum-image distance is within r_P
    hf, sf = s.atom_func_off, S2.atom_func_off
    dmin = synth.min_image_distances(S2)
    P2 = np.zeros((S2.n_bf, S2.n_bf))
    for X, (a, _) in enumerate(sup_atoms):
        for Y, (b, _) in enumerate(sup_atoms):
            if dmin[X, Y] <= r_P:
                P2[sf[X]:sf[X + 1], sf[Y]:sf[Y + 1]] = P[hf[a]:hf[a + 1], hf[b]:hf[b + 1]]
    opts = dict(kernel=oracle.KERNEL_ERFC, screen=True, tau=1e-14, density_screen=False)
    K1, e1, _ = oracle.K_periodic(s, P, A, r_ext, r_P, **opts)
    K2, e2, _ = oracle.K_periodic(S2, P2, A2, r_ext, r_P, **opts)
    pos = lambda sysobj, Amat, a, n: tuple(np.round(sysobj.atom_xyz[a] + np.array(n, float) @ Amat, 9))
    b1 = {pos(s, A, a, n): v for (a, n), v in rows_by_key(s, K1, e1).items()}
    b2 = {pos(S2, A2, a, n): v for (a, n), v in rows_by_key(S2, K2, e2).items()}
    nb = s.n_bf
    compared = 0
    for p, v in b1.items():
        near = np.linalg.norm(np.array(p)[None, :] - s.atom_xyz, axis=1).min() <= 5.0
        if not near:
            continue
        assert p in b2
        # rows of the cell's own atoms: the first nb rows of the supercell
        np.testing.assert_allclose(v, b2[p][:nb], rtol=0, atol=1e-12 * np.abs(K1).max())
        compared += 1
    assert compared >= s.n_atoms + 2


def test_per_cell_energy_converges_in_r_ext():
    """Truncation of the image set: the home rows K^G_{mu lambda} need the
    images sigma^H within the overlap range of every lambda^G in the density
    pattern (at most r_P from the home cell), so the per-cell exchange energy
    is converged once r_ext exceeds r_P by the overlap range.  With r_P = 4 bohr
    on a small skewed cell (s and p shells): r_ext = r_P + 4 and r_P + 6 agree to
    1e-8 of E_x, while r_ext = r_P + 2 still misses a part well above that."""
    from periodic_helpers import oracle_rows_by_key
    s = synth.periodic_cell(2, SKEW, sub=41, recipe={"C": [0, 1], "H": [0, 1]})
    P = synth.periodic_density_matrix(s, cutoff=4.0, sub=41)
    kw = dict(kernel=oracle.KERNEL_ERFC, screen=True, density_screen=True, tau=1e-10, eps=1e-10)
    E = {rx: oracle_rows_by_key(s, P, SKEW, rx, 4.0, **kw)[1] for rx in (6.0, 8.0, 10.0)}
    assert abs(E[10.0] - E[8.0]) <= 1e-8 * abs(E[10.0])
    assert abs(E[10.0] - E[6.0]) > 1e-6 * abs(E[10.0])
