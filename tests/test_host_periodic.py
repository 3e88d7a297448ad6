"""Host side of the library's periodic path (CPU, no GPU): the image table
(hfx_periodic_images), the extended shell set and pattern, and the
real-space density laid onto the extended pattern (hfx_periodic_pack_host).

The library's extended set, fed to the CPU oracle's molecular exchange,
must reproduce the oracle's own periodic rows (Eq. H-HFX summed by brute force
over the oracle's independently built image set), so every host step the GPU
path takes before hfx_build_K is checked here; the GPU test then only swaps
the oracle's molecular exchange for hfx_build_K.
"""
import numpy as np
import pytest

import oracle
import synth
from periodic_helpers import extended_system, formed_blocks_error

SKEW = np.array([[6.0, 0.0, 0.0], [1.0, 6.0, 0.0], [0.0, 1.0, 6.0]])
FCC = 7.0 * np.array([[0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
D_RECIPE = {"C": [0, 1, 2], "H": [0, 1]}


@pytest.fixture(scope="module")
def hfx():
    from paper_2009_03555_gb300 import hfx as h
    try:
        h.load()
    except ImportError as e:  # the library is built by __graft_entry__.build()
        pytest.skip(str(e))
    return h


def unpack(sysobj, mask, val):
    """Dense matrix from pattern values (blocks in CSR order, row-major)."""
    fo = sysobj.atom_func_off
    out = np.zeros((sysobj.n_bf, sysobj.n_bf))
    v = 0
    for X in range(sysobj.n_atoms):
        for Y in np.flatnonzero(mask[X]):
            n = (fo[X + 1] - fo[X]) * (fo[Y + 1] - fo[Y])
            out[fo[X]:fo[X + 1], fo[Y]:fo[Y + 1]] = val[v:v + n].reshape(fo[X + 1] - fo[X], fo[Y + 1] - fo[Y])
            v += n
    assert v == len(val)
    return out


@pytest.mark.parametrize("A,n_atoms,r_ext", [(SKEW, 3, 5.0), (FCC, 2, 6.5), (np.diag([5.0, 7.0, 9.0]), 2, 8.0),
                                             (np.eye(3) * 100.0, 3, 10.0)])
def test_image_table_matches_oracle(hfx, A, n_atoms, r_ext):
    s = synth.periodic_cell(n_atoms, A, sub=21)
    atom, shift = hfx.hfx_periodic_images(s.atom_xyz, A, r_ext)
    ref = oracle.periodic_images(s.atom_xyz, A, r_ext)
    got = [(int(a),) + tuple(int(x) for x in n) for a, n in zip(atom, shift)]
    assert len(set(got)) == len(got)
    assert set(got) == {tuple(int(x) for x in r) for r in ref}
    assert [g[1:] + g[:1] for g in got] == sorted(g[1:] + g[:1] for g in got)  # by shift, then atom


def test_image_table_si216(hfx):
    s = synth.si_supercell()
    atom, shift = hfx.hfx_periodic_images(s.atom_xyz, s.lattice, 10.0)
    # every image lies within 10 bohr of a home atom and outside the home cell
    pos = s.atom_xyz[atom] + shift @ s.lattice
    d = np.linalg.norm(pos[:, None, :] - s.atom_xyz[None, :, :], axis=-1).min(axis=1)
    assert np.all(d <= 10.0) and np.all(np.any(shift != 0, axis=1))
    # r_ext is below the 30.78-bohr cell side: only the 26 neighbouring cells can hold images
    want = set()
    for n in np.array(np.meshgrid([-1, 0, 1], [-1, 0, 1], [-1, 0, 1])).T.reshape(-1, 3):
        if not n.any():
            continue
        p = s.atom_xyz + n @ s.lattice
        dd = np.linalg.norm(p[:, None, :] - s.atom_xyz[None, :, :], axis=-1).min(axis=1)
        want |= {(int(a),) + tuple(int(x) for x in n) for a in np.flatnonzero(dd <= 10.0)}
    assert {(int(a),) + tuple(int(x) for x in n) for a, n in zip(atom, shift)} == want
    assert len(atom) == len(want) == 430


def test_image_table_rejects_bad_input(hfx):
    x = np.zeros((1, 3))
    with pytest.raises(hfx.HFXError, match="singular"):
        hfx.hfx_periodic_images(x, np.array([[1.0, 0, 0], [2.0, 0, 0], [0, 0, 1.0]]), 3.0)
    with pytest.raises(hfx.HFXError, match="r_ext"):
        hfx.hfx_periodic_images(x, np.eye(3) * 5.0, -1.0)


CASES = [
    dict(kernel=oracle.KERNEL_COULOMB, screen=False, density_screen=False),
    dict(kernel=oracle.KERNEL_ERFC, screen=True, density_screen=True, tau=1e-8, eps=1e-8),
]


@pytest.mark.parametrize("opts", CASES, ids=["coulomb", "erfc-screened"])
@pytest.mark.parametrize("A,n_atoms,r_ext,r_P", [(SKEW, 2, 5.0, 4.0), (FCC, 2, 4.6, 4.5)], ids=["skew", "fcc"])
def test_extended_set_and_density_reproduce_oracle_rows(hfx, opts, A, n_atoms, r_ext, r_P):
    s = synth.periodic_cell(n_atoms, A, sub=22, recipe=D_RECIPE)
    P = synth.periodic_density_matrix(s, cutoff=r_P, sub=22)
    per = hfx.Periodic(s, A, r_ext=r_ext, r_P=r_P)
    e = extended_system(per)
    assert per.n_home_bf == s.n_bf and e.n_atoms == len(per.ext_home) == per.system.n_atoms
    np.testing.assert_array_equal(e.atom_func_off, per.system.atom_func_off)
    assert e.n_shells == per.system.n_shells and e.n_bf == per.system.n_bf
    # the library's extended coordinates and density pattern
    np.testing.assert_allclose(per.system.atom_xyz, s.atom_xyz[per.ext_home] + per.ext_shift @ A, rtol=0, atol=1e-12)
    d = np.linalg.norm(e.atom_xyz[:, None, :] - e.atom_xyz[None, :, :], axis=-1)
    np.testing.assert_array_equal(per.mask, d <= r_P)
    Pv = per.pack(P)
    Pe = unpack(e, per.mask, Pv)
    np.testing.assert_array_equal(Pe, Pe.T)
    Km, _ = oracle.build_K(e, Pe, **opts)
    Kref, ext, _ = oracle.K_periodic(s, P, A, r_ext, r_P, **opts)
    nf = np.diff(s.atom_func_off)
    ef = e.atom_func_off
    col = {}
    c = 0
    for a, n1, n2, n3 in ext:
        col[(int(a), (int(n1), int(n2), int(n3)))] = (c, c + nf[a])
        c += nf[a]
    keys = [(int(h), tuple(int(x) for x in n)) for h, n in zip(per.ext_home, per.ext_shift)]
    assert set(keys) == set(col)
    scale = np.abs(Kref).max()
    for X, k in enumerate(keys):
        c0, c1 = col[k]
        np.testing.assert_allclose(Km[:s.n_bf, ef[X]:ef[X + 1]], Kref[:, c0:c1], rtol=0, atol=1e-12 * scale)
    # what the GPU test sees: K kept on the pattern only (the library forms no
    # other block), compared on the formed blocks with zeros required elsewhere
    Kv = hfx._SystemInput(e, per.mask).pack(Km)
    assert len(Kv) == per.n_values
    Kpat = unpack(e, per.mask, Kv)[:s.n_bf]
    ref = {k: Kref[:, col[k][0]:col[k][1]] for k in keys}
    err, outside, n_formed = formed_blocks_error(Kpat, per, ref, s.atom_func_off)
    assert n_formed > s.n_atoms
    assert err <= 1e-12 * scale and outside == 0.0
    # per-cell exchange energy from the value prefix of the home rows
    E_prefix = -0.5 * float(np.dot(Pv[:per.n_home_values], Kv[:per.n_home_values]))
    E_rows = -0.5 * float(np.sum(Pe[:s.n_bf] * Km[:s.n_bf]))
    assert abs(E_prefix - E_rows) <= 1e-13 * abs(E_rows)


def test_pack_rejects_bad_home_index(hfx):
    s = synth.periodic_cell(2, SKEW, sub=23)
    per = hfx.Periodic(s, SKEW, r_ext=5.0, r_P=4.0)
    per.ext_home = per.ext_home.copy()
    per.ext_home[-1] = s.n_atoms  # out of range
    with pytest.raises(hfx.HFXError, match="ext_home"):
        per.pack(synth.periodic_density_matrix(s, cutoff=4.0, sub=23))


def test_lattice_density_pack(hfx):
    """hfx_periodic_pack_lattice_host: one P^L per shift difference equal to
    P_home gives the Gamma-point pack; a two-point k grid gives the blocks of
    the definition P^{n_Y - n_X}(home X, home Y), zero where a shift is not
    listed."""
    from periodic_helpers import extended_density, kgrid_lattice_density, shift_differences
    s = synth.periodic_cell(2, SKEW, sub=24, recipe=D_RECIPE)
    P = synth.periodic_density_matrix(s, cutoff=4.0, sub=24)
    per = hfx.Periodic(s, SKEW, r_ext=5.0, r_P=4.0)
    L = shift_differences(per)
    assert len(L) > 1
    np.testing.assert_array_equal(per.pack_lattice(L, np.stack([P] * len(L))), per.pack(P))
    P0 = synth.periodic_density_matrix(s, cutoff=4.0, sub=25)
    Ppi = synth.periodic_density_matrix(s, cutoff=4.0, sub=26)
    Lk, PL = kgrid_lattice_density(P0, Ppi, L)
    v = per.pack_lattice(Lk, PL)
    Pe = extended_density(per, lambda n: 0.5 * (P0 + np.cos(np.pi * n[0]) * Ppi), 4.0)
    ref = hfx._SystemInput(extended_system(per), per.mask).pack(Pe)
    np.testing.assert_array_equal(v, ref)
    # a shift left out of the list gives zero blocks
    keep = np.any(Lk != Lk[0], axis=1)
    v2 = per.pack_lattice(Lk[keep], PL[keep])
    assert np.count_nonzero(v2) < np.count_nonzero(v)
