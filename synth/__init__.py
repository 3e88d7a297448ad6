"""Seeded synthetic inputs for the HFX hot path (geometry, shells, density matrix).

This module is shared by the CUDA path's tests/benchmark and by the CPU oracle's
tests.  It holds none of the method's arithmetic: no normalisation, no
integrals, no screening.  It only draws numbers: atom positions, raw (not
normalised) contraction coefficients, exponents and a density matrix
P = C C^T built from random orthonormal columns.

The paper's own workloads (DNA, TiO2 surface, Si supercells; Table 1) need its
numerical-atomic-orbital basis and pseudopotentials, which are not available.
These generators stand in for them with synthetic Gaussian shells on molecules
and 1D/2D/3D solids of the same kinds (Sec. 4).

Draw order (fixed, part of the recipe):
  1. geometry (positions, then jitter),
  2. shells, atom by atom in atom order, shell by shell: exponents then
     coefficients,
  3. the density matrix, from its own seed stream (so P can be redrawn).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 2009_03555

#: nuclear charge per element symbol used by the generators
ZNUC = {"H": 1, "C": 6, "O": 8, "Si": 14}


def ncart(l: int) -> int:
    """Number of Cartesian components of a shell of angular momentum l."""
    return (l + 1) * (l + 2) // 2


@dataclasses.dataclass
class System:
    """A molecule or a periodic cell's home atoms plus (optionally) images.

    Shells are stored atom-major so that every atom's functions are
    contiguous.  ``coef`` holds raw contraction coefficients; normalising
    them is the job of whoever consumes the system.
    """

    name: str
    atom_Z: np.ndarray  # (n_atoms,) int32
    atom_xyz: np.ndarray  # (n_atoms, 3) float64, bohr
    shell_atom: np.ndarray  # (n_shells,) int32
    shell_l: np.ndarray  # (n_shells,) int32
    prim_off: np.ndarray  # (n_shells + 1,) int32 into alpha/coef
    alpha: np.ndarray  # (n_prims,) float64, bohr^-2
    coef: np.ndarray  # (n_prims,) float64, raw
    lattice: np.ndarray | None = None  # (3, 3) lattice vectors as rows (bohr); None = molecule

    @property
    def n_atoms(self) -> int:
        return int(self.atom_xyz.shape[0])

    @property
    def n_shells(self) -> int:
        return int(self.shell_l.shape[0])

    @property
    def shell_nprim(self) -> np.ndarray:
        return np.diff(self.prim_off).astype(np.int32)

    @property
    def shell_nfunc(self) -> np.ndarray:
        return np.array([ncart(int(l)) for l in self.shell_l], dtype=np.int32)

    @property
    def func_off(self) -> np.ndarray:
        """(n_shells + 1,) first Cartesian function of each shell."""
        return np.concatenate([[0], np.cumsum(self.shell_nfunc)]).astype(np.int64)

    @property
    def n_bf(self) -> int:
        return int(self.shell_nfunc.sum())

    @property
    def atom_func_off(self) -> np.ndarray:
        """(n_atoms + 1,) first function of each atom (shells are atom-major)."""
        off = np.zeros(self.n_atoms + 1, dtype=np.int64)
        nf = self.shell_nfunc
        for s in range(self.n_shells):
            off[self.shell_atom[s] + 1] += nf[s]
        return np.cumsum(off)

    @property
    def n_occ(self) -> int:
        """Half the number of electrons (all-electron count)."""
        return int(self.atom_Z.sum()) // 2

    def translated(self, shift) -> "System":
        s = dataclasses.replace(self)
        s.atom_xyz = self.atom_xyz + np.asarray(shift, dtype=np.float64)[None, :]
        return s


def _rng(config_idx: int, stream: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([BASE_SEED, config_idx, stream]))


def _draw_shells(rng, elements, recipe, nprim, alpha_lo=0.1, alpha_hi=50.0):
    """recipe: element -> list of l values (one entry per shell)."""
    shell_atom, shell_l, alpha, coef, off = [], [], [], [], [0]
    lo, hi = math.log(alpha_lo), math.log(alpha_hi)
    for ia, el in enumerate(elements):
        for l in recipe[el]:
            a = np.sort(np.exp(rng.uniform(lo, hi, size=nprim)))[::-1]
            # U(0.1, 1]: 1 - U[0,1) lies in (0, 1]
            c = 0.1 + 0.9 * (1.0 - rng.uniform(0.0, 1.0, size=nprim))
            shell_atom.append(ia)
            shell_l.append(l)
            alpha.extend(a.tolist())
            coef.extend(c.tolist())
            off.append(off[-1] + nprim)
    return (np.array(shell_atom, dtype=np.int32), np.array(shell_l, dtype=np.int32),
            np.array(off, dtype=np.int32), np.array(alpha, dtype=np.float64),
            np.array(coef, dtype=np.float64))


def _make(name, elements, xyz, recipe, nprim, rng, alpha_range=(0.1, 50.0)) -> System:
    sa, sl, off, a, c = _draw_shells(rng, elements, recipe, nprim, *alpha_range)
    return System(name=name, atom_Z=np.array([ZNUC[e] for e in elements], dtype=np.int32),
                  atom_xyz=np.ascontiguousarray(xyz, dtype=np.float64), shell_atom=sa,
                  shell_l=sl, prim_off=off, alpha=a, coef=c)


# -- shell recipes ---------------------------------------------------------------
WATER_RECIPE = {"O": [0, 0, 0, 1, 1], "H": [0, 0, 1]}  # O: 3s+2p, H: 2s+1p
CH_RECIPE = {"C": [0, 0, 1, 1, 2], "H": [0, 0, 1, 1, 2]}  # 2s+2p+1d per atom
SI_RECIPE = {"Si": [0, 0, 0, 1, 1, 1, 2]}  # 3s+3p+1d


def water_dimer(config_idx: int = 0) -> System:
    """Two water-like molecules: O-H 1.81 bohr, H-O-H 104.5 deg, O-O 5.5 bohr,
    every coordinate jittered by U(-0.1, 0.1); 3 primitives per shell."""
    rng = _rng(config_idx, 0)
    half = math.radians(104.5 / 2.0)
    xyz, el = [], []
    for ox in (0.0, 5.5):
        xyz.append([ox, 0.0, 0.0]); el.append("O")
        for sgn in (+1.0, -1.0):
            xyz.append([ox + 1.81 * math.cos(half), sgn * 1.81 * math.sin(half), 0.0]); el.append("H")
    xyz = np.array(xyz) + rng.uniform(-0.1, 0.1, size=(len(el), 3))
    return _make("water_dimer", el, xyz, WATER_RECIPE, 3, rng)


def ch_cluster(n_atoms: int, config_idx: int = 2, sub: int = 0, min_dist: float = 2.2,
               box: float | None = None, nprim: int = 4) -> System:
    """C/H molecular cluster by random sequential addition in a cubic box of side
    30*(N/400)^(1/3) bohr (the 400-atom, 30-bohr density), minimum spacing
    ``min_dist``; elements alternate C, H, C, H, ...; 2s+2p+1d shells."""
    rng = _rng(config_idx, 1000 + sub)
    L = box if box is not None else 30.0 * (n_atoms / 400.0) ** (1.0 / 3.0)
    pts = np.zeros((0, 3))
    tries = 0
    while pts.shape[0] < n_atoms:
        cand = rng.uniform(0.0, L, size=3)
        tries += 1
        if tries > 2_000_000:
            raise RuntimeError("random sequential addition did not converge")
        if pts.shape[0] and np.min(np.sum((pts - cand) ** 2, axis=1)) < min_dist ** 2:
            continue
        pts = np.vstack([pts, cand])
    el = ["C" if i % 2 == 0 else "H" for i in range(n_atoms)]
    return _make(f"ch_cluster_{n_atoms}", el, pts, CH_RECIPE, nprim, rng)


def ch_chain(n_atoms: int, config_idx: int = 4, sub: int = 0, spacing: float = 2.8) -> System:
    """1D C/H chain along x, spacing 2.8 bohr, 0.1 bohr jitter."""
    rng = _rng(config_idx, 2000 + sub)
    xyz = np.zeros((n_atoms, 3))
    xyz[:, 0] = spacing * np.arange(n_atoms)
    xyz += rng.uniform(-0.1, 0.1, size=xyz.shape)
    el = ["C" if i % 2 == 0 else "H" for i in range(n_atoms)]
    return _make(f"ch_chain_{n_atoms}", el, xyz, CH_RECIPE, 4, rng)


def ch_slab(n_atoms: int, config_idx: int = 4, sub: int = 0, spacing: float = 4.0) -> System:
    """2D C/H square-lattice slab (4.0 bohr), filled row by row, 0.1 bohr jitter."""
    rng = _rng(config_idx, 3000 + sub)
    side = int(math.ceil(math.sqrt(n_atoms)))
    idx = np.arange(n_atoms)
    xyz = np.zeros((n_atoms, 3))
    xyz[:, 0] = spacing * (idx % side)
    xyz[:, 1] = spacing * (idx // side)
    xyz += rng.uniform(-0.1, 0.1, size=xyz.shape)
    el = ["C" if i % 2 == 0 else "H" for i in range(n_atoms)]
    return _make(f"ch_slab_{n_atoms}", el, xyz, CH_RECIPE, 4, rng)


def si_supercell(ncell: int = 3, config_idx: int = 4, sub: int = 0, a: float = 10.26, nprim: int = 4) -> System:
    """Silicon in the diamond structure: ncell^3 conventional cubic cells of side
    ``a`` bohr (8 atoms each; 3x3x3 = 216 atoms), atoms on the exact lattice
    sites (no jitter), 3s+3p+1d shells with ``nprim`` primitives drawn per atom
    like the other recipes.  ``lattice`` is the supercell (ncell a on each axis)."""
    rng = _rng(config_idx, 4000 + sub)
    fcc = np.array([[0, 0, 0], [0, 0.5, 0.5], [0.5, 0, 0.5], [0.5, 0.5, 0]])
    basis = np.vstack([fcc, fcc + 0.25])
    cells = np.array([[i, j, k] for i in range(ncell) for j in range(ncell) for k in range(ncell)], dtype=np.float64)
    xyz = a * (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3)
    s = _make(f"si_{len(xyz)}", ["Si"] * len(xyz), xyz, SI_RECIPE, nprim, rng)
    s.lattice = np.eye(3) * (ncell * a)
    return s


#: a light shell recipe (one s and one p shell per atom) for small periodic cells
LIGHT_RECIPE = {"C": [0, 1], "H": [0, 1], "Si": [0, 1, 2]}


def periodic_cell(n_atoms: int, lattice, config_idx: int = 4, sub: int = 0, min_dist: float = 2.0,
                  recipe: dict | None = None, nprim: int = 2, alpha_range=(0.1, 50.0)) -> System:
    """A small periodic cell for tests: ``n_atoms`` atoms (C, H alternating)
    at uniform random fractional coordinates, at least ``min_dist`` bohr from
    each other and from each other's images; shells from ``recipe``
    (default LIGHT_RECIPE), exponents log-uniform in ``alpha_range``."""
    rng = _rng(config_idx, 6000 + sub)
    A = np.asarray(lattice, dtype=np.float64).reshape(3, 3)
    shifts = np.array([[i, j, k] for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)], dtype=np.float64) @ A
    if np.linalg.norm(shifts[np.any(shifts != 0, axis=1)], axis=1).min() < min_dist:
        raise ValueError("lattice vectors shorter than min_dist")
    pts = np.zeros((0, 3))
    tries = 0
    while pts.shape[0] < n_atoms:
        tries += 1
        if tries > 100_000:
            raise RuntimeError("cell too small for the requested atoms")
        cand = rng.uniform(0.0, 1.0, size=3) @ A
        if pts.shape[0]:
            d = np.linalg.norm(pts[:, None, :] + shifts[None, :, :] - cand[None, None, :], axis=-1)
            if d.min() < min_dist:
                continue
        pts = np.vstack([pts, cand])
    el = ["C" if i % 2 == 0 else "H" for i in range(n_atoms)]
    s = _make(f"cell_{n_atoms}", el, pts, recipe or LIGHT_RECIPE, nprim, rng, alpha_range)
    s.lattice = A.copy()
    return s


def min_image_distances(sys: System) -> np.ndarray:
    """(n_atoms, n_atoms) distance from atom a to the nearest periodic image of
    atom b (plain distances for a molecule)."""
    if sys.lattice is None:
        return atom_distances(sys)
    A = np.asarray(sys.lattice, dtype=np.float64)
    x = sys.atom_xyz
    diam = atom_distances(sys).max()
    # a minimum image is no farther than the direct distance, so its lattice
    # vector L has |L| <= 2 * diam and |n_i| <= 2 * diam / h_i (h_i: cell heights)
    h = abs(np.linalg.det(A)) / np.linalg.norm(np.cross(A[[1, 2, 0]], A[[2, 0, 1]]), axis=1)
    m = np.ceil(2.0 * diam / h).astype(int)
    best = np.full((sys.n_atoms, sys.n_atoms), np.inf)
    for n1 in range(-m[0], m[0] + 1):
        for n2 in range(-m[1], m[1] + 1):
            for n3 in range(-m[2], m[2] + 1):
                L = np.array([n1, n2, n3], dtype=np.float64) @ A
                d = np.linalg.norm(x[:, None, :] - x[None, :, :] - L[None, None, :], axis=-1)
                np.minimum(best, d, out=best)
    return best


def periodic_density_matrix(sys: System, config_idx: int = 4, cutoff: float | None = 14.0, sub: int = 0,
                            n_occ: int | None = None) -> np.ndarray:
    """Home-cell density matrix of a periodic system: P = C C^T as in
    ``density_matrix``, with every atom-pair block whose minimum-image
    distance exceeds ``cutoff`` set to zero."""
    P = density_matrix(sys, config_idx, n_occ=n_occ, sub=sub)
    if cutoff is not None:
        P = P * expand_atom_mask(sys, min_image_distances(sys) <= cutoff)
    return np.ascontiguousarray(P)


def shell_subset(sys: System, P: np.ndarray, keep_l) -> tuple[System, np.ndarray]:
    """The shells of ``sys`` whose angular momentum is in ``keep_l`` (same atoms
    and centres, shells in the original order) and the matching rows and
    columns of the density matrix ``P``.  Used to isolate one angular-momentum
    class of quartets (e.g. only d shells: every quartet is (dd|dd))."""
    keep = [S for S in range(sys.n_shells) if int(sys.shell_l[S]) in set(keep_l)]
    po = sys.prim_off
    take = np.concatenate([np.arange(po[S], po[S + 1]) for S in keep])
    n_p = np.array([po[S + 1] - po[S] for S in keep])
    sub = System(name=sys.name + "_l" + "".join(str(l) for l in sorted(set(keep_l))), atom_Z=sys.atom_Z.copy(),
                 atom_xyz=sys.atom_xyz.copy(), shell_atom=sys.shell_atom[keep].astype(np.int32),
                 shell_l=sys.shell_l[keep].astype(np.int32),
                 prim_off=np.concatenate([[0], np.cumsum(n_p)]).astype(np.int32),
                 alpha=sys.alpha[take].copy(), coef=sys.coef[take].copy(),
                 lattice=None if sys.lattice is None else sys.lattice.copy())
    fo = sys.func_off
    f = np.concatenate([np.arange(fo[S], fo[S + 1]) for S in keep])
    return sub, np.ascontiguousarray(P[np.ix_(f, f)])


def atom_distances(sys: System) -> np.ndarray:
    d = sys.atom_xyz[:, None, :] - sys.atom_xyz[None, :, :]
    return np.sqrt(np.sum(d * d, axis=-1))


def density_matrix(sys: System, config_idx: int, n_occ: int | None = None,
                   cutoff: float | None = None, sub: int = 0) -> np.ndarray:
    """Dense symmetric P = C C^T, C the Q factor of a seeded n_bf x n_occ Gaussian
    matrix (Euclidean-orthonormal columns).  If ``cutoff`` is given, every
    atom-pair block whose atoms are farther apart than ``cutoff`` bohr is set
    to zero."""
    rng = _rng(config_idx, 5000 + sub)
    nbf = sys.n_bf
    nocc = sys.n_occ if n_occ is None else n_occ
    nocc = min(nocc, nbf)
    G = rng.standard_normal((nbf, nocc))
    C, _ = np.linalg.qr(G)
    P = C @ C.T
    P = 0.5 * (P + P.T)
    if cutoff is not None:
        mask = atom_pair_mask(sys, cutoff)
        P = P * expand_atom_mask(sys, mask)
    return np.ascontiguousarray(P)


def atom_pair_mask(sys: System, cutoff: float) -> np.ndarray:
    """(n_atoms, n_atoms) bool: atom pairs within ``cutoff`` bohr."""
    return atom_distances(sys) <= cutoff


def expand_atom_mask(sys: System, mask: np.ndarray) -> np.ndarray:
    """Expand an atom-pair mask to a dense (n_bf, n_bf) 0/1 float matrix."""
    fo = sys.atom_func_off
    atom_of_func = np.repeat(np.arange(sys.n_atoms), np.diff(fo))
    return mask[atom_of_func[:, None], atom_of_func[None, :]].astype(np.float64)


def perturb_density(P: np.ndarray, rng: np.random.Generator, rel: float = 1e-3) -> np.ndarray:
    """P <- P o (1 + rel * xi), xi symmetric standard normal; the pattern is kept."""
    xi = rng.standard_normal(P.shape)
    xi = 0.5 * (xi + xi.T) * math.sqrt(2.0)
    return np.ascontiguousarray(P * (1.0 + rel * xi))


def config0():
    """Two water-like molecules, dense P with 10 occupied columns."""
    s = water_dimer(0)
    return s, density_matrix(s, 0, n_occ=10)


def config2(n_atoms: int = 400, sub: int = 0):
    """C/H cluster (400 atoms by default), P cut at 14 bohr."""
    s = ch_cluster(n_atoms, 2, sub=sub)
    return s, density_matrix(s, 2, cutoff=14.0, sub=sub)
