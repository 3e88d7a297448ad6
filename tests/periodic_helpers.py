"""Comparison of periodic exchange rows on the blocks the library forms.

The library forms K only on the sparsity pattern of P (atom-pair blocks, the
paper's one sparse format for the density and exchange matrices, Sec. 3 and
Table 1).  For a periodic cell that pattern is every pair of extended atoms at
most r_P apart, so of the home rows K^G_{mu lambda} (Sec. 2, Eq. H-HFX) only the
blocks (home atom h, extended atom X) with |R_h - R_X| <= r_P are formed; the
rest come back as zeros.  The oracle's brute-force rows cover every extended
column, so both the GPU test and its CPU stand-in compare exactly the formed
blocks and require zeros elsewhere.
"""
import numpy as np


def formed_blocks_error(K_rows, per, ref_blocks, home_func_off):
    """Largest |K - K_ref| over the formed blocks, and the largest |K| outside them.

    K_rows: home nbf x extended nbf (library column order); per: the
    ``hfx.Periodic`` whose pattern the build used; ref_blocks: oracle rows keyed
    by (home atom, shift) as (home nbf x nf) arrays; home_func_off: function
    offsets of the home atoms."""
    ef = per.system.atom_func_off
    hf = home_func_off
    n_home = len(hf) - 1
    keys = [(int(h), tuple(int(x) for x in n)) for h, n in zip(per.ext_home, per.ext_shift)]
    err, outside, n_formed = 0.0, 0.0, 0
    for X, k in enumerate(keys):
        cols = slice(ef[X], ef[X + 1])
        for h in range(n_home):
            rows = slice(hf[h], hf[h + 1])
            if per.mask[h, X]:
                err = max(err, float(np.abs(K_rows[rows, cols] - ref_blocks[k][rows]).max()))
                n_formed += 1
            else:
                outside = max(outside, float(np.abs(K_rows[rows, cols]).max()))
    return err, outside, n_formed


def extended_system(per):
    """The extended atom set of a ``hfx.Periodic`` as a plain molecular system
    (every extended atom with its home atom's shells at its own centre), built
    from the library's ext_home and extended coordinates; lets the oracle's
    molecular exchange, or the library's molecular path, run on the same set."""
    import synth
    home = per.home
    sa = np.asarray(home.shell_atom)
    s0 = np.searchsorted(sa, np.arange(home.n_atoms + 1))
    src = np.concatenate([np.arange(s0[h], s0[h + 1]) for h in per.ext_home])
    po = np.asarray(home.prim_off)
    n_p = (po[1:] - po[:-1])[src]
    take = np.concatenate([np.arange(po[S], po[S + 1]) for S in src])
    return synth.System(name=home.name + "_ext", atom_Z=np.asarray(home.atom_Z)[per.ext_home],
                        atom_xyz=np.ascontiguousarray(per.system.atom_xyz),
                        shell_atom=np.repeat(np.arange(len(per.ext_home), dtype=np.int32), np.diff(s0)[per.ext_home]),
                        shell_l=np.asarray(home.shell_l, dtype=np.int32)[src],
                        prim_off=np.concatenate([[0], np.cumsum(n_p)]).astype(np.int32),
                        alpha=np.asarray(home.alpha, dtype=np.float64)[take],
                        coef=np.asarray(home.coef, dtype=np.float64)[take])


def oracle_rows_by_key(s, P, A, r_ext, r_P, **kw):
    """Oracle rows keyed by extended atom (home atom, shift), and the per-cell
    energy -1/2 sum P^G_{mu lambda} K^G_{mu lambda} over those rows."""
    import oracle
    K, ext, _ = oracle.K_periodic(s, P, A, r_ext, r_P, **kw)
    nf = np.diff(s.atom_func_off)
    hf = s.atom_func_off
    blocks, E, c = {}, 0.0, 0
    for a, n1, n2, n3 in ext:
        key = (int(a), (int(n1), int(n2), int(n3)))
        blk = K[:, c:c + nf[a]]
        blocks[key] = blk
        pos = s.atom_xyz[a] + np.array([n1, n2, n3], dtype=np.float64) @ A
        for b in range(s.n_atoms):  # P^G rows: home block where the atoms are within r_P
            if np.linalg.norm(s.atom_xyz[b] - pos) <= r_P:
                E += -0.5 * float(np.sum(P[hf[b]:hf[b + 1], hf[a]:hf[a + 1]] * blk[hf[b]:hf[b + 1]]))
        c += nf[a]
    return blocks, E


def kgrid_lattice_density(P0, Ppi, shifts):
    """Real-space densities of a two-point k grid along the first lattice
    vector, k in {0, pi}: P^L = (P(0) + cos(pi n1) P(pi)) / 2 for each lattice
    shift L = (n1, n2, n3) (Eq. dm as a Fourier sum over the grid).  Returns the
    distinct shifts (n_L x 3) and the stacked P^L."""
    L = np.unique(np.asarray(shifts, dtype=np.int32).reshape(-1, 3), axis=0)
    PL = np.stack([0.5 * (P0 + np.cos(np.pi * n[0]) * Ppi) for n in L])
    return L, PL


def extended_density(per, P_of_shift, r_P):
    """Dense density of the extended set from the definition: block (X, Y) is
    P^{n_Y - n_X}(home X, home Y) where the atoms are at most r_P apart."""
    ef = per.system.atom_func_off
    hf = per.home.atom_func_off
    x = per.system.atom_xyz
    Pe = np.zeros((per.system.n_bf, per.system.n_bf))
    for X in range(per.system.n_atoms):
        for Y in range(per.system.n_atoms):
            if np.linalg.norm(x[X] - x[Y]) > r_P:
                continue
            hx, hy = per.ext_home[X], per.ext_home[Y]
            PL = P_of_shift(tuple(int(v) for v in per.ext_shift[Y] - per.ext_shift[X]))
            Pe[ef[X]:ef[X + 1], ef[Y]:ef[Y + 1]] = PL[hf[hx]:hf[hx + 1], hf[hy]:hf[hy + 1]]
    return Pe


def shift_differences(per):
    """Every lattice-shift difference n_Y - n_X over the pattern's blocks."""
    out = set()
    for X in range(len(per.ext_home)):
        for Y in per.col[per.row_ptr[X]:per.row_ptr[X + 1]]:
            out.add(tuple(int(v) for v in per.ext_shift[Y] - per.ext_shift[X]))
    return np.array(sorted(out), dtype=np.int32)
