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
