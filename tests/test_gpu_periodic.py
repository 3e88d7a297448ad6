"""GPU parity of periodic systems: the exchange rows K^G_{mu lambda} of the
home cell (Sec. 2, Eq. H-HFX) built by the CUDA path on the library's extended
atom set (hfx_create_basis_periodic, hfx_distance_pattern,
hfx_periodic_pack_host, then hfx_build_K with only the quartets that have a
home-cell shell), against the oracle's brute-force lattice sum over its own
image set.

The library forms K on the pattern of P only (the pairs of extended atoms at
most r_P apart), so the rows are compared on those blocks and must be zero on
the others (periodic_helpers.formed_blocks_error).  Tolerances as for
molecules: FP64 |dK|max <= 1e-10 and per-cell |dE_x| <= 1e-9 |E_x|; mixed
precision |dE_x| <= 1e-6 Ha.
"""
import numpy as np
import pytest

import oracle
import synth
from periodic_helpers import extended_system, formed_blocks_error, oracle_rows_by_key

pytestmark = pytest.mark.gpu

SKEW = np.array([[6.0, 0.0, 0.0], [1.0, 6.0, 0.0], [0.0, 1.0, 6.0]])
FCC = 7.0 * np.array([[0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
D_RECIPE = {"C": [0, 1, 2], "H": [0, 1]}


def gpu_periodic(s, P, A, r_ext, r_P, **opt_kw):
    """K rows (home nbf x extended nbf, library column order) and the per-cell
    exchange energy from the CUDA path."""
    import torch
    from paper_2009_03555_gb300 import hfx

    per = hfx.Periodic(s, A, r_ext=r_ext, r_P=r_P)
    q = per.quartets(hfx.make_opts(**opt_kw))
    assert q.n_values == per.n_values
    dev = torch.device("cuda")
    Pv = torch.from_numpy(per.pack(P)).to(dev)
    Kv = torch.empty_like(Pv)
    q.build_K(Pv, Kv)
    E = q.exchange_energy(Pv, Kv)  # image rows are zero: the energy per cell
    E_pre = torch.zeros(1, dtype=torch.float64, device=dev)
    hfx.hfx_exchange_energy_noalloc(Pv, Kv, per.n_home_values, E_pre)  # the home rows are the value prefix
    Kd = torch.empty((per.system.n_bf, per.system.n_bf), dtype=torch.float64, device=dev)
    q.unpack(Kv, Kd)
    torch.cuda.synchronize()
    assert abs(E - float(E_pre.item())) <= 1e-13 * abs(E)
    assert float(Kv[per.n_home_values:].abs().max()) == 0.0  # rows of image atoms
    return Kd[:per.n_home_bf].cpu().numpy(), E, per


KW = {"coulomb": dict(kernel=oracle.KERNEL_COULOMB, screen=False, density_screen=False),
      "erfc": dict(kernel=oracle.KERNEL_ERFC, screen=True, density_screen=True, tau=1e-8, eps=1e-8)}


@pytest.mark.parametrize("kname", ["coulomb", "erfc"])
@pytest.mark.parametrize("A,n_atoms,r_ext,r_P,sub", [(SKEW, 3, 5.0, 4.0, 31), (FCC, 2, 4.6, 4.5, 32)],
                         ids=["skew", "fcc"])
def test_periodic_rows_fp64(kname, A, n_atoms, r_ext, r_P, sub):
    from paper_2009_03555_gb300 import hfx
    s = synth.periodic_cell(n_atoms, A, sub=sub, recipe=D_RECIPE)
    P = synth.periodic_density_matrix(s, cutoff=r_P, sub=sub)
    kw = KW[kname]
    hk = dict(kernel={"coulomb": hfx.HFX_KERNEL_COULOMB, "erfc": hfx.HFX_KERNEL_ERFC}[kname], screen=kw["screen"],
              density_screen=kw["density_screen"], precision=hfx.HFX_PREC_FP64)
    K, E, per = gpu_periodic(s, P, A, r_ext, r_P, **hk)
    ref, E_ref = oracle_rows_by_key(s, P, A, r_ext, r_P, **kw)
    keys = [(int(h), tuple(int(x) for x in n)) for h, n in zip(per.ext_home, per.ext_shift)]
    assert set(keys) == set(ref)
    err, outside, n_formed = formed_blocks_error(K, per, ref, s.atom_func_off)
    assert n_formed > s.n_atoms  # blocks beyond the home cell's own
    assert err <= 1e-10, err
    assert outside == 0.0
    assert abs(E - E_ref) <= 1e-9 * abs(E_ref), (E, E_ref)


def test_periodic_energy_mixed():
    from paper_2009_03555_gb300 import hfx
    s = synth.periodic_cell(3, SKEW, sub=33, recipe=D_RECIPE)
    P = synth.periodic_density_matrix(s, cutoff=4.0, sub=33)
    _, E, _ = gpu_periodic(s, P, SKEW, 5.0, 4.0, kernel=hfx.HFX_KERNEL_ERFC, precision=hfx.HFX_PREC_MIXED)
    _, E_ref = oracle_rows_by_key(s, P, SKEW, 5.0, 4.0, **KW["erfc"])
    assert abs(E - E_ref) <= 1e-6, (E, E_ref)


def test_home_cell_quartets_only():
    """The periodic basis evaluates only the quartets with a home-cell shell:
    fewer than the molecular exchange of the same extended set (library's
    molecular path on the same shells and pattern), with the same home rows
    (the skipped quartets reach image rows only)."""
    import torch
    from paper_2009_03555_gb300 import hfx
    s = synth.periodic_cell(3, SKEW, sub=34, recipe=D_RECIPE)
    P = synth.periodic_density_matrix(s, cutoff=4.0, sub=34)
    per = hfx.Periodic(s, SKEW, r_ext=6.0, r_P=4.0)
    opts = hfx.make_opts(kernel=hfx.HFX_KERNEL_ERFC, screen=True, density_screen=True,
                         precision=hfx.HFX_PREC_FP64)
    dev = torch.device("cuda")
    Pv = torch.from_numpy(per.pack(P)).to(dev)
    qp = per.quartets(opts)
    Kp = torch.empty_like(Pv)
    qp.build_K(Pv, Kp)
    qm = hfx.Quartets(hfx.Basis(extended_system(per)), opts, per.mask)
    Km = torch.empty_like(Pv)
    qm.build_K(Pv, Km)
    torch.cuda.synchronize()
    n_p, n_m = sum(qp.stats().n_quartets_computed), sum(qm.stats().n_quartets_computed)
    assert 0 < n_p < n_m
    h = per.n_home_values
    scale = float(Km[:h].abs().max())
    assert float((Kp[:h] - Km[:h]).abs().max()) <= 1e-12 * scale


@pytest.mark.parametrize("kname", ["coulomb", "erfc"])
def test_kpoint_density_rows(kname):
    """A two-point k grid (k = 0 and pi along a1): the real-space densities
    P^L = (P(0) + cos(pi n1) P(pi)) / 2 packed per lattice shift
    (hfx_periodic_pack_lattice_host), built on the periodic basis, against the
    oracle's molecular exchange of the extended set with the density of the
    definition P^{H-N}: home rows on the formed blocks (FP64, 1e-10) and the
    per-cell energy."""
    import torch
    from paper_2009_03555_gb300 import hfx
    from periodic_helpers import extended_density, kgrid_lattice_density, shift_differences
    A, r_ext, r_P = SKEW, 5.0, 4.0
    s = synth.periodic_cell(3, A, sub=36, recipe=D_RECIPE)
    P0 = synth.periodic_density_matrix(s, cutoff=r_P, sub=36)
    Ppi = synth.periodic_density_matrix(s, cutoff=r_P, sub=37)
    per = hfx.Periodic(s, A, r_ext=r_ext, r_P=r_P)
    Lk, PL = kgrid_lattice_density(P0, Ppi, shift_differences(per))
    kw = KW[kname]
    hk = dict(kernel={"coulomb": hfx.HFX_KERNEL_COULOMB, "erfc": hfx.HFX_KERNEL_ERFC}[kname], screen=kw["screen"],
              density_screen=kw["density_screen"], precision=hfx.HFX_PREC_FP64)
    q = per.quartets(hfx.make_opts(**hk))
    dev = torch.device("cuda")
    Pv = torch.from_numpy(per.pack_lattice(Lk, PL)).to(dev)
    Kv = torch.empty_like(Pv)
    q.build_K(Pv, Kv)
    E = q.exchange_energy(Pv, Kv)
    Kd = torch.empty((per.system.n_bf, per.system.n_bf), dtype=torch.float64, device=dev)
    q.unpack(Kv, Kd)
    torch.cuda.synchronize()
    K = Kd[:per.n_home_bf].cpu().numpy()
    e = extended_system(per)
    Pe = extended_density(per, lambda n: 0.5 * (P0 + np.cos(np.pi * n[0]) * Ppi), r_P)
    Km, _ = oracle.build_K(oracle.Basis(e), Pe, **kw)
    md = synth.expand_atom_mask(e, per.mask)[:per.n_home_bf] != 0
    assert np.abs((K - Km[:per.n_home_bf]) * md).max() <= 1e-10
    assert np.all(K[~md] == 0)
    E_ref = -0.5 * float(np.sum(Pe[:per.n_home_bf] * Km[:per.n_home_bf] * md))
    assert abs(E - E_ref) <= 1e-9 * abs(E_ref)
