"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (stated by the method's accuracy target):
  * FP64 path: |dK|max <= 1e-10 and |dE_x| <= 1e-9 * |E_x|;
    individual integrals within 1e-12 of the largest integral of the quartet.
  * mixed path (FP32 recursions with compensated FP32 contraction, FP64
    Boys/prefactors/accumulation): |dE_x| <= 1e-6 Ha; integrals within
    2e-4 Q_IJ Q_KL (the Schwarz bound of the quartet; FP32 cancellation in the
    vertical recursion of d-shell classes reaches ~6e-5 of it).
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import mask_dense, pattern_mask, run_gpu_K

pytestmark = pytest.mark.gpu

KMAP = {"coulomb": oracle.KERNEL_COULOMB, "erfc": oracle.KERNEL_ERFC, "erf": oracle.KERNEL_ERF}


@pytest.fixture(scope="module")
def ch3():
    return synth.ch_cluster(3, 97, nprim=4)


def _all_class_quartets(s, rng, per_class=3):
    """Shell quartets covering every (la lb | lc ld) pattern in random orders."""
    by = {l: [S for S in range(s.n_shells) if s.shell_l[S] == l] for l in (0, 1, 2)}
    out = []
    for la in range(3):
        for lb in range(3):
            for lc in range(3):
                for ld in range(3):
                    for _ in range(per_class):
                        out.append(tuple(int(rng.choice(by[l])) for l in (la, lb, lc, ld)))
    return out


@pytest.mark.parametrize("kname", ["coulomb", "erfc", "erf"])
def test_quartet_integrals_fp64(ch3, kname):
    from paper_2009_03555_gb300 import hfx
    rng = np.random.default_rng(21)
    qs = _all_class_quartets(ch3, rng, per_class=2)
    b = hfx.Basis(ch3)
    got = b.eval_quartets(qs, kernel=KMAP[kname], omega=0.11, precision=hfx.HFX_PREC_FP64)
    ref = oracle.quartets(oracle.Basis(ch3), qs, KMAP[kname], 0.11)
    for q, g, r in zip(qs, got, ref):
        scale = max(np.abs(r).max(), 1e-300)
        assert np.abs(g - r).max() <= 1e-12 * max(scale, 1.0), (q, np.abs(g - r).max(), scale)


@pytest.mark.parametrize("kname", ["coulomb", "erfc"])
def test_quartet_integrals_mixed(ch3, kname):
    from paper_2009_03555_gb300 import hfx
    rng = np.random.default_rng(22)
    qs = _all_class_quartets(ch3, rng, per_class=1)
    b = hfx.Basis(ch3)
    got = b.eval_quartets(qs, kernel=KMAP[kname], omega=0.11, precision=hfx.HFX_PREC_MIXED)
    ob = oracle.Basis(ch3)
    ref = oracle.quartets(ob, qs, KMAP[kname], 0.11)
    Q = oracle.schwarz(ob, KMAP[kname], 0.11)
    for q, g, r in zip(qs, got, ref):
        qq = Q[q[0], q[1]] * Q[q[2], q[3]]
        assert np.abs(g - r).max() <= 2e-4 * qq + 1e-15, (q, np.abs(g - r).max(), qq)


def test_water_dimer_coulomb_fp64():
    """Two water-like molecules, full Coulomb, no screening, dense P."""
    s, P = synth.config0()
    Kref, n = oracle.build_K(oracle.Basis(s), P)
    K, E, q = run_gpu_K(s, P, kernel=0, screen=False, density_screen=False, prim_cutoff=0.0)
    st = q.stats()
    assert sum(st.n_quartets_computed) == n == 32131
    assert np.abs(K - Kref).max() <= 1e-10
    Eref = oracle.exchange_energy(P, Kref)
    assert abs(E - Eref) <= 1e-9 * abs(Eref)
    np.testing.assert_allclose(K, K.T, rtol=0, atol=1e-13)


@pytest.mark.parametrize("n_block", [1, 7, 128])
def test_water_dimer_batch_sizes(n_block):
    """The work-queue batch size must not change the result (ragged tails)."""
    s, P = synth.config0()
    Kref, _ = oracle.build_K(oracle.Basis(s), P)
    K, _, _ = run_gpu_K(s, P, kernel=0, screen=False, density_screen=False, prim_cutoff=0.0, n_block=n_block)
    assert np.abs(K - Kref).max() <= 1e-10


@pytest.mark.parametrize("n_atoms,seed", [(3, 11), (5, 12)])
def test_hse_cluster_screened_fp64(n_atoms, seed):
    """C/H cluster with d shells, erfc kernel (w = 0.11), Schwarz 1e-8 and
    density screening, P cut beyond 6 bohr (sparse pattern)."""
    s = synth.ch_cluster(n_atoms, seed)
    mask = pattern_mask(s, 6.0)
    P = synth.density_matrix(s, seed) * mask_dense(s, mask)
    kw = dict(kernel=oracle.KERNEL_ERFC, omega=0.11, screen=True, tau=1e-8, density_screen=True, eps=1e-8)
    Kref, n = oracle.build_K(oracle.Basis(s), P, **kw)
    K, E, q = run_gpu_K(s, P, mask=mask, prim_cutoff=1e-14, **kw)
    md = mask_dense(s, mask)
    assert np.abs((K - Kref) * md).max() <= 1e-10
    assert np.all(K[md == 0] == 0)
    assert sum(q.stats().n_quartets_computed) == n
    Eref = oracle.exchange_energy(P, Kref)
    assert abs(E - Eref) <= 1e-9 * abs(Eref)


def test_hse_cluster_mixed_energy():
    s = synth.ch_cluster(5, 12)
    mask = pattern_mask(s, 6.0)
    P = synth.density_matrix(s, 12) * mask_dense(s, mask)
    kw = dict(kernel=oracle.KERNEL_ERFC, omega=0.11, screen=True, tau=1e-8, density_screen=True, eps=1e-8)
    Kref, _ = oracle.build_K(oracle.Basis(s), P, **kw)
    Eref = oracle.exchange_energy(P, Kref)
    from paper_2009_03555_gb300 import hfx
    K, E, _ = run_gpu_K(s, P, mask=mask, precision=hfx.HFX_PREC_MIXED, **kw)
    assert abs(E - Eref) <= 1e-6
    K2, E2, _ = run_gpu_K(s, P, mask=mask, precision=hfx.HFX_PREC_MIXED, fp64_promote_bound=1e-3, **kw)
    assert abs(E2 - Eref) <= abs(E - Eref) + 1e-9


def test_zero_density_gives_zero_K():
    s, P = synth.config0()
    K, E, q = run_gpu_K(s, np.zeros_like(P), kernel=0, screen=True, density_screen=True)
    assert np.all(K == 0) and E == 0.0
    assert sum(q.stats().n_quartets_computed) == 0


def test_single_s_shell():
    s = synth.System(name="one", atom_Z=np.array([1], dtype=np.int32), atom_xyz=np.zeros((1, 3)),
                     shell_atom=np.array([0], dtype=np.int32), shell_l=np.array([0], dtype=np.int32),
                     prim_off=np.array([0, 1], dtype=np.int32), alpha=np.array([0.7]), coef=np.array([1.0]))
    P = np.array([[1.0]])
    Kref, _ = oracle.build_K(oracle.Basis(s), P)
    K, E, _ = run_gpu_K(s, P, kernel=0, screen=False, density_screen=False, prim_cutoff=0.0)
    # (ss|ss) of one unit Gaussian charge: 2 sqrt(mu/pi), mu = (2a)(2a)/(4a) = a
    assert K[0, 0] == pytest.approx(2.0 * np.sqrt(0.7 / np.pi), rel=1e-14)
    assert K[0, 0] == pytest.approx(Kref[0, 0], rel=1e-14)


def _joined(a, b):
    """Systems a and b as one system (b's atoms after a's)."""
    return synth.System(name=a.name + "+" + b.name, atom_Z=np.concatenate([a.atom_Z, b.atom_Z]),
                        atom_xyz=np.concatenate([a.atom_xyz, b.atom_xyz]),
                        shell_atom=np.concatenate([a.shell_atom, b.shell_atom + a.n_atoms]).astype(np.int32),
                        shell_l=np.concatenate([a.shell_l, b.shell_l]).astype(np.int32),
                        prim_off=np.concatenate([a.prim_off, b.prim_off[1:] + a.prim_off[-1]]).astype(np.int32),
                        alpha=np.concatenate([a.alpha, b.alpha]), coef=np.concatenate([a.coef, b.coef]))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_disconnected_molecules(prec):
    """Two HSE clusters 200 bohr apart with a block-diagonal density pattern: no
    shell pair spans the gap (its Schwarz bound underflows) and every cross
    quartet has P_scr = 0, so K is the two clusters' own exchange matrices side
    by side, each equal to the build of that cluster alone (to the rounding of
    the FP64 accumulation order), and the build computes exactly the two
    clusters' quartets.  FP64: also against the oracle on each cluster."""
    from paper_2009_03555_gb300 import hfx
    a, b = synth.ch_cluster(4, 21), synth.ch_cluster(3, 22)
    Pa, Pb = synth.density_matrix(a, 21), synth.density_matrix(b, 22)
    s = _joined(a, b.translated([200.0, 0.0, 0.0]))
    na, nfa = a.n_atoms, a.n_bf
    P = np.zeros((s.n_bf, s.n_bf))
    P[:nfa, :nfa], P[nfa:, nfa:] = Pa, Pb
    mask = np.zeros((s.n_atoms, s.n_atoms), dtype=bool)
    mask[:na, :na] = True
    mask[na:, na:] = True
    precision = hfx.HFX_PREC_FP64 if prec == "fp64" else hfx.HFX_PREC_MIXED
    kw = dict(kernel=hfx.HFX_KERNEL_ERFC, omega=0.11, screen=True, tau=1e-8, density_screen=True, eps=1e-8,
              precision=precision)
    K, E, q = run_gpu_K(s, P, mask, **kw)
    Ka, Ea, qa = run_gpu_K(a, Pa, **kw)
    Kb, Eb, qb = run_gpu_K(b, Pb, **kw)
    n = sum(q.stats().n_quartets_computed)
    assert n == sum(qa.stats().n_quartets_computed) + sum(qb.stats().n_quartets_computed)
    assert np.all(K[:nfa, nfa:] == 0) and np.all(K[nfa:, :nfa] == 0)
    scale = max(np.abs(Ka).max(), np.abs(Kb).max())
    assert np.abs(K[:nfa, :nfa] - Ka).max() <= 1e-12 * scale
    assert np.abs(K[nfa:, nfa:] - Kb).max() <= 1e-12 * scale
    assert abs(E - (Ea + Eb)) <= 1e-12 * abs(Ea + Eb)
    if prec == "fp64":
        okw = dict(kernel=oracle.KERNEL_ERFC, omega=0.11, screen=True, tau=1e-8, density_screen=True, eps=1e-8)
        Kra, n_a = oracle.build_K(oracle.Basis(a), Pa, **okw)
        Krb, n_b = oracle.build_K(oracle.Basis(b), Pb, **okw)
        assert n == n_a + n_b
        assert np.abs(Ka - Kra).max() <= 1e-10 and np.abs(Kb - Krb).max() <= 1e-10


def test_empty_basis_is_rejected():
    from paper_2009_03555_gb300 import hfx
    empty = synth.System(name="empty", atom_Z=np.zeros(0, dtype=np.int32), atom_xyz=np.zeros((0, 3)),
                         shell_atom=np.zeros(0, dtype=np.int32), shell_l=np.zeros(0, dtype=np.int32),
                         prim_off=np.zeros(1, dtype=np.int32), alpha=np.zeros(0), coef=np.zeros(0))
    with pytest.raises(hfx.HFXError) as ei:
        hfx.Basis(empty)
    assert ei.value.status == 1


def test_errors_are_reported():
    from paper_2009_03555_gb300 import hfx
    s = synth.ch_cluster(2, 5)
    bad = synth.System(name="f", atom_Z=s.atom_Z, atom_xyz=s.atom_xyz, shell_atom=s.shell_atom,
                       shell_l=np.where(s.shell_l == 2, 3, s.shell_l).astype(np.int32), prim_off=s.prim_off,
                       alpha=s.alpha, coef=s.coef)
    with pytest.raises(hfx.HFXError) as ei:
        hfx.Basis(bad)
    assert ei.value.status == 4
    nan = synth.System(name="n", atom_Z=s.atom_Z, atom_xyz=s.atom_xyz, shell_atom=s.shell_atom,
                       shell_l=s.shell_l, prim_off=s.prim_off, alpha=np.where(np.arange(len(s.alpha)) == 3,
                                                                              np.nan, s.alpha), coef=s.coef)
    with pytest.raises(hfx.HFXError) as ei:
        hfx.Basis(nan)
    assert ei.value.status == 1
    b = hfx.Basis(s)
    asym = np.array([[True, True], [False, True]])
    with pytest.raises(hfx.HFXError) as ei:
        hfx.Quartets(b, hfx.make_opts(), asym)
    assert ei.value.status == 1


@pytest.mark.parametrize("min_l,d_only", [(0, False), (8, True)], ids=["every-class", "dddd-only"])
def test_promoted_pass_elementwise_fp64(min_l, d_only):
    """The FP64-promoted pass of the mixed path (the launch the benchmark's
    (dd|dd) promotion runs) element by element against the oracle at the FP64
    tolerance: promotion bound 0 sends every surviving quartet of the promoted
    classes to FP64.  With classes of total l >= 8 only, a system of d shells
    alone makes every quartet (dd|dd), so the whole K comes from that pass."""
    from paper_2009_03555_gb300 import hfx
    s = synth.ch_cluster(4, 13)
    mask = pattern_mask(s, 6.0)
    P = synth.density_matrix(s, 13) * mask_dense(s, mask)
    if d_only:
        s, P = synth.shell_subset(s, P, [2])
    kw = dict(kernel=oracle.KERNEL_ERFC, omega=0.11, screen=True, tau=1e-8, density_screen=True, eps=1e-8)
    Kref, n = oracle.build_K(oracle.Basis(s), P, **kw)
    K, E, q = run_gpu_K(s, P, mask=mask, prim_cutoff=1e-14, precision=hfx.HFX_PREC_MIXED,
                        fp64_promote_bound=0.0, promote_min_l=min_l, **kw)
    st = q.stats()
    assert sum(st.n_quartets_pass[0]) == 0 and sum(st.n_quartets_pass[1]) == n
    md = mask_dense(s, mask)
    assert np.abs((K - Kref) * md).max() <= 1e-10
    Eref = oracle.exchange_energy(P, Kref)
    assert abs(E - Eref) <= 1e-9 * abs(Eref)


def test_promotion_routing_matches_oracle_count():
    """Mixed build with (dd|dd) promotion above Q_IJ Q_KL P_scr = 1e-3 (classes
    of total l >= 8): the FP64 pass evaluates exactly the (dd|dd) quartets the
    oracle counts with eps = 1e-3 on the d shells alone, the FP32 pass the rest
    of the surviving quartets, and the energy stays within 1e-6 Ha."""
    from paper_2009_03555_gb300 import hfx
    s = synth.ch_cluster(6, 14)
    mask = pattern_mask(s, 8.0)
    P = synth.density_matrix(s, 14) * mask_dense(s, mask)
    kw = dict(kernel=oracle.KERNEL_ERFC, omega=0.11, tau=1e-8, density_screen=True, eps=1e-8)
    Kref, n = oracle.build_K(oracle.Basis(s), P, screen=True, **kw)
    sd, Pd = synth.shell_subset(s, P, [2])
    n_dd, _ = oracle.count_quartets(oracle.Basis(sd), Pd, kernel=oracle.KERNEL_ERFC, omega=0.11, tau=1e-8,
                                    density_screen=True, eps=1e-3)
    assert 0 < n_dd
    K, E, q = run_gpu_K(s, P, mask=mask, screen=True, precision=hfx.HFX_PREC_MIXED, fp64_promote_bound=1e-3,
                        promote_min_l=8, **kw)
    st = q.stats()
    dd = [c for c in range(hfx.N_CLASSES) if hfx.hfx_get_class_info(c).bra_class == 5
          and hfx.hfx_get_class_info(c).ket_class == 5]
    assert st.n_quartets_pass[1][dd[0]] == n_dd == sum(st.n_quartets_pass[1])
    assert sum(st.n_quartets_pass[0]) + n_dd == n
    Eref = oracle.exchange_energy(P, Kref)
    assert abs(E - Eref) <= 1e-6


def _sixteen_primitive_d_system():
    """Two atoms: a d shell of 16 primitives (the library's primitive limit,
    256 primitive pairs per shell pair) plus an s shell on atom 0, an s and a
    p shell of 2 primitives on atom 1; exponents log-uniform in [0.1, 50]."""
    rng = np.random.default_rng(2009_03555 + 16)
    shells = [(0, 2, 16), (0, 0, 2), (1, 0, 2), (1, 1, 2)]  # (atom, l, nprim)
    alpha, coef, off = [], [], [0]
    for _, _, k in shells:
        alpha.extend(sorted(np.exp(rng.uniform(np.log(0.1), np.log(50.0), size=k)), reverse=True))
        coef.extend(rng.uniform(0.1, 1.0, size=k))
        off.append(off[-1] + k)
    return synth.System(name="d16", atom_Z=np.array([6, 1], dtype=np.int32),
                        atom_xyz=np.array([[0.0, 0.0, 0.0], [1.2, 0.9, -0.7]]),
                        shell_atom=np.array([a for a, _, _ in shells], dtype=np.int32),
                        shell_l=np.array([l for _, l, _ in shells], dtype=np.int32),
                        prim_off=np.array(off, dtype=np.int32), alpha=np.array(alpha), coef=np.array(coef))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sixteen_primitive_d_shell(prec):
    """A d shell at the 16-primitive limit through the warp-split (d-shell
    class) path: FP64 at |dK|max <= 1e-10, mixed at |dE_x| <= 1e-6 Ha."""
    from paper_2009_03555_gb300 import hfx
    s = _sixteen_primitive_d_system()
    P = synth.density_matrix(s, 16, n_occ=3)
    kw = dict(kernel=oracle.KERNEL_ERFC, omega=0.11, screen=False, density_screen=False)
    Kref, n = oracle.build_K(oracle.Basis(s), P, **kw)
    p = hfx.HFX_PREC_FP64 if prec == "fp64" else hfx.HFX_PREC_MIXED
    K, E, q = run_gpu_K(s, P, prim_cutoff=0.0, precision=p, **kw)
    assert sum(q.stats().n_quartets_computed) == n
    Eref = oracle.exchange_energy(P, Kref)
    if prec == "fp64":
        assert np.abs(K - Kref).max() <= 1e-10
        assert abs(E - Eref) <= 1e-9 * abs(Eref)
    else:
        assert abs(E - Eref) <= 1e-6


def test_promotion_per_primitive_quartet():
    """Promotion per primitive quartet: of the quartets above the bound, the
    primitive quartets with bound_ab bound_cd P_scr above it run in FP64, the
    rest in FP32.  Every primitive quartet runs exactly once over the two
    launches (their counts add up to the unpromoted build's), bound 0 sends
    every primitive quartet to FP64 (K at the FP64 tolerance), and a bound in
    between keeps the energy within 1e-6 Ha of the oracle."""
    from paper_2009_03555_gb300 import hfx
    s = synth.ch_cluster(5, 15)
    mask = pattern_mask(s, 6.0)
    P = synth.density_matrix(s, 15) * mask_dense(s, mask)
    kw = dict(kernel=oracle.KERNEL_ERFC, omega=0.11, screen=True, tau=1e-8, density_screen=True, eps=1e-8)
    Kref, n = oracle.build_K(oracle.Basis(s), P, **kw)
    Eref = oracle.exchange_energy(P, Kref)
    md = mask_dense(s, mask)
    _, _, q0 = run_gpu_K(s, P, mask=mask, prim_cutoff=1e-14, precision=hfx.HFX_PREC_MIXED, **kw)
    npq0 = sum(q0.stats().n_prim_quartets_pass[0])
    K, E, q = run_gpu_K(s, P, mask=mask, prim_cutoff=1e-14, precision=hfx.HFX_PREC_MIXED, fp64_promote_bound=0.0,
                        promote_prims=True, **kw)
    st = q.stats()
    assert sum(st.n_prim_quartets_pass[0]) == 0 and sum(st.n_prim_quartets_pass[1]) == npq0
    assert sum(st.n_quartets_computed) == n
    assert np.abs((K - Kref) * md).max() <= 1e-10
    K, E, q = run_gpu_K(s, P, mask=mask, prim_cutoff=1e-14, precision=hfx.HFX_PREC_MIXED, fp64_promote_bound=1e-4,
                        promote_prims=True, **kw)
    st = q.stats()
    n1 = sum(st.n_prim_quartets_pass[1])
    assert 0 < n1 < npq0 and sum(st.n_prim_quartets_pass[0]) + n1 == npq0
    assert sum(st.n_quartets_computed) == n
    assert abs(E - Eref) <= 1e-6


def test_distance_screening_drops_only_negligible_pairs():
    """Distance screening (extent_eps = 1e-12: shell pairs farther apart than the
    sum of their most diffuse primitives' 1e-12 radii are dropped before their
    Schwarz bounds are formed): on a 24-atom chain (s and p shells) it removes
    half of the shell pairs, and the build still equals the oracle's
    unscreened-by-distance K (FP64, 1e-10) with the same number of surviving
    quartets -- the dropped pairs are far below the Schwarz threshold."""
    s = synth.ch_chain(24, sub=7)
    mask = pattern_mask(s, 14.0)
    P = synth.density_matrix(s, 4, cutoff=14.0, sub=7)
    s, P = synth.shell_subset(s, P, [0, 1])
    kw = dict(kernel=oracle.KERNEL_ERFC, omega=0.11, screen=True, tau=1e-8, density_screen=True, eps=1e-8)
    Kref, n = oracle.build_K(oracle.Basis(s), P, **kw)
    K, E, q = run_gpu_K(s, P, mask=mask, prim_cutoff=1e-14, extent_eps=1e-12, **kw)
    st = q.stats()
    all_pairs = s.n_shells * (s.n_shells + 1) // 2
    assert st.n_pairs_distance < 0.7 * all_pairs
    assert sum(st.n_quartets_computed) == n
    md = mask_dense(s, mask)
    assert np.abs((K - Kref) * md).max() <= 1e-10
    Eref = oracle.exchange_energy(P, Kref)
    assert abs(E - Eref) <= 1e-9 * abs(Eref)
