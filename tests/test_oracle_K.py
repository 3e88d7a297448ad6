"""Pins for the oracle's exchange matrix K_ij = sum_kl (ik|jl) P_kl (Eq. H-HFX
without the -1/2) and E_x = -1/2 sum_ij P_ij K_ij.

Pinned against: the brute-force loop over all ordered shell quartets; the full
ERI tensor contracted with P by einsum; positive semi-definiteness of the ERI
supermatrix (so E_x <= 0 for a positive semi-definite P); symmetry of K;
linearity in P; translation invariance; a relabelling of atoms; and, for the
screening of Sec. 2 (Eq. schwarz, Eq. dmscreening), a rigorous bound on what
the dropped quartets could have contributed.
"""
import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def c0():
    s, P = synth.config0()
    return s, P, oracle.Basis(s)


@pytest.fixture(scope="module")
def tiny():
    s = synth.ch_cluster(3, 98, nprim=2)
    P = synth.density_matrix(s, 98, cutoff=3.0)
    return s, P, oracle.Basis(s)


def test_canonical_quartet_count(c0):
    s, P, b = c0
    npair = s.n_shells * (s.n_shells + 1) // 2
    _, n = oracle.build_K(b, P)
    assert n == npair * (npair + 1) // 2 == 32131


def test_brute_equals_symmetric_unscreened(c0):
    s, P, b = c0
    K, _ = oracle.build_K(b, P)
    Kb, nb = oracle.build_K(b, P, brute=True)
    assert nb == s.n_shells ** 4
    np.testing.assert_allclose(K, Kb, rtol=0, atol=1e-13 * np.abs(Kb).max())


def test_brute_equals_symmetric_screened(tiny):
    s, P, b = tiny
    for k in (oracle.KERNEL_ERFC, oracle.KERNEL_COULOMB):
        kw = dict(kernel=k, screen=True, tau=1e-5, density_screen=True, eps=1e-5)
        K, n = oracle.build_K(b, P, **kw)
        Kb, nb = oracle.build_K(b, P, brute=True, **kw)
        npair = s.n_shells * (s.n_shells + 1) // 2
        assert 0 < n < npair * (npair + 1) // 2
        np.testing.assert_allclose(K, Kb, rtol=0, atol=1e-13 * np.abs(Kb).max())


def _full_tensor(s, b, kernel):
    ns, nbf = s.n_shells, s.n_bf
    fo = s.func_off
    quads = [(I, J, K, L) for I in range(ns) for J in range(ns) for K in range(ns) for L in range(ns)]
    G = np.zeros((nbf, nbf, nbf, nbf))
    for (I, J, K, L), g in zip(quads, oracle.quartets(b, quads, kernel)):
        G[fo[I]:fo[I + 1], fo[J]:fo[J + 1], fo[K]:fo[K + 1], fo[L]:fo[L + 1]] = g
    return G


def test_K_from_full_tensor_psd_and_energy_sign(c0):
    s, P, b = c0
    G = _full_tensor(s, b, oracle.KERNEL_COULOMB)
    Kref = np.einsum("ikjl,kl->ij", G, P)
    K, _ = oracle.build_K(b, P)
    np.testing.assert_allclose(K, Kref, rtol=0, atol=1e-13 * np.abs(Kref).max())
    nbf = s.n_bf
    M = G.reshape(nbf * nbf, nbf * nbf)
    np.testing.assert_allclose(M, M.T, rtol=0, atol=1e-13 * np.abs(M).max())
    ev = np.linalg.eigvalsh(0.5 * (M + M.T))
    assert ev.min() >= -1e-12 * ev.max()
    assert oracle.exchange_energy(P, K) < 0.0


def test_K_symmetric_and_linear(c0):
    s, P, b = c0
    rng = np.random.default_rng(3)
    X = rng.standard_normal(P.shape)
    X = X + X.T
    K1, _ = oracle.build_K(b, P)
    K2, _ = oracle.build_K(b, X)
    K3, _ = oracle.build_K(b, P - 2.5 * X)
    np.testing.assert_allclose(K1, K1.T, rtol=0, atol=1e-14 * np.abs(K1).max())
    np.testing.assert_allclose(K3, K1 - 2.5 * K2, rtol=0, atol=1e-12 * np.abs(K3).max())


def test_K_translation_invariance(tiny):
    s, P, b = tiny
    kw = dict(kernel=oracle.KERNEL_ERFC, screen=True, tau=1e-8, density_screen=True, eps=1e-8)
    K1, n1 = oracle.build_K(b, P, **kw)
    K2, n2 = oracle.build_K(oracle.Basis(s.translated([-4.0, 2.5, 7.25])), P, **kw)
    assert n1 == n2
    np.testing.assert_allclose(K2, K1, rtol=0, atol=1e-12 * np.abs(K1).max())


def test_K_atom_relabelling(tiny):
    """Reversing the atom order (shells and functions move with their atom)
    permutes K the same way."""
    s, P, b = tiny
    order = np.arange(s.n_atoms)[::-1]
    shells = [S for a in order for S in range(s.n_shells) if s.shell_atom[S] == a]
    newpos = {int(a): i for i, a in enumerate(order)}
    alpha, coef, off = [], [], [0]
    for S in shells:
        p0, p1 = s.prim_off[S], s.prim_off[S + 1]
        alpha.extend(s.alpha[p0:p1]); coef.extend(s.coef[p0:p1]); off.append(off[-1] + p1 - p0)
    s2 = synth.System(name="rev", atom_Z=s.atom_Z[order], atom_xyz=s.atom_xyz[order],
                      shell_atom=np.array([newpos[int(s.shell_atom[S])] for S in shells], dtype=np.int32),
                      shell_l=s.shell_l[shells], prim_off=np.array(off, dtype=np.int32),
                      alpha=np.array(alpha), coef=np.array(coef))
    fo = s.func_off
    perm = np.concatenate([np.arange(fo[S], fo[S + 1]) for S in shells])
    P2 = P[np.ix_(perm, perm)]
    kw = dict(kernel=oracle.KERNEL_ERFC, screen=True, tau=1e-8, density_screen=True, eps=1e-8)
    K1, _ = oracle.build_K(b, P, **kw)
    K2, _ = oracle.build_K(oracle.Basis(s2), P2, **kw)
    np.testing.assert_allclose(K2, K1[np.ix_(perm, perm)], rtol=0, atol=1e-13 * np.abs(K1).max())


def test_screening_error_bound(tiny):
    """Each dropped canonical quartet has integrals |(ab|cd)| <= Q_IJ Q_KL
    (Eq. schwarz) and reaches any K element through at most 8 permutations,
    each a sum of at most 6 x 6 products with P.  A quartet dropped by the
    Schwarz test has Q_IJ Q_KL <= tau, one dropped by density screening has
    P_scr Q_IJ Q_KL <= eps, and one with P_scr = 0 contributes nothing, so
    |K_screened - K_full| <= n_dropped * 8 * 36 * max(tau * max|P|, eps)."""
    s, P, b = tiny
    k = oracle.KERNEL_ERFC
    tau = eps = 1e-4
    Kf, nf = oracle.build_K(b, P, kernel=k)
    Ks, ns_ = oracle.build_K(b, P, kernel=k, screen=True, tau=tau, density_screen=True, eps=eps)
    dropped = nf - ns_
    assert dropped > 0
    bound = dropped * 8 * 36 * max(tau * np.abs(P).max(), eps)
    diff = np.abs(Ks - Kf).max()
    assert 0.0 < diff <= bound


def test_K_shell_pairs_equals_full_tensor(tiny):
    """Single exchange blocks from the definition equal the full ERI tensor
    contracted with P (unscreened), for every shell pair, with W0 = sum |P|."""
    s, P, b = tiny
    G = _full_tensor(s, b, oracle.KERNEL_ERFC)
    Kref = np.einsum("ikjl,kl->ij", G, P)
    fo = s.func_off
    pairs = [(I, J) for I in range(s.n_shells) for J in range(s.n_shells)]
    blocks, _, W0, n = oracle.K_shell_pairs(b, P, pairs, kernel=oracle.KERNEL_ERFC)
    assert n == s.n_shells ** 4
    for (I, J), k, w0 in zip(pairs, blocks, W0):
        np.testing.assert_allclose(k, Kref[fo[I]:fo[I + 1], fo[J]:fo[J + 1]], rtol=0,
                                   atol=1e-13 * np.abs(Kref).max())
        np.testing.assert_allclose(w0, np.abs(P).sum(), rtol=1e-13)


def test_K_shell_pairs_screened_equals_brute(tiny):
    """With Schwarz and density screening the blocks equal the brute-force K
    (all ordered quartets, same predicate) and count the same quartets."""
    s, P, b = tiny
    kw = dict(kernel=oracle.KERNEL_ERFC, screen=True, tau=1e-5, density_screen=True, eps=1e-5)
    Kb, nb = oracle.build_K(b, P, brute=True, **kw)
    fo = s.func_off
    pairs = [(I, J) for I in range(s.n_shells) for J in range(s.n_shells)]
    blocks, W1, W0, n = oracle.K_shell_pairs(b, P, pairs, **kw)
    assert n == nb
    Q = oracle.schwarz(b, oracle.KERNEL_ERFC)
    for (I, J), k, w1, w0 in zip(pairs, blocks, W1, W0):
        np.testing.assert_allclose(k, Kb[fo[I]:fo[I + 1], fo[J]:fo[J + 1]], rtol=0,
                                   atol=1e-13 * np.abs(Kb).max())
        # Schwarz: |K_ij| <= sum over surviving (K,L) of Q_IK Q_JL sum |P_kl| = W1
        assert np.all(np.abs(k) <= w1 * (1 + 1e-12) + 1e-300)
        assert np.all(w1 <= Q.max() ** 2 * w0 * (1 + 1e-12))


@pytest.mark.parametrize("dscreen", [False, True])
def test_count_quartets_equals_canonical_loop(tiny, dscreen):
    """The ranked-prefix count of surviving canonical quartets equals the
    count of the canonical quartet loop with the same screening, and its
    Schwarz bounds are the oracle's."""
    s, P, b = tiny
    kw = dict(kernel=oracle.KERNEL_ERFC, tau=1e-6, density_screen=dscreen, eps=1e-6)
    _, n_loop = oracle.build_K(b, P, screen=True, **kw)
    n, Q = oracle.count_quartets(b, P, **kw)
    assert n == n_loop > 0
    np.testing.assert_array_equal(Q, oracle.schwarz(b, oracle.KERNEL_ERFC))


def _canonical_survivors(s, Pmax_nonzero, pairing):
    """Brute-force count of canonical shell quartets (I>=J, K>=L, IJ>=KL) whose
    P_scr is nonzero, with P_scr built from the shell-pair blocks ``pairing``
    names: 'exchange' = the four blocks (IK, IL, JK, JL) of Eq. dmscreening,
    'coulomb' = (IJ, KL), a plausible wrong reading."""
    ns = s.n_shells
    pairs = [(i, j) for i in range(ns) for j in range(i + 1)]
    n = 0
    for a in range(len(pairs)):
        I, J = pairs[a]
        for c in range(a + 1):
            K, L = pairs[c]
            if pairing == "exchange":
                nz = Pmax_nonzero[I, K] or Pmax_nonzero[I, L] or Pmax_nonzero[J, K] or Pmax_nonzero[J, L]
            else:
                nz = Pmax_nonzero[I, J] or Pmax_nonzero[K, L]
            n += bool(nz)
    return n


def test_exact_pscr_skip_uses_the_four_exchange_blocks():
    """The exact P_scr = 0 skip alone (Schwarz threshold 0, no density
    screening) with P nonzero in one off-diagonal atom-pair block only: every
    skipped quartet has all four exchange blocks P_IK, P_IL, P_JK, P_JL zero
    (Eq. dmscreening), so it contributes nothing and the screened K equals the
    unscreened K; the number of survivors equals a brute-force count over the
    canonical quartets with those four blocks.  Pairing the blocks as
    (P_IJ, P_KL) instead changes both for this P."""
    s = synth.ch_cluster(4, 97, nprim=2)
    b = oracle.Basis(s)
    rng = np.random.default_rng(97)
    fo = s.atom_func_off
    X, Y = 0, 2
    P = np.zeros((s.n_bf, s.n_bf))
    blk = rng.standard_normal((fo[X + 1] - fo[X], fo[Y + 1] - fo[Y]))
    P[fo[X]:fo[X + 1], fo[Y]:fo[Y + 1]] = blk
    P[fo[Y]:fo[Y + 1], fo[X]:fo[X + 1]] = blk.T
    k = oracle.KERNEL_ERFC
    Kf, nf = oracle.build_K(b, P, kernel=k)
    Ks, ns_ = oracle.build_K(b, P, kernel=k, screen=True, tau=0.0, density_screen=False)
    assert 0 < ns_ < nf
    assert np.abs(Kf).max() > 0
    np.testing.assert_allclose(Ks, Kf, rtol=0, atol=1e-14 * np.abs(Kf).max())
    # shell-pair |P| maxima, then the brute-force survivor counts
    sf = s.func_off
    nz = np.zeros((s.n_shells, s.n_shells), dtype=bool)
    for I in range(s.n_shells):
        for J in range(s.n_shells):
            nz[I, J] = np.abs(P[sf[I]:sf[I + 1], sf[J]:sf[J + 1]]).max() > 0
    n_exch = _canonical_survivors(s, nz, "exchange")
    assert ns_ == n_exch
    n_count, _ = oracle.count_quartets(b, P, kernel=k, tau=0.0, density_screen=False)
    assert n_count == n_exch
    assert _canonical_survivors(s, nz, "coulomb") != n_exch
