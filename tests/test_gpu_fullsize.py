"""Parity at the full benchmark size, in the launch configuration the benchmark
times: the 400-atom C/H cluster (5600 Cartesian functions), HSE erfc kernel
(w = 0.11), Schwarz 1e-8 with density screening, P cut at 14 bohr, mixed
precision with the (dd|dd) quartets above Q_IJ Q_KL P_scr = 1e-5 promoted to
FP64 (promotion bound 1e-5, classes of total l >= 8), primitive cutoff 1e-13,
work-queue batches of 128 quartets: the options bench.py times.

The oracle cannot build the whole K at this size, so it computes sampled
exchange blocks K_IJ one shell pair at a time straight from the definition
(every ordered (K, L) whose quartet (I K | J L) survives the same screening),
and two quartet counts stored by oracle/count_quartets.py, which the build
must match exactly: the surviving canonical quartets (both precision passes
together) and the (dd|dd) quartets above the promotion bound (the FP64 pass).

Tolerance, derived from the per-integral bounds of the mixed path: each
integral of a surviving quartet is within 2e-4 Q_IK Q_JL of the exact value
(FP32 recursions; the bound tested per integral in test_gpu_parity), and the
primitive cutoff drops at most 256 primitive quartets per shell quartet, each
below 1e-13; so |dK_ij| <= 2e-4 W1_ij + 256e-13 W0_ij with the oracle's
weights W1 = sum Q_IK Q_JL sum|P_kl| and W0 = sum sum|P_kl| over the surviving
(K, L).  The observed errors are also required to stay below 1e-7 of the
largest sampled |K| element, a much tighter check that catches a dropped or
misplaced contribution (those are of the order of K itself).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

N_ATOMS = 400


def _workload():
    s, P = synth.config2(N_ATOMS)
    mask = synth.atom_pair_mask(s, 14.0)
    return s, P * synth.expand_atom_mask(s, mask), mask


def _sample_pairs(s, rng):
    """Shell pairs (I, J) inside the P pattern covering the angular-momentum
    combinations and the distance range of the pattern."""
    d = synth.atom_distances(s)
    sa, sl = s.shell_atom, s.shell_l
    want = [  # (l_I, l_J, distance range in bohr)
        (2, 2, (0.0, 0.0)),     # a diagonal d block (same shell)
        (2, 2, (2.0, 4.0)),
        (2, 1, (4.0, 8.0)),
        (1, 0, (8.0, 12.0)),
        (0, 0, (0.0, 0.0)),
        (1, 2, (2.0, 6.0)),
        (2, 2, (12.0, 14.0)),
    ]
    out = []
    for li, lj, (r0, r1) in want:
        I_all = np.flatnonzero(sl == li)
        J_all = np.flatnonzero(sl == lj)
        if r1 == 0.0:
            I = int(rng.choice(I_all))
            out.append((I, I))
            continue
        dd = d[sa[I_all][:, None], sa[J_all][None, :]]
        ii, jj = np.nonzero((dd >= r0) & (dd <= r1))
        k = int(rng.integers(len(ii)))
        out.append((int(I_all[ii[k]]), int(J_all[jj[k]])))
    return out


def test_sampled_blocks_400_atoms_mixed():
    import torch
    from paper_2009_03555_gb300 import hfx

    s, P, mask = _workload()
    opts = hfx.make_opts(kernel=hfx.HFX_KERNEL_ERFC, omega=0.11, screen=True, tau=1e-8, density_screen=True,
                         eps=1e-8, prim_cutoff=1e-13, precision=hfx.HFX_PREC_MIXED, n_block=128,
                         fp64_promote_bound=1e-5, promote_min_l=8)
    basis = hfx.Basis(s)
    q = hfx.Quartets(basis, opts, mask)
    dev = torch.device("cuda")
    Pd = torch.from_numpy(P).to(dev)
    Pv = torch.empty(q.n_values, dtype=torch.float64, device=dev)
    Kv = torch.empty(q.n_values, dtype=torch.float64, device=dev)
    q.pack(Pd, Pv)
    q.build_K(Pv, Kv)
    E = q.exchange_energy(Pv, Kv)
    Kd = torch.empty_like(Pd)
    q.unpack(Kv, Kd)
    torch.cuda.synchronize()
    K = Kd.cpu().numpy()
    del Kd, Pd
    assert np.isfinite(E) and E < 0.0
    np.testing.assert_array_equal(K, K.T)
    # every surviving canonical quartet computed once: the oracle's count of the
    # same screening (oracle/count_quartets.py, tests/golden/)
    import json
    import os
    gold = os.path.join(os.path.dirname(__file__), "golden")
    with open(os.path.join(gold, f"quartet_count_hse_c{N_ATOMS}.json")) as fh:
        n_oracle = json.load(fh)["canonical_quartets"]
    with open(os.path.join(gold, f"quartet_count_hse_c{N_ATOMS}_dddd_above1e-05.json")) as fh:
        n_promoted = json.load(fh)["canonical_quartets"]
    st = q.stats()
    assert sum(st.n_quartets_computed) == n_oracle
    assert sum(st.n_quartets_pass[0]) + sum(st.n_quartets_pass[1]) == n_oracle
    dddd = [c for c in range(hfx.N_CLASSES) if hfx.hfx_get_class_info(c).la + hfx.hfx_get_class_info(c).lb
            + hfx.hfx_get_class_info(c).lc + hfx.hfx_get_class_info(c).ld == 8]
    assert len(dddd) == 1
    assert st.n_quartets_pass[1][dddd[0]] == n_promoted > 0
    assert sum(st.n_quartets_pass[1]) == n_promoted  # no other class promoted

    pairs = _sample_pairs(s, np.random.default_rng(2009_03555 + 400))
    blocks, W1, W0, n = oracle.K_shell_pairs(oracle.Basis(s), P, pairs, kernel=oracle.KERNEL_ERFC,
                                             omega=0.11, screen=True, tau=1e-8, density_screen=True, eps=1e-8)
    assert n > 0
    fo = s.func_off
    kmax = max(np.abs(b).max() for b in blocks)
    worst = 0.0
    for (I, J), kb, w1, w0 in zip(pairs, blocks, W1, W0):
        got = K[fo[I]:fo[I + 1], fo[J]:fo[J + 1]]
        err = np.abs(got - kb)
        bound = 2e-4 * w1 + 256e-13 * w0 + 1e-14
        assert np.all(err <= bound), ((I, J), float(err.max()), float((err / bound).max()))
        worst = max(worst, float(err.max()))
    assert worst <= 1e-7 * kmax, (worst, kmax)
