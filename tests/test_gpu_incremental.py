"""Incremental exchange builds (hfx_build_K_delta): K(P2) = K(P1) + K(P2 - P1),
the exchange matrix being linear in the density (Eq. H-HFX).

* Schwarz screening only: the composed K equals the full build of P2 to
  rounding (FP64, 1e-12 of the largest element).
* With density screening the difference build screens on the shell maxima of
  |P2 - P1| (Eq. dmscreening): the composed K equals the oracle's K(P1) + K(dP)
  under the same screening element by element (1e-10), and the difference
  build evaluates fewer quartets than a full build.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import mask_dense, pattern_mask

pytestmark = pytest.mark.gpu


def _system(seed):
    s = synth.ch_cluster(4, seed)
    mask = pattern_mask(s, 8.0)
    P1 = synth.density_matrix(s, seed) * mask_dense(s, mask)
    P2 = synth.perturb_density(P1, np.random.default_rng(seed), rel=1e-3)
    return s, mask, P1, P2


def _gpu(s, mask, P1, P2, **opt_kw):
    """K(P1) + K(P2 - P1) through hfx_build_K_delta, K(P2) through hfx_build_K,
    and the quartets evaluated by each build."""
    import torch
    from paper_2009_03555_gb300 import hfx

    q = hfx.Quartets(hfx.Basis(s), hfx.make_opts(**opt_kw), mask)
    dev = torch.device("cuda")

    def values(P):
        v = torch.empty(q.n_values, dtype=torch.float64, device=dev)
        q.pack(torch.from_numpy(np.ascontiguousarray(P)).to(dev), v)
        return v

    P1v, P2v, dPv = values(P1), values(P2), values(P2 - P1)
    K2 = torch.empty_like(P2v)
    q.build_K(P2v, K2)
    n_full = sum(q.stats().n_quartets_computed)
    K = torch.empty_like(P1v)
    q.build_K(P1v, K)
    q.build_K_delta(dPv, K)
    n_delta = sum(q.stats().n_quartets_computed)

    def dense(v):
        d = torch.empty((s.n_bf, s.n_bf), dtype=torch.float64, device=dev)
        q.unpack(v, d)
        return d.cpu().numpy()

    torch.cuda.synchronize()
    return dense(K), dense(K2), n_full, n_delta


def test_delta_equals_full_build_without_density_screening():
    s, mask, P1, P2 = _system(41)
    K, K2, n_full, n_delta = _gpu(s, mask, P1, P2, density_screen=False)
    assert n_delta == n_full  # the same pattern: the same quartets survive
    assert np.abs(K - K2).max() <= 1e-12 * np.abs(K2).max()


def test_delta_with_density_screening_matches_oracle():
    s, mask, P1, P2 = _system(42)
    K, _, n_full, n_delta = _gpu(s, mask, P1, P2, density_screen=True)
    kw = dict(kernel=oracle.KERNEL_ERFC, screen=True, tau=1e-8, density_screen=True, eps=1e-8)
    b = oracle.Basis(s)
    K1o, _ = oracle.build_K(b, P1, **kw)
    Kdo, n_d = oracle.build_K(b, P2 - P1, **kw)
    assert n_delta == n_d < n_full
    ref = K1o + Kdo
    assert np.abs(K - ref).max() <= 1e-10, np.abs(K - ref).max()
