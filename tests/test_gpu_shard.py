"""Sharded builds (hfx_build_K_shard): the shares of n ranks, run one after
another on one GPU, add up to the whole build -- the sum all-reduce of the
paper's distributed construction (Sec. 3, Algorithm 4) done on the host here.
Every quartet is evaluated by exactly one share (counts add up), and the summed
K equals hfx_build_K's to rounding (summation order differs)."""
import numpy as np
import pytest

import synth
from gpu_helpers import mask_dense, pattern_mask

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_ranks", [2, 3, 8])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_shards_sum_to_whole_build(n_ranks, prec):
    import torch
    from paper_2009_03555_gb300 import hfx
    s = synth.ch_cluster(6, 21)
    mask = pattern_mask(s, 8.0)
    P = synth.density_matrix(s, 21) * mask_dense(s, mask)
    p = hfx.HFX_PREC_FP64 if prec == "fp64" else hfx.HFX_PREC_MIXED
    opts = hfx.make_opts(kernel=hfx.HFX_KERNEL_ERFC, precision=p, fp64_promote_bound=1e-4, promote_min_l=8,
                         n_block=7)
    q = hfx.Quartets(hfx.Basis(s), opts, mask)
    dev = torch.device("cuda")
    Pv = torch.empty(q.n_values, dtype=torch.float64, device=dev)
    q.pack(torch.from_numpy(P).to(dev), Pv)
    K = torch.empty_like(Pv)
    q.build_K(Pv, K)
    n_all = sum(q.stats().n_quartets_computed)
    Ksum = torch.zeros_like(Pv)
    Kr = torch.empty_like(Pv)
    n_sum = 0
    for r in range(n_ranks):
        q.build_K_shard(Pv, Kr, r, n_ranks)
        Ksum += Kr
        n_r = sum(q.stats().n_quartets_computed)
        assert n_r < n_all
        n_sum += n_r
    torch.cuda.synchronize()
    assert n_sum == n_all
    scale = float(K.abs().max())
    assert float((Ksum - K).abs().max()) <= 1e-12 * scale
    assert abs(q.exchange_energy(Pv, Ksum) - q.exchange_energy(Pv, K)) <= 1e-12 * abs(q.exchange_energy(Pv, K))


def test_shard_rejects_bad_rank():
    import torch
    from paper_2009_03555_gb300 import hfx
    s, P = synth.config0()
    q = hfx.Quartets(hfx.Basis(s), hfx.make_opts(kernel=0, screen=False, density_screen=False),
                     np.ones((s.n_atoms, s.n_atoms), dtype=bool))
    v = torch.zeros(q.n_values, dtype=torch.float64, device="cuda")
    with pytest.raises(hfx.HFXError):
        q.build_K_shard(v, v, 2, 2)
