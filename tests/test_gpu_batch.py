"""Batched builds (several systems per launch, CUDA-graph capture, autotuner):
each member's K and E_x equal its stand-alone build (FP64: |dK| <= 1e-12;
mixed: |dE_x| <= 1e-9, the same arithmetic in a different atomic order), the
graph replays with new P/K pointers, and the autotuned shapes leave results
unchanged."""
import numpy as np
import pytest

import synth
from gpu_helpers import mask_dense, pattern_mask

pytestmark = pytest.mark.gpu


def _systems():
    out = []
    for n, seed in ((3, 41), (5, 42), (7, 43), (4, 44)):
        s = synth.ch_cluster(n, seed)
        mask = pattern_mask(s, 6.0)
        P = synth.density_matrix(s, seed) * mask_dense(s, mask)
        out.append((s, mask, P))
    return out


def _setup(precision):
    import torch
    from paper_2009_03555_gb300 import hfx
    opts = hfx.make_opts(kernel=hfx.HFX_KERNEL_ERFC, precision=precision)
    mem = []
    for s, mask, P in _systems():
        b = hfx.Basis(s)
        q = hfx.Quartets(b, opts, mask)
        Pv = torch.empty(q.n_values, dtype=torch.float64, device="cuda")
        q.pack(torch.from_numpy(P).cuda(), Pv)
        mem.append((b, q, Pv, torch.empty_like(Pv)))
    return mem


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_equals_single(precision, use_graph):
    import torch
    from paper_2009_03555_gb300 import hfx
    mem = _setup(precision)
    ref_K, ref_E = [], []
    for b, q, Pv, Kv in mem:
        q.build_K(Pv, Kv)
        ref_E.append(q.exchange_energy(Pv, Kv))
        ref_K.append(Kv.clone())
    batch = hfx.Batch([m[1] for m in mem])
    Ks = [torch.full_like(m[3], np.nan) for m in mem]
    for rep in range(2):  # second build replays the captured graph
        batch.build_K([m[2] for m in mem], Ks, use_graph=use_graph)
        E = batch.energies()
        for i in range(len(mem)):
            dK = (Ks[i] - ref_K[i]).abs().max().item()
            assert dK <= (1e-12 if precision == 0 else 1e-9), (rep, i, dK)
            assert abs(E[i] - ref_E[i]) <= 1e-9 * abs(ref_E[i]) + 1e-12, (rep, i, E[i], ref_E[i])
    st = batch.stats()
    assert sum(st.n_quartets_computed) > 0


def test_graph_replay_follows_new_pointers():
    import torch
    from paper_2009_03555_gb300 import hfx
    mem = _setup(0)
    batch = hfx.Batch([m[1] for m in mem])
    K1 = [torch.empty_like(m[3]) for m in mem]
    batch.build_K([m[2] for m in mem], K1, use_graph=True)
    E1 = batch.energies()
    # K is linear in P; -P keeps every |P|-based screening decision
    P2 = [-m[2] for m in mem]
    K2 = [torch.empty_like(m[3]) for m in mem]
    batch.build_K(P2, K2, use_graph=True)
    E2 = batch.energies()
    for i in range(len(mem)):
        assert (K2[i] + K1[i]).abs().max().item() <= 1e-12 * max(1.0, K1[i].abs().max().item())
        assert E2[i] == pytest.approx(E1[i], rel=1e-12)


def test_autotune_keeps_results():
    import torch
    from paper_2009_03555_gb300 import hfx
    mem = _setup(1)
    batch = hfx.Batch([m[1] for m in mem])
    Ks = [torch.empty_like(m[3]) for m in mem]
    batch.build_K([m[2] for m in mem], Ks, use_graph=False)
    E0 = batch.energies()
    batch.autotune([m[2] for m in mem], Ks)
    nb, grid = batch.tuning()
    assert set(nb[nb > 0].tolist()) <= {32, 128, 512} and np.all(grid[nb > 0] > 0)
    batch.build_K([m[2] for m in mem], Ks, use_graph=True)
    E1 = batch.energies()
    np.testing.assert_allclose(E1, E0, rtol=0, atol=1e-9)
