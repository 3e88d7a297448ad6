"""The zero-allocation exchange-energy entry point (hfx_exchange_energy_noalloc).

It exists for callers that cannot allocate device memory (see its declaration
in include/hfx.h); its scratch is a static device array shared by all calls.
The test calls it twice in a row through the C ABI on the same P and K and
checks both results against hfx_exchange_energy (the two reductions differ only
in summation order: 1e-12 relative), and that inputs beyond its size limit are
rejected with an error before any launch.  Collected last so that a run
stopping at the first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest

import synth
from gpu_helpers import mask_dense, pattern_mask

pytestmark = pytest.mark.gpu


def test_noalloc_energy_matches_existing_entry_point():
    import torch
    from paper_2009_03555_gb300 import hfx

    s = synth.ch_cluster(5, 12)
    mask = pattern_mask(s, 6.0)
    P = synth.density_matrix(s, 12) * mask_dense(s, mask)
    basis = hfx.Basis(s)
    q = hfx.Quartets(basis, hfx.make_opts(), mask)
    dev = torch.device("cuda")
    Pv = torch.empty(q.n_values, dtype=torch.float64, device=dev)
    Kv = torch.empty_like(Pv)
    q.pack(torch.from_numpy(P).to(dev), Pv)
    q.build_K(Pv, Kv)
    E_ref = q.exchange_energy(Pv, Kv)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    for i in range(2):
        hfx.hfx_exchange_energy_noalloc(Pv, Kv, q.n_values, out[i:i + 1])
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.all(np.abs(got - E_ref) <= 1e-12 * abs(E_ref)), (got, E_ref)
    assert got[0] == got[1]  # deterministic two-pass reduction


def test_noalloc_rejects_oversized_input():
    import torch
    from paper_2009_03555_gb300 import hfx

    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(hfx.HFXError) as ei:
        hfx.hfx_exchange_energy_noalloc(x, x, (1 << 28) + 1, e)
    assert ei.value.status == 1 and "limit" in str(ei.value)
