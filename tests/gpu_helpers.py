"""Shared helpers of the GPU tests: run the CUDA path through the C ABI on a
seeded system and bring the dense K back for comparison with the oracle."""
import numpy as np

import synth


def run_gpu_K(sysobj, P, mask=None, **opt_kw):
    """Build K (dense numpy, FP64) and E_x with the CUDA library."""
    import torch
    from paper_2009_03555_gb300 import hfx

    if mask is None:
        mask = np.ones((sysobj.n_atoms, sysobj.n_atoms), dtype=bool)
    basis = hfx.Basis(sysobj)
    q = hfx.Quartets(basis, hfx.make_opts(**opt_kw), mask)
    dev = torch.device("cuda")
    Pd = torch.from_numpy(np.ascontiguousarray(P)).to(dev)
    Pv = torch.empty(q.n_values, dtype=torch.float64, device=dev)
    Kv = torch.empty(q.n_values, dtype=torch.float64, device=dev)
    q.pack(Pd, Pv)
    q.build_K(Pv, Kv)
    E = q.exchange_energy(Pv, Kv)
    Kd = torch.empty_like(Pd)
    q.unpack(Kv, Kd)
    torch.cuda.synchronize()
    return Kd.cpu().numpy(), E, q


def pattern_mask(sysobj, cutoff):
    return synth.atom_pair_mask(sysobj, cutoff)


def mask_dense(sysobj, mask):
    return synth.expand_atom_mask(sysobj, mask)
