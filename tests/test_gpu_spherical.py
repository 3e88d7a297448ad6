"""Spherical-harmonic layout (hfx_opts.spherical; Sec. 2: the Cartesian
integrals are transformed to real spherical harmonics): P and K hold 2l+1
solid harmonics per shell.  Against the oracle's Cartesian K transformed with
the tests' own (pinned) transform, K_sph = T K(T^T P_sph T) T^T:
FP64 |dK|max <= 1e-10 and |dE_x| <= 1e-9 |E_x|; mixed: the Cartesian mixed build
transformed (1e-12), and |dE_x| <= 1e-6 Ha with FP64 promotion above 1e-5.
Also the rotational-symmetry pin on the library's own output: for an s and a d
shell on one centre and P = the s projector, the d block of K is a multiple of
the identity."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import mask_dense, pattern_mask, run_gpu_K
from spherical_helpers import spherical_K, system_transform

pytestmark = pytest.mark.gpu


def _sph_mask(sysobj, T, mask):
    """Spherical-layout dense mask of an atom-pair pattern."""
    Mc = mask_dense(sysobj, mask)
    return (np.abs(T) @ Mc @ np.abs(T).T) > 0


def _gpu_sph(sysobj, P_sph, mask, **kw):
    import torch
    from paper_2009_03555_gb300 import hfx
    q = hfx.Quartets(hfx.Basis(sysobj), hfx.make_opts(spherical=True, **kw), mask)
    dev = torch.device("cuda")
    Pd = torch.from_numpy(np.ascontiguousarray(P_sph)).to(dev)
    Pv = torch.empty(q.n_values, dtype=torch.float64, device=dev)
    Kv = torch.empty_like(Pv)
    q.pack(Pd, Pv)
    q.build_K(Pv, Kv)
    E = q.exchange_energy(Pv, Kv)
    Kd = torch.empty_like(Pd)
    q.unpack(Kv, Kd)
    torch.cuda.synchronize()
    return Kd.cpu().numpy(), E, q


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_spherical_K_matches_transformed_oracle(prec):
    from paper_2009_03555_gb300 import hfx
    s = synth.ch_cluster(4, 17)
    mask = pattern_mask(s, 6.0)
    T = system_transform(s)
    n_s = T.shape[0]
    rng = np.random.default_rng(17)
    C, _ = np.linalg.qr(rng.standard_normal((n_s, 6)))
    Ms = _sph_mask(s, T, mask)
    P_sph = (C @ C.T) * Ms
    kw = dict(kernel=oracle.KERNEL_ERFC, omega=0.11, screen=True, tau=1e-8, density_screen=True, eps=1e-8)
    b = oracle.Basis(s)
    Kref = spherical_K(lambda Pc: oracle.build_K(b, Pc, **kw)[0], T, P_sph)
    Eref = -0.5 * float(np.sum(P_sph * Kref))
    p = hfx.HFX_PREC_FP64 if prec == "fp64" else hfx.HFX_PREC_MIXED
    K, E, q = _gpu_sph(s, P_sph, mask, prim_cutoff=1e-14, precision=p, **kw)
    assert q.n_values == int(Ms.sum())
    if prec == "fp64":
        assert np.abs((K - Kref) * Ms).max() <= 1e-10
        assert np.all(K[~Ms] == 0)
        assert abs(E - Eref) <= 1e-9 * abs(Eref)
    else:
        # the mixed arithmetic of the Cartesian build of T^T P T, transformed
        Kc, Ec, _ = run_gpu_K(s, T.T @ P_sph @ T, mask=mask, prim_cutoff=1e-14, precision=p, **kw)
        assert abs(E - Ec) <= 1e-12 * abs(Ec)
        assert np.abs(K - T @ Kc @ T.T).max() <= 1e-12 * np.abs(K).max()
        # with the largest quartets promoted to FP64, within 1e-6 Ha of the oracle
        _, E2, _ = _gpu_sph(s, P_sph, mask, prim_cutoff=1e-14, precision=p, fp64_promote_bound=1e-5, **kw)
        assert abs(E2 - Eref) <= 1e-6


def test_spherical_d_block_is_isotropic():
    s = synth.System(name="sd", atom_Z=np.array([6], dtype=np.int32), atom_xyz=np.zeros((1, 3)),
                     shell_atom=np.array([0, 0], dtype=np.int32), shell_l=np.array([0, 2], dtype=np.int32),
                     prim_off=np.array([0, 2, 5], dtype=np.int32),
                     alpha=np.array([3.0, 0.4, 5.0, 1.1, 0.3]), coef=np.array([0.5, 0.7, 0.3, 0.6, 0.8]))
    P = np.zeros((6, 6))
    P[0, 0] = 1.0  # the s function only: K_dd = (d_m s | d_m' s)
    K, _, _ = _gpu_sph(s, P, np.ones((1, 1), dtype=bool), kernel=0, screen=False, density_screen=False,
                       prim_cutoff=0.0)
    Kdd = K[1:, 1:]
    d = np.diag(Kdd)
    assert np.abs(Kdd - np.diag(d)).max() <= 1e-13 * d.max()
    assert np.ptp(d) <= 1e-13 * d.max()
