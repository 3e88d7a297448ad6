"""The serving layer (continuous batching of SCF-like requests).

Each request is one system with a short sequence of density matrices (P
perturbed by 1e-3 per build, the pattern kept).  Checked here:
  * a request served in a mix with others gives the results it gives alone
    (FP64: |dE| <= 1e-12 |E|, |dK| <= 1e-12 max|K|, the same arithmetic in a
    different atomic order; mixed: 1e-9, as for batches);
  * every build equals a direct hfx_build_K of the same P, and the first
    build of a small system equals the oracle (FP64 parity, 1e-9 |E|);
  * admission by device memory: under a budget that holds one request at a
    time the server runs them one by one; a request larger than the whole
    budget fails with HFX_ERR_OOM and the others still complete;
  * CUDA-graph replay gives the same energies as plain launches.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _requests(n_builds=(3, 2, 4)):
    """Three small systems of different shapes (chain, slab, cluster)."""
    systems = [synth.ch_chain(10, sub=1), synth.ch_slab(9, sub=2), synth.ch_cluster(6, 4, sub=3)]
    out = []
    for k, (s, nb) in enumerate(zip(systems, n_builds)):
        mask = synth.atom_pair_mask(s, 8.0)
        P0 = synth.density_matrix(s, 4, sub=k) * synth.expand_atom_mask(s, mask)
        rng = np.random.default_rng(2009_03555 + 40 + k)
        Ps = [P0]
        for _ in range(nb - 1):
            Ps.append(synth.perturb_density(Ps[-1], rng))
        out.append((s, mask, Ps))
    return out


def _opts(precision):
    from paper_2009_03555_gb300 import hfx
    return hfx.make_opts(kernel=hfx.HFX_KERNEL_ERFC, omega=0.11, screen=True, tau=1e-8, density_screen=True,
                         eps=1e-8, precision=precision)


def _run(server, reqs, opts, order=None):
    from paper_2009_03555_gb300 import hfx
    order = list(range(len(reqs))) if order is None else order
    tickets = {}
    for i in order:
        s, mask, Ps = reqs[i]
        tickets[i] = server.submit(s, mask, opts, Ps)
    for _ in range(100):
        server.step()
        infos = [server.poll(t)[0] for t in tickets.values()]
        if all(x.state in (hfx.HFX_REQ_DONE, hfx.HFX_REQ_FAILED) for x in infos):
            break
    res = {}
    for i, t in tickets.items():
        info, E = server.poll(t)
        res[i] = (info, E, server.K_values(t).copy())
    return res


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
def test_alone_equals_mix(precision, tol):
    from paper_2009_03555_gb300 import hfx
    reqs = _requests()
    opts = _opts(precision)
    alone = {}
    for i in range(len(reqs)):
        srv = hfx.Server()
        alone[i] = _run(srv, reqs[i:i + 1], opts)[0]
        del srv
    srv = hfx.Server()
    mix = _run(srv, reqs, opts, order=[1, 0, 2])
    info = srv.info()
    assert info.max_active_seen == 3 and info.n_active == 0 and info.used_bytes == 0
    for i in range(len(reqs)):
        ia, Ea, Ka = alone[i]
        im, Em, Km = mix[i]
        assert ia.state == im.state == hfx.HFX_REQ_DONE
        assert len(Ea) == len(Em) == len(reqs[i][2])
        np.testing.assert_allclose(Em, Ea, rtol=tol, atol=0)
        assert np.abs(Km - Ka).max() <= tol * np.abs(Ka).max()
        assert im.t_submit <= im.t_admit <= im.t_done


def test_builds_match_direct_api_and_oracle():
    import torch
    from paper_2009_03555_gb300 import hfx
    reqs = _requests()
    opts = _opts(0)
    srv = hfx.Server()
    res = _run(srv, reqs, opts)
    for i, (s, mask, Ps) in enumerate(reqs):
        info, E, Kv = res[i]
        b = hfx.Basis(s)
        q = hfx.Quartets(b, opts, mask)
        Pv = torch.empty(q.n_values, dtype=torch.float64, device="cuda")
        Kd = torch.empty_like(Pv)
        for k, P in enumerate(Ps):
            q.pack(torch.from_numpy(P).cuda(), Pv)
            q.build_K(Pv, Kd)
            Ed = q.exchange_energy(Pv, Kd)
            assert abs(E[k] - Ed) <= 1e-12 * abs(Ed)
        np.testing.assert_allclose(Kv, Kd.cpu().numpy(), rtol=0, atol=1e-12 * np.abs(Kv).max())
    # FP64 parity of the first build of the smallest system with the oracle
    s, mask, Ps = reqs[1]
    Kref, _ = oracle.build_K(oracle.Basis(s), Ps[0], kernel=oracle.KERNEL_ERFC, omega=0.11, screen=True,
                             tau=1e-8, density_screen=True, eps=1e-8)
    Eref = oracle.exchange_energy(Ps[0], Kref)
    assert abs(res[1][1][0] - Eref) <= 1e-9 * abs(Eref)


def test_admission_by_memory():
    from paper_2009_03555_gb300 import hfx
    reqs = _requests()
    opts = _opts(1)
    est = []
    for s, mask, Ps in reqs:
        inp = hfx._SystemInput(s, mask)
        est.append(inp.setup_bytes_estimate() + 2 * 8 * inp.value_count())
    # three copies of one request under a budget of one estimate: once the
    # first is admitted (holding its actual bytes) the next estimate no longer
    # fits, so the copies run one after another, with equal results
    same = [reqs[0]] * 3
    srv = hfx.Server(mem_budget=est[0] + 1)
    res = _run(srv, same, opts)
    info = srv.info()
    assert info.max_active_seen == 1 and info.steps == 3 * len(reqs[0][2])
    assert info.peak_used_bytes <= info.mem_budget
    for i in range(3):
        assert res[i][0].state == hfx.HFX_REQ_DONE
        np.testing.assert_allclose(res[i][1], res[0][1], rtol=1e-9, atol=0)
    assert res[0][0].t_done <= res[1][0].t_admit and res[1][0].t_done <= res[2][0].t_admit
    # a request larger than the whole budget fails, the others complete
    big = int(np.argmax(est))
    srv2 = hfx.Server(mem_budget=sorted(est)[1] + 1)
    res2 = _run(srv2, reqs, opts)
    assert res2[big][0].state == hfx.HFX_REQ_FAILED and res2[big][0].status == 2
    ref = _run(hfx.Server(), reqs, opts)
    for i in range(len(reqs)):
        if i != big:
            assert res2[i][0].state == hfx.HFX_REQ_DONE
            np.testing.assert_allclose(res2[i][1], ref[i][1], rtol=1e-9, atol=0)


def test_graph_replay_equals_launches():
    from paper_2009_03555_gb300 import hfx
    reqs = _requests(n_builds=(3, 3, 3))
    opts = _opts(0)
    a = _run(hfx.Server(use_graph=False), reqs, opts)
    b = _run(hfx.Server(use_graph=True), reqs, opts)
    for i in range(len(reqs)):
        np.testing.assert_allclose(b[i][1], a[i][1], rtol=1e-12, atol=0)


def test_cancel_and_injected_setup_failure():
    """Host-side failure handling: a cancelled queued request never runs, an
    active one leaves at the next step with its memory released, and a setup
    failure injected on the host fails that request only."""
    from paper_2009_03555_gb300 import hfx
    reqs = _requests(n_builds=(3, 3, 3))
    opts = _opts(1)
    ref = _run(hfx.Server(), reqs, opts)
    srv = hfx.Server()
    t = [srv.submit(s, mask, opts, Ps) for s, mask, Ps in reqs]
    srv.inject_setup_failure(t[2], 2)   # as if its allocation had failed
    srv.cancel(t[1])                    # still queued
    assert srv.poll(t[1])[0].state == hfx.HFX_REQ_CANCELLED
    srv.step()                          # t[0] admitted and built once; t[2] fails at setup
    assert srv.poll(t[2])[0].state == hfx.HFX_REQ_FAILED and srv.poll(t[2])[0].status == 2
    assert srv.poll(t[0])[0].state == hfx.HFX_REQ_ACTIVE
    for _ in range(10):
        srv.step()
        if srv.poll(t[0])[0].state == hfx.HFX_REQ_DONE:
            break
    info, E = srv.poll(t[0])
    assert info.state == hfx.HFX_REQ_DONE
    np.testing.assert_allclose(E, ref[0][1], rtol=1e-9, atol=0)
    # an active request cancelled between steps leaves at the next one
    srv2 = hfx.Server()
    u = srv2.submit(*reqs[0][:2], opts, reqs[0][2])
    srv2.step()
    assert srv2.poll(u)[0].state == hfx.HFX_REQ_ACTIVE and srv2.info().used_bytes > 0
    srv2.cancel(u)
    srv2.step()
    ri, E2 = srv2.poll(u)
    assert ri.state == hfx.HFX_REQ_CANCELLED and ri.builds_done == 1
    assert srv2.info().used_bytes == 0 and srv2.info().n_active == 0
    srv2.release(u)


def test_incremental_server_matches_direct_delta_builds():
    """With incremental builds every build after a request's first is
    K(P_{n-1}) + K(P_n - P_{n-1}) (hfx_build_K_delta through the batched path):
    its energies equal those of the direct API's same sequence (1e-10 |E|, the
    same arithmetic in a different atomic order), stay within 1e-7 Ha of full
    builds, and the request also gives them in a mix."""
    import torch
    from paper_2009_03555_gb300 import hfx
    reqs = _requests(n_builds=(4, 3, 3))
    opts = _opts(0)
    srv = hfx.Server(incremental=True)
    res = _run(srv, reqs, opts)
    full = _run(hfx.Server(), reqs, opts)
    for i, (s, mask, Ps) in enumerate(reqs):
        q = hfx.Quartets(hfx.Basis(s), opts, mask)
        dev = torch.device("cuda")
        vals = []
        for P in Ps:
            v = torch.empty(q.n_values, dtype=torch.float64, device=dev)
            q.pack(torch.from_numpy(np.ascontiguousarray(P)).to(dev), v)
            vals.append(v)
        K = torch.empty_like(vals[0])
        q.build_K(vals[0], K)
        E = [q.exchange_energy(vals[0], K)]
        for n in range(1, len(Ps)):
            q.build_K_delta(vals[n] - vals[n - 1], K)
            E.append(q.exchange_energy(vals[n], K))
        info, Es, Ks = res[i]
        assert info.state == hfx.HFX_REQ_DONE and info.builds_done == len(Ps)
        np.testing.assert_allclose(Es, E, rtol=1e-10, atol=0)
        np.testing.assert_allclose(Es, full[i][1], rtol=0, atol=1e-7)
        assert np.abs(Ks - K.cpu().numpy()).max() <= 1e-10 * np.abs(Ks).max()


def test_periodic_request_alone_and_in_mix():
    """A periodic cell served (hfx_server_submit_periodic) gives the per-cell
    energies of the library's periodic path built directly, alone and mixed
    with molecular requests."""
    import torch
    from paper_2009_03555_gb300 import hfx
    A = np.array([[6.0, 0.0, 0.0], [1.0, 6.0, 0.0], [0.0, 1.0, 6.0]])
    cell = synth.periodic_cell(3, A, sub=35, recipe={"C": [0, 1, 2], "H": [0, 1]})
    P0 = synth.periodic_density_matrix(cell, cutoff=4.0, sub=35)
    rng = np.random.default_rng(2009_03555 + 77)
    Ps = [P0, synth.perturb_density(P0, rng), None]
    Ps[2] = synth.perturb_density(Ps[1], rng)
    per = hfx.Periodic(cell, A, r_ext=5.0, r_P=4.0)
    opts = _opts(0)
    # direct
    q = per.quartets(opts)
    dev = torch.device("cuda")
    E_dir = []
    for P in Ps:
        Pv = torch.from_numpy(per.pack(P)).to(dev)
        Kv = torch.empty_like(Pv)
        q.build_K(Pv, Kv)
        E_dir.append(q.exchange_energy(Pv, Kv))
    for mix in (False, True):
        srv = hfx.Server()
        t = srv.submit_periodic(per, opts, Ps)
        others = {}
        if mix:
            for i, (s, mask, Pm) in enumerate(_requests()):
                others[i] = srv.submit(s, mask, opts, Pm)
        for _ in range(100):
            srv.step()
            if srv.info().n_active == 0 and srv.info().n_queued == 0:
                break
        info, E = srv.poll(t)
        assert info.state == hfx.HFX_REQ_DONE, info.status
        np.testing.assert_allclose(E, E_dir, rtol=1e-12, atol=0)
        assert np.all(srv.K_values(t)[per.n_home_values:] == 0.0)
        for tt in others.values():
            assert srv.poll(tt)[0].state == hfx.HFX_REQ_DONE
