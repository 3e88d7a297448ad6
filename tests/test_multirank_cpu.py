"""Multi-rank paths on CPU ranks (gloo, world size 2, 127.0.0.1).

* The benchmark's N > 1 timing: every rank times its own replica; the step
  time is the maximum over ranks (all-reduce MAX), the same on every rank.
* The sharding of one build across ranks (interleaved static split of the
  canonical bra pairs, one sum all-reduce of K; the paper's distribution of
  batched ERIs over processes with an MPI_ALLREDUCE of the exchange matrix,
  Sec. 3, Algorithm 4): each rank runs the oracle on its share of the bra
  pairs, and the all-reduced K equals the oracle's K of the whole system.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle
        import synth
        ms = bench.max_over_ranks(10.0 * (rank + 1), world, torch.device("cpu"))
        s = synth.ch_cluster(3, 98, nprim=2)
        P = synth.density_matrix(s, 98, cutoff=6.0)
        kw = dict(kernel=oracle.KERNEL_ERFC, screen=True, tau=1e-8, density_screen=True, eps=1e-8)
        K, n = oracle.build_K(oracle.Basis(s), P, bra_stride=world, bra_offset=rank, nthreads=1, **kw)
        t = torch.from_numpy(K)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        nt = torch.tensor([n], dtype=torch.int64)
        dist.all_reduce(nt, op=dist.ReduceOp.SUM)
        np.save(os.path.join(out_dir, f"r{rank}.npy"), t.numpy())
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as fh:
            fh.write(f"{ms} {int(nt.item())} {n}\n")
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_and_sharded_build(tmp_path):
    import oracle
    import synth
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    s = synth.ch_cluster(3, 98, nprim=2)
    P = synth.density_matrix(s, 98, cutoff=6.0)
    kw = dict(kernel=oracle.KERNEL_ERFC, screen=True, tau=1e-8, density_screen=True, eps=1e-8)
    Kfull, nfull = oracle.build_K(oracle.Basis(s), P, nthreads=1, **kw)
    shares = []
    for r in range(world):
        ms, ntot, n = open(tmp_path / f"r{r}.txt").read().split()
        assert float(ms) == 20.0            # the slowest rank's time on every rank
        assert int(ntot) == nfull           # the shares partition the canonical quartets
        shares.append(int(n))
        np.testing.assert_allclose(np.load(tmp_path / f"r{r}.npy"), Kfull, rtol=0,
                                   atol=1e-13 * np.abs(Kfull).max())
    assert all(x > 0 for x in shares)
