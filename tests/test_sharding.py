"""Spectral sharding across ranks (host logic, CPU, gloo): the ranks' grid
ranges partition the grid (contiguous on tile boundaries, or chunks dealt
round-robin), and the sum of their partial fluxes (each with the whole
grid's trapezoid weights) over a 2-rank gloo group equals the unsharded
flux."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2604_11856_gb300.solver import shard_range, shard_ranges


@pytest.mark.parametrize("n,world", [(1_000_000, 2), (1_000_000, 8), (65536, 3), (1000, 4), (513, 2)])
def test_shards_partition_the_grid(n, world):
    parts = [shard_range(n, r, world) for r in range(world)]
    k = 0
    for k0, nk in parts:
        assert k0 == k and nk >= 0
        assert k0 % 512 == 0 or k0 == n
        k += nk
    assert k == n


@pytest.mark.parametrize("n,world,chunk", [(1_000_000, 2, 65536), (1_000_000, 3, 65536), (1000, 4, 300),
                                           (513, 2, None), (65536, 8, None)])
def test_shard_ranges_cover_the_grid_once(n, world, chunk):
    cover = np.zeros(n, np.int64)
    for r in range(world):
        for k0, nk in shard_ranges(n, r, world, chunk):
            assert nk > 0
            cover[k0:k0 + nk] += 1
    assert np.all(cover == 1)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out, chunk):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2604_11856_gb300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    grid = synth.Grid(50.0, 2000.0, 20001)
    rng = np.random.default_rng(5)
    qlam = rng.uniform(0.0, 3.0, (3, grid.n))           # three surface points
    part = torch.zeros(3, dtype=torch.float64)
    for k0, nk in shard_ranges(grid.n, rank, world, chunk):
        part += torch.tensor([oracle.spectral_integral(qlam[p, k0:k0 + nk], grid, k0) for p in range(3)],
                             dtype=torch.float64)
    dist.all_reduce(part, op=dist.ReduceOp.SUM)
    full = [oracle.spectral_integral(qlam[p], grid, 0) for p in range(3)]
    out[rank] = (part.numpy().tolist(), full)
    dist.destroy_process_group()


@pytest.mark.parametrize("chunk", [None, 4096])
def test_sharded_flux_sum_gloo(chunk):
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, port, out, chunk), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        got, full = out[r]
        np.testing.assert_allclose(got, full, rtol=1e-13)
