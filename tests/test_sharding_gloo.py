"""Chain sharding over two gloo ranks on the CPU.

Each rank owns a contiguous chain-id range and runs its chains (the CPU
oracle stands in for the device here); the gathered result must equal one
process running every chain -- the random streams are keyed by chain id, so
the partition cannot change any chain."""
import os
import socket

import numpy as np
import pytest

from _common import ROOT  # noqa: F401  (sys.path set-up)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _run_chains(start, count, n_total):
    import crbm_workloads as wl
    from oracle import chain
    W, hb, vb = wl.gaussian_crbm(2, 3, 0.3)
    T = wl.ising_ladder(n_total, 4)[start:start + count]
    ch = chain.make_chains(chain.ISING, W, hb, vb, 6, T, (1.0,), 11, np.arange(start, start + count))
    chain.run(ch, 6)
    return np.concatenate([wl.pack_bits(ch.v).astype(np.float64), ch.obs, ch.accepts[:, None]], axis=1)


def _worker(rank, world, port, n_total, out_path):
    import torch.distributed as dist
    from paper_2008_05401_gb300.sharding import gather_rows, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    start, count = shard(n_total, rank, world)
    full = gather_rows(_run_chains(start, count, n_total), n_total)
    if rank == 0:
        np.save(out_path, full)
    dist.destroy_process_group()


def test_shard_ranges_cover_every_chain_once():
    from paper_2008_05401_gb300.sharding import shard
    for n in (0, 1, 7, 64, 1001):
        for world in (1, 2, 3, 8):
            ranges = [shard(n, r, world) for r in range(world)]
            ids = np.concatenate([np.arange(s, s + c) for s, c in ranges])
            np.testing.assert_array_equal(ids, np.arange(n))
            assert max(c for _, c in ranges) - min(c for _, c in ranges) <= 1
    with pytest.raises(ValueError):
        shard(4, 2, 2)


def test_two_gloo_ranks_equal_one_process(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    n_total = 9
    out = str(tmp_path / "full.npy")
    mp.start_processes(_worker, args=(2, _free_port(), n_total, out), nprocs=2, join=True, start_method="spawn")
    full = np.load(out)
    np.testing.assert_array_equal(full, _run_chains(0, n_total, n_total))
