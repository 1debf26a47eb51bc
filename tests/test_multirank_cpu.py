"""The N>1 path of the benchmark on CPU with the gloo backend (world size 2):
per-rank shards are independent, timing is the max over ranks, and the
element-local operator needs no exchange between shards."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mesh = bench.shard_seed_workload(rank, "cpu", E=6)
    w = oracle.sem_ax(mesh.u, mesh.G, mesh.D)
    t = bench.max_over_ranks(0.5 + rank, world)
    bench.barrier(world)
    np.save(os.path.join(out_dir, f"u{rank}.npy"), mesh.u.numpy())
    np.save(os.path.join(out_dir, f"G{rank}.npy"), mesh.G.numpy())
    np.save(os.path.join(out_dir, f"w{rank}.npy"), w)
    np.save(os.path.join(out_dir, f"t{rank}.npy"), np.array([t]))
    dist.destroy_process_group()


def test_two_rank_shards_and_max_timing(tmp_path, oracle_mod):
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    u = [np.load(tmp_path / f"u{r}.npy") for r in range(2)]
    G = [np.load(tmp_path / f"G{r}.npy") for r in range(2)]
    w = [np.load(tmp_path / f"w{r}.npy") for r in range(2)]
    t = [float(np.load(tmp_path / f"t{r}.npy")[0]) for r in range(2)]
    assert t == [1.5, 1.5]                               # max over ranks on every rank
    assert not np.array_equal(u[0], u[1])                 # independent shards
    import sem_inputs as si
    D = si.gll_diff_matrix(7)
    whole = oracle_mod.sem_ax(np.concatenate(u), np.concatenate(G), D)
    assert np.array_equal(whole, np.concatenate(w))       # no exchange step is needed
