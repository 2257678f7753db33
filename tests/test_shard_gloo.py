"""The N > 1 walker-sharding path on CPU: two gloo ranks, each running its
shard of walkers with offset Philox walker indices (on the CPU oracle), give
bitwise the single-process result; timings reduce by max, accumulators by sum."""
import os
import socket

import numpy as np
import pytest

import oracle
import synth
from paper_2002_07401_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, W, sweeps, out_dir):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sysm = synth.config1()
    w0 = shard.walker_offset(W, rank)
    x = np.ascontiguousarray(synth.init_walkers(sysm, W * world, seed=0)[w0:w0 + W])
    eL, _, nacc = oracle.Oracle(sysm).vmc(x, sweeps, seed=4, walker0=w0, nthreads=1)
    tmax = shard.max_over_ranks(float(rank + 1))
    tot = shard.sum_over_ranks([eL.sum(), float(nacc.sum())])
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), x=x, eL=eL, tmax=tmax, tot=tot.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_equal_single_run(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    W, sweeps, world = 6, 3, 2
    mp.spawn(_rank_main, args=(world, _free_port(), W, sweeps, str(tmp_path)), nprocs=world, join=True)
    sysm = synth.config1()
    x = np.ascontiguousarray(synth.init_walkers(sysm, W * world, seed=0))
    eL, _, nacc = oracle.Oracle(sysm).vmc(x, sweeps, seed=4, walker0=0, nthreads=1)
    parts = [np.load(os.path.join(tmp_path, f"rank{k}.npz")) for k in range(world)]
    assert np.array_equal(np.concatenate([p["x"] for p in parts]), x)
    assert np.array_equal(np.concatenate([p["eL"] for p in parts], axis=1), eL)
    for p in parts:
        assert float(p["tmax"]) == 2.0
        assert np.allclose(p["tot"], [eL.sum(), float(nacc.sum())], rtol=1e-13)


def test_walker_offset_rejects_bad_input():
    assert shard.walker_offset(4096, 3) == 12288
    with pytest.raises(ValueError):
        shard.walker_offset(0, 1)
