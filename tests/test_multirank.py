"""The multi-rank path on CPU (gloo, world size 2): ray shards traced by
separate ranks add up to the single-process result, and bench.py's
reduction takes the slowest rank's time and the sum of the work."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    import scenes
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    per = 1500
    rng_kw, n_total = bench.shard(rank, world, per)
    sc = scenes.shoebox(n_rays=n_total, n_bounces=15)
    ids = np.arange(rng_kw["ray_begin"], rng_kw["ray_begin"] + rng_kw["ray_count"])
    tr = oracle.trace(oracle.OracleScene(sc, tree=False), ray_ids=ids, threads=2)
    H = torch.tensor(oracle.rir(oracle.image_sources(sc, tr), 1, sc.fs, duration=0.3))
    dist.all_reduce(H, op=dist.ReduceOp.SUM)            # the merge of shard histograms
    t_max, e2e_max, q, e2e_q = bench.reduce_over_ranks(dist, torch, torch.device("cpu"), 1.0 + rank, 2.0 - rank,
                                                       tr.queries, 10 * (rank + 1))
    if rank == 0:
        np.save(os.path.join(out_dir, "merged.npy"), H.numpy())
        np.save(os.path.join(out_dir, "reduced.npy"), np.array([t_max, e2e_max, q, e2e_q]))
        np.save(os.path.join(out_dir, "q0.npy"), np.array([tr.queries]))
    dist.barrier()
    dist.destroy_process_group()


def test_shards_merge_over_gloo(tmp_path):
    import oracle
    import scenes
    world, per = 2, 1500
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    merged = np.load(tmp_path / "merged.npy")
    sc = scenes.shoebox(n_rays=world * per, n_bounces=15)
    tr = oracle.trace(oracle.OracleScene(sc, tree=False), threads=2)
    full = oracle.rir(oracle.image_sources(sc, tr), 1, sc.fs, duration=0.3)
    assert np.allclose(merged, full, rtol=1e-12, atol=1e-18)
    t_max, e2e_max, q, e2e_q = np.load(tmp_path / "reduced.npy")
    assert t_max == 2.0 and e2e_max == 2.0 and e2e_q == 30
    assert q == tr.queries                               # queries of both shards add up
