"""Multi-rank host path on CPU: world_size 2 over gloo, no GPU.

Each rank simulates its contiguous share of trajectories (here with the oracle,
standing in for one GPU per rank), the shares are gathered host-side, and the
result must equal a single-process run: trajectories are independent and their
draws are keyed by global trajectory index.
"""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads as W
from paper_2204_11404_gb300.shard import interleaved_index, run_sharded, shard_range

D, R, GATES = 3, 2, "cr"


def oracle_run(first, n):
    from oracle import run_trajectory
    syn, bits, log = [], [], []
    for t in range(first, first + n):
        o = run_trajectory(D, R, GATES, "reduced", W.STRESS, seed=9, traj=t)
        syn.append(o["syndromes"])
        bits.append(o["data_bits"])
        log.append(o["raw_logical"])
    return (np.array(syn, dtype=np.uint8).reshape(n, R + 1, D * D - 1),
            np.array(bits, dtype=np.uint8).reshape(n, D * D), np.array(log, dtype=np.uint8))


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = run_sharded(oracle_run, 5, 13, rank, world)
        np.savez(os.path.join(out_dir, "rank%d.npz" % rank), *got)
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_shard_ranges_partition():
    for n in (0, 1, 7, 13, 100):
        for world in (1, 2, 3, 8):
            spans = [shard_range(5, n, r, world) for r in range(world)]
            assert spans[0][0] == 5 and spans[-1][1] == 5 + n
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))


def test_interleaved_indices_disjoint():
    seen = set()
    for rank in range(4):
        for step in range(36):
            seen.add((step % 9, interleaved_index(step, 9, rank, 4)))
    assert len(seen) == 4 * 36


def test_two_rank_gloo_gather_equals_single_process(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    ref = oracle_run(5, 13)
    for rank in range(world):
        z = np.load(os.path.join(tmp_path, "rank%d.npz" % rank))
        for i, r in enumerate(ref):
            assert (z["arr_%d" % i] == r).all()
