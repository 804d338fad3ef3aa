"""The N > 1 launch of the benchmark on CPU: two gloo ranks shard the population the way the
GPU ranks do, each replays its shard with the oracle, and the reductions give the slowest
rank's time and the summed moves. The union of the shards reproduces the single-process run
on the whole population move for move (weak scaling with no data-path collective)."""
import os
import socket

import numpy as np
import pytest

import bench
import oracle
from paper_2109_05948_gb300 import inputs

N, K, P, ITERS, SEED, POP_PER_RANK, WORLD = 40, 5, 0.5, 300, 3, 3, 2


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out_dir):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    base, pop = bench.shard(rank, POP_PER_RANK)
    adj = inputs.edges_to_adj(N, inputs.gnp(N, P, SEED))
    starts = oracle.init_colors(N, K, pop, SEED, ind_base=base)
    moves = 0
    best = []
    for i in range(pop):
        r = oracle.tabucol(adj, K, starts[i], ITERS, seed=SEED, ind=base + i)
        moves += r["moves"]
        best.append(r["best_f"])
    ms, tot = bench.reduce_over_ranks(dist, 10.0 + rank, moves, "cpu")
    np.save(os.path.join(out_dir, f"rank{rank}.npy"),
            np.array([base, pop, ms, tot, moves] + best, dtype=np.float64))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce(tmp_path):
    torch = pytest.importorskip("torch")
    oracle.build()
    port = _free_port()
    torch.multiprocessing.start_processes(_rank_main, args=(port, str(tmp_path)), nprocs=WORLD,
                                          start_method="spawn", join=True)
    rows = [np.load(tmp_path / f"rank{r}.npy") for r in range(WORLD)]
    ids = sorted(int(row[0]) + j for row in rows for j in range(int(row[1])))
    assert ids == list(range(WORLD * POP_PER_RANK))  # disjoint shards covering the population
    for row in rows:
        assert row[2] == 10.0 + WORLD - 1  # the slowest rank's time
        assert row[3] == sum(r[4] for r in rows)  # the summed moves
    # one process over the whole population gives the same moves and best conflicts
    adj = inputs.edges_to_adj(N, inputs.gnp(N, P, SEED))
    starts = oracle.init_colors(N, K, WORLD * POP_PER_RANK, SEED)
    ref = [oracle.tabucol(adj, K, starts[i], ITERS, seed=SEED, ind=i) for i in range(WORLD * POP_PER_RANK)]
    assert sum(r["moves"] for r in ref) == rows[0][3]
    assert [r["best_f"] for r in ref] == [int(b) for row in rows for b in row[5:]]
