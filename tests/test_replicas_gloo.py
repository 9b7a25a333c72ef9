"""The multi-GPU path shards chains across ranks with no data-path collective;
the ranks' FP64 sums are combined once at the end.  Tested here with two
gloo ranks on the CPU: each rank samples its shard with the oracle (global
chain ids via the chain offset), and the combined average equals the
single-process run over all chains."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import oracle as O
from paper_1912_01379_gb300 import replicas, workloads as W

CHAINS, BURN, SWEEPS, SEED = 10, 20, 60, 31


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = W.small_problem(12, 30, seed=4, levels=[[0], [0, 10, 20]])
        op = O.OracleProblem(p.K, p.G, p.C, p.levels)
        off, n = replicas.shard(CHAINS, rank, world)
        r = op.run(n, BURN, SWEEPS, seed=SEED, threads=1, chain_offset=off)
        res = replicas.combine(replicas.chain_moments(r["S1"], r["S2"], r["kept"]))
        out[rank] = (res["mean_fbar"].tolist(), res["sem_fbar"].tolist(), res["chains"], r["f_final"].tolist(), off)
    finally:
        dist.destroy_process_group()


def test_shard_ranges():
    for total in (1, 7, 1024, 1025):
        for world in (1, 2, 3, 8):
            spans = [replicas.shard(total, r, world) for r in range(world)]
            assert sum(n for _, n in spans) == total
            assert all(spans[r][0] + spans[r][1] == spans[r + 1][0] for r in range(world - 1))


def test_two_gloo_ranks_reproduce_the_unsharded_run():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    p = W.small_problem(12, 30, seed=4, levels=[[0], [0, 10, 20]])
    op = O.OracleProblem(p.K, p.G, p.C, p.levels)
    whole = op.run(CHAINS, BURN, SWEEPS, seed=SEED, threads=1)
    ref = O.summarize(whole["S1"], whole["S2"], whole["kept"])
    for rank in range(2):
        mean, sem, chains, f_final, off = out[rank]
        assert chains == CHAINS
        assert np.allclose(mean, ref["mean_fbar"], rtol=1e-12, atol=0)
        assert np.allclose(sem, ref["sem_fbar"], rtol=1e-9, atol=0)
        # every chain of the shard is the same chain of the unsharded run
        f_final = np.array(f_final)
        assert np.array_equal(f_final, whole["f_final"][off:off + len(f_final)])
