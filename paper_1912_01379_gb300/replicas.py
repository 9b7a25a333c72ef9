"""Multi-GPU replicas of the sampler: chains are independent, so the path
shards by chain with no data-path collective.  Each rank samples a
contiguous range of global chain ids (asm_set_stream_ids makes the random
numbers follow the global id, so the union of the shards is the unsharded
run chain by chain); the only exchange is one sum of the FP64 per-grid-point
accumulators at the end (a host-side reduction over torch.distributed, gloo
or NCCL)."""
from __future__ import annotations

import numpy as np


def shard(total_chains: int, rank: int, world: int) -> tuple[int, int]:
    """(chain_offset, chains) of `rank`: contiguous, sizes differ by at most one."""
    base, extra = divmod(total_chains, world)
    count = base + (1 if rank < extra else 0)
    offset = rank * base + min(rank, extra)
    return offset, count


def chain_moments(S1: np.ndarray, S2: np.ndarray, kept: int) -> np.ndarray:
    """Per-rank FP64 partial sums over its chains: [sum of chain means, sum of
    squared chain means, sum of second moments, number of chains] per grid point."""
    cm = np.asarray(S1, dtype=np.float64) / kept
    return np.stack([cm.sum(0), (cm * cm).sum(0), np.asarray(S2, dtype=np.float64).sum(0) / kept,
                     np.full(cm.shape[1], cm.shape[0], dtype=np.float64)])


def partial_from_average(mean_fbar, sem_fbar, ess, chains: int) -> np.ndarray:
    """The same partial sums, rebuilt from one rank's asm_average outputs
    (mean, standard error from its chain means, ESS = variance / sem^2)."""
    mean = np.asarray(mean_fbar, dtype=np.float64)
    sem2 = np.asarray(sem_fbar, dtype=np.float64) ** 2
    var = np.nan_to_num(np.asarray(ess, dtype=np.float64) * sem2)
    C = float(chains)
    return np.stack([C * mean, (C - 1.0) * C * sem2 + C * mean * mean, C * (var + mean * mean),
                     np.full(mean.shape, C)])


def combine(partial: np.ndarray, group=None) -> dict:
    """Sum the ranks' partials (all_reduce over the default or given group) and
    return <fbar>, its standard error from the chain means and the ESS."""
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.ascontiguousarray(partial))
    if dist.is_available() and dist.is_initialized():
        if dist.get_backend(group) == "nccl":
            t = t.cuda()
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    tot = t.cpu().numpy()
    C = tot[3]
    mean = tot[0] / C
    var_cm = np.maximum(tot[1] / C - mean * mean, 0.0) * C / np.maximum(C - 1, 1)
    sem = np.sqrt(var_cm / C)
    var = np.maximum(tot[2] / C - mean * mean, 0.0)
    ess = np.where(sem > 0, var / np.maximum(sem, 1e-300) ** 2, np.nan)
    return {"mean_fbar": mean, "sem_fbar": sem, "ess": ess, "chains": int(C[0])}
