"""Host-side logic of multi-GPU runs: one process per GPU, chains sharded.

Markov chains are independent, so N GPUs run N replicas of the sampling
kernel on disjoint chains with the same PEPS tensors (weak scaling: chains per
GPU fixed).  The data path has no collective.  What crosses ranks is host
bookkeeping: the timing of a step (the slowest rank sets it), the whole-job
sample rate, and the Monte Carlo energy estimate, whose sums over samples add
across ranks.  These functions take a torch.distributed process group (NCCL
on GPUs, gloo on CPU) or None for a single process.
"""

from __future__ import annotations

import math


def rank_seeds(rank: int, base_tensor_seed: int = 2, base_chain_seed: int = 102):
    """Seeds of one rank: the tensors are shared by all ranks (one wave
    function), the chains' starting configurations and Metropolis streams are
    distinct per rank."""
    return {"tensors": base_tensor_seed, "chains": base_chain_seed + rank,
            "step": lambda i: 10_000 + 1000 * i + rank}


def _tensor(x, device):
    import torch

    return torch.tensor(x, dtype=torch.float64, device=device)


def max_over_ranks(value: float, group=None, device="cpu") -> float:
    """The largest value over ranks (e.g. a step time)."""
    if group is None:
        return float(value)
    import torch.distributed as dist

    t = _tensor([value], device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sum_over_ranks(values, group=None, device="cpu"):
    """Element-wise sum over ranks of a list of floats."""
    if group is None:
        return [float(v) for v in values]
    import torch.distributed as dist

    t = _tensor(list(values), device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return [float(v) for v in t.tolist()]


def whole_job_rate(units_per_rank_step: float, steps: int, world: int, max_ms: float) -> float:
    """Units per second of the whole job: all ranks' units over the slowest
    rank's time."""
    return units_per_rank_step * steps * world / (max_ms / 1000.0)


def energy_sums(e_loc_re, n_chains: int):
    """Per-rank sums for the energy estimate: (number of samples, sum of
    E_loc, sum over chains of the chain mean, sum of squared chain means,
    number of chains).  e_loc_re holds the samples chain-major."""
    n = len(e_loc_re)
    per = n // n_chains
    s = 0.0
    cm = 0.0
    cm2 = 0.0
    for c in range(n_chains):
        m = sum(e_loc_re[c * per:(c + 1) * per]) / per
        cm += m
        cm2 += m * m
    for v in e_loc_re:
        s += v
    return [float(n), s, cm, cm2, float(n_chains)]


def energy_estimate(sums, group=None, device="cpu"):
    """Global <E_loc> and its standard error from per-rank energy_sums: the
    error treats chain means as independent (the same estimator a single
    process uses over all chains)."""
    n, s, cm, cm2, nc = sum_over_ranks(sums, group, device)
    mean = s / n
    var = max(0.0, cm2 / nc - (cm / nc) ** 2)
    err = math.sqrt(var / max(1.0, nc - 1.0))
    return mean, err
