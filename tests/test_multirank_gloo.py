"""Multi-rank host logic on CPU: two gloo ranks (one process each).

A multi-GPU run shards chains over ranks and reduces only host bookkeeping:
the slowest rank's time, the whole-job rate and the energy estimate.  Two CPU
ranks run the same helpers as the benchmark and are compared with a single
process holding all chains.
"""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2503_20566_gb300 import replicas  # noqa: E402

N_CHAINS, PER_CHAIN = 6, 5


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _samples(seed):
    rng = np.random.default_rng(seed)
    return list(rng.normal(-3.0, 0.4, size=N_CHAINS * PER_CHAIN))


def _worker(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        g = dist.group.WORLD
        seeds = replicas.rank_seeds(rank)
        e = _samples(seeds["chains"])
        sums = replicas.energy_sums(e, N_CHAINS)
        mean, err = replicas.energy_estimate(sums, g)
        tmax = replicas.max_over_ranks(10.0 + rank, g)
        total = replicas.sum_over_ranks([1.0, float(rank)], g)
        out[rank] = (seeds["tensors"], seeds["chains"], seeds["step"](3), mean, err, tmax, total)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_match_one_process():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    r0, r1 = res[0], res[1]
    # one wave function, distinct chains and Metropolis streams
    assert r0[0] == r1[0]
    assert r0[1] != r1[1] and r0[2] != r1[2]
    # reductions agree on every rank
    for a, b in zip(r0[3:], r1[3:]):
        assert a == b
    # the energy estimate equals the single-process one over all chains
    e_all = _samples(replicas.rank_seeds(0)["chains"]) + _samples(replicas.rank_seeds(1)["chains"])
    mean1, err1 = replicas.energy_estimate(replicas.energy_sums(e_all, 2 * N_CHAINS))
    assert abs(r0[3] - mean1) < 1e-12
    assert abs(r0[4] - err1) < 1e-12
    chain_means = np.asarray(e_all).reshape(2 * N_CHAINS, PER_CHAIN).mean(axis=1)
    assert abs(r0[3] - np.mean(e_all)) < 1e-12
    assert abs(r0[4] - chain_means.std(ddof=1) / np.sqrt(len(chain_means))) < 1e-12
    assert r0[5] == 11.0
    assert r0[6] == [2.0, 1.0]


def test_whole_job_rate_counts_all_ranks_over_the_slowest():
    assert replicas.whole_job_rate(1000, 3, 4, 1500.0) == pytest.approx(8000.0)
