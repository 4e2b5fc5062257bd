"""The CPU oracle on several host cores: one spawned single-thread process
per shard, each on its own random stream (request id), results combined as
independent estimates of the same dose (D = sum n_i D_i / N and
sigma^2 = sum n_i^2 sigma_i^2 / N^2 per voxel).  Spawned, so a test
process that already holds a CUDA context can use it."""
import multiprocessing as mp
import os

import numpy as np


def _shard(args):
    prob, n, rid = args
    from oracle import oracle as O
    d, s, led = O.run(prob.with_(n_histories=n, request_id=rid))
    return n, d, s


def _shard_dose(args):
    prob, n, rid = args
    from oracle import oracle as O
    d, _, led = O.run(prob.with_(n_histories=n, request_id=rid))
    return n, d, led


def run_shards(prob, n_total, procs=None, first_request_id=1000):
    """The shards themselves: a list of (histories, dose, ledger), one per
    process, each an independent estimate of the dose (use them as batches)."""
    procs = procs or min(16, os.cpu_count() or 1)
    n = [n_total // procs + (1 if k < n_total % procs else 0) for k in range(procs)]
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_shard_dose, [(prob, n[k], first_request_id + k) for k in range(procs)])


def run_sharded(prob, n_total, procs=None, first_request_id=1000):
    procs = procs or min(16, os.cpu_count() or 1)
    n = [n_total // procs + (1 if k < n_total % procs else 0) for k in range(procs)]
    with mp.get_context("spawn").Pool(procs) as pool:
        parts = pool.map(_shard, [(prob, n[k], first_request_id + k) for k in range(procs)])
    N = float(sum(p[0] for p in parts))
    dose = sum(p[0] * p[1] for p in parts) / N
    sigma = np.sqrt(sum((p[0] * p[2]) ** 2 for p in parts)) / N
    return dose, sigma
