"""The multi-rank path of bench.py on CPU: two gloo ranks.

Histories are independent, so N GPUs run N replicas with disjoint random
streams (the rank is the request id in the Philox key) and no data-path
collective; the only exchange is the max over ranks of the timed region.
These checks run the rank logic and the streams' independence with the
oracle standing in for the device.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    from oracle import oracle as O
    from paper_1107_3355_gb300 import workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, loc = bench.rank_env()
        assert (w, r, loc) == (world, rank, rank)
        # slowest rank's timed region, seen by every rank
        t_max = bench.max_over_ranks(10.0 * (rank + 1), world)
        rate = bench.whole_job_rate(world, 3, 1000, t_max)
        # each rank's replica: the same problem with its rank as request id
        prob = W.tiny_problem(n_histories=2000, n_batches=10).with_(request_id=rank)
        dose, _, led = O.run(prob)
        np.save(os.path.join(out_dir, "dose%d.npy" % rank), dose)
        np.save(os.path.join(out_dir, "meta%d.npy" % rank),
                np.array([t_max, rate, led["compton"], led["deposited"]]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    meta = [np.load(tmp_path / ("meta%d.npy" % r)) for r in range(world)]
    dose = [np.load(tmp_path / ("dose%d.npy" % r)) for r in range(world)]
    # every rank sees the slowest rank's time; the rate counts all ranks' histories
    for m in meta:
        assert m[0] == pytest.approx(20.0)
        assert m[1] == pytest.approx(world * 3 * 1000 / 0.020)
    # disjoint streams: the replicas differ, but agree statistically
    assert not np.array_equal(dose[0], dose[1])
    assert meta[0][2] != meta[1][2]
    assert meta[0][3] == pytest.approx(meta[1][3], rel=0.1)


def test_single_rank_defaults(monkeypatch):
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.rank_env() == (1, 0, 0)
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.whole_job_rate(1, 2, 100, 1000.0) == pytest.approx(200.0)


def test_parallel_oracle_baseline_runs_disjoint_processes():
    """The CPU baseline's multi-process timing: spawned single-thread oracle
    processes started together, one rate per step."""
    import bench
    rates = bench.oracle_rate_parallel("water32_1MeV_pencil", 300, 2, steps=2)
    assert len(rates) == 2 and all(r > 0 for r in rates)
    assert bench.host_cores() >= 1


def test_sharded_oracle_matches_one_process():
    """The test helper that spreads the oracle over host cores: four shards
    on disjoint streams, combined, agree with one process of the same size
    (per-voxel t-test, Sec. 3.1) and carry the N^-1/2 uncertainty."""
    from oracle import oracle as O
    from paper_1107_3355_gb300 import workloads as W
    from tests._oracle_parallel import run_sharded
    from tests._stats import sigma_over_dmax, t_test
    prob = W.tiny_problem(n_histories=8000, n_batches=10)
    d1, s1, _ = O.run(prob)
    d4, s4 = run_sharded(prob, 8000, procs=4)
    r = t_test(d1, s1, d4, s4, high_frac=0.1)
    assert r["P_high"] > 0.9, r
    assert sigma_over_dmax(d4, s4) == pytest.approx(sigma_over_dmax(d1, s1), rel=0.25)
