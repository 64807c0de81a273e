"""Multi-replica path on CPU: two gloo ranks each run a disjoint shard of the
ensemble (noise streams offset by the shard start, as bench.py does per GPU)
with the FP64 oracle, merge their raw accumulators with
paper_2406_12157_gb300.replica, and must reproduce the statistics of one
process running the whole ensemble (the shards' sample paths are identical
to the corresponding paths of the single run)."""
import os
import socket

import numpy as np
import pytest

import she_workloads as W

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, R, steps, out_q):
    import torch.distributed as dist

    from oracle import she as O
    from paper_2406_12157_gb300 import replica
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = W.oracle_rod(n=(24, 1, 1), wall_lo=1.0, wall_hi=2.0, stats_interval=5, relax_steps=50, tc_lags=4)
    shard = R // world
    o = O.run(p, shard, steps, stream0=rank * shard, want_cov=1)
    raw = {"n": float(o["n_samples"]), "sum_d": o["sum_d"], "sum_d2": o["sum_d2"],
           "sum_dd": o["sum_dd"], "sum_tc": o["sum_tc"], "n_tc": o["n_tc"].astype(np.float64)}
    merged = replica.allreduce_raw(raw)
    fin = replica.finalize(merged, O.reference_profile(p))
    if rank == 0:
        out_q.put({k: np.asarray(v) for k, v in fin.items()})
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_merge_equals_single_run():
    import torch.multiprocessing as mp

    from oracle import she as O
    O.lib()
    R, steps, world = 8, 300, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, R, steps, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = q.get(timeout=120)
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    p = W.oracle_rod(n=(24, 1, 1), wall_lo=1.0, wall_hi=2.0, stats_interval=5, relax_steps=50, tc_lags=4)
    ref = O.finalize(p, O.run(p, R, steps, want_cov=1))
    assert got["n"] == ref["n"]
    assert np.allclose(got["mean"], ref["mean"], rtol=1e-13, atol=1e-15)
    assert np.allclose(got["var"], ref["var"], rtol=1e-10, atol=1e-18)
    assert np.allclose(got["cov"], ref["cov"], rtol=1e-9, atol=1e-18)
    assert np.allclose(got["time_corr"], ref["time_corr"], rtol=1e-12, atol=1e-18)


def test_raw_from_stats_roundtrip():
    from paper_2406_12157_gb300 import replica
    rng = np.random.default_rng(0)
    d = rng.normal(size=(50, 6))
    stats = {"n_samples": 50, "sum_d": d.sum(0), "sum_d2": (d * d).sum(0)}
    mu = d.mean(0)
    stats["cov"] = d.T @ d / 50 - np.outer(mu, mu)
    raw = replica.raw_from_stats(stats)
    assert np.allclose(raw["sum_dd"], d.T @ d)
    fin = replica.finalize(raw, np.zeros(6))
    assert np.allclose(fin["var"], d.var(0))


def test_time_corr_raw_roundtrip():
    # time_corr finalised over R (n/R - l) pairs per lag back to raw lag sums
    from paper_2406_12157_gb300 import replica
    R, ns, L = 4, 7, 3
    rng = np.random.default_rng(1)
    sums = rng.normal(size=(L, 5))
    pairs = np.array([R * (ns - l) for l in range(L)], dtype=np.float64)
    stats = {"n_samples": R * ns, "sum_d": np.zeros(5), "sum_d2": np.ones(5), "time_corr": sums / pairs[:, None]}
    raw = replica.raw_from_stats(stats, realizations=R)
    assert np.allclose(raw["sum_tc"], sums) and np.array_equal(raw["n_tc"], pairs)
    assert np.allclose(replica.finalize(raw, np.zeros(5))["time_corr"], sums / pairs[:, None])
