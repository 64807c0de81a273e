"""Multi-replica path on CPU: two gloo ranks each run a disjoint shard of the
ensemble (noise streams offset by the shard start, as bench.py does per GPU)
with the FP64 oracle, put their accumulators into libshe's raw block layout
(she_raw: per-batch sums with their sample counts, sum of delta delta^T, the
time correlation's lag sums and pair counts), sum the blocks with
paper_2406_12157_gb300.replica.allreduce_raw, and finalise them with the
library's host-only she_finalize -- the same code she_stats runs.  The
result must reproduce the statistics of one process running the whole
ensemble (the shards' sample paths are those of the single run).  No GPU is
used: she_finalize makes no device call."""
import os
import socket

import numpy as np
import pytest

import she_workloads as W

torch = pytest.importorskip("torch")

N, R, STEPS, WORLD, B = 24, 8, 300, 2, 2


def _prob():
    return W.oracle_rod(n=(N, 1, 1), wall_lo=1.0, wall_hi=2.0, stats_interval=5, relax_steps=50, tc_lags=4)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _raw_from_oracle(p, first, count):
    """Raw block of realizations [first, first + count) in B batches."""
    from oracle import she as O
    per = count // B
    raw = {"batches": B, "batch_n": np.zeros(B, dtype=np.int64), "batch_sum_d": np.zeros((B, N)),
           "batch_sum_d2": np.zeros((B, N)), "sum_dd": np.zeros((N, N)), "tc_sum": np.zeros((4, N)),
           "tc_pairs": np.zeros(4, dtype=np.int64), "n_samples": 0}
    for b in range(B):
        o = O.run(p, per, STEPS, stream0=first + b * per, want_cov=1)
        raw["batch_n"][b] = o["n_samples"]
        raw["batch_sum_d"][b] = o["sum_d"]
        raw["batch_sum_d2"][b] = o["sum_d2"]
        raw["sum_dd"] += o["sum_dd"]
        raw["tc_sum"] += o["sum_tc"]
        raw["tc_pairs"] += o["n_tc"]
        raw["n_samples"] += o["n_samples"]
    return {k: (np.ascontiguousarray(v) if isinstance(v, np.ndarray) else v) for k, v in raw.items()}


def _worker(rank, world, port, out_q):
    import torch.distributed as dist

    import paper_2406_12157_gb300 as S
    from paper_2406_12157_gb300 import replica
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = _prob()
    shard = R // world
    raw = _raw_from_oracle(p, rank * shard, shard)
    merged = replica.allreduce_raw(raw)
    fin = replica.finalize(S.params_from_problem(p), merged, cov=True, time_corr=True)
    if rank == 0:
        out_q.put({k: np.asarray(v) for k, v in fin.items()})
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_merge_through_she_finalize_equals_single_run():
    import torch.multiprocessing as mp

    from oracle import she as O
    O.lib()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, WORLD, port, q)) for r in range(WORLD)]
    for pr in procs:
        pr.start()
    got = q.get(timeout=120)
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    p = _prob()
    ref = O.finalize(p, O.run(p, R, STEPS, want_cov=1))
    assert got["n_samples"] == ref["n"]
    assert np.allclose(got["mean"], ref["mean"], rtol=1e-13, atol=1e-15)
    assert np.allclose(got["var"], ref["var"], rtol=1e-10, atol=1e-18)
    assert np.allclose(got["cov"], ref["cov"], rtol=1e-9, atol=1e-18)
    assert np.allclose(got["time_corr"], ref["time_corr"], rtol=1e-12, atol=1e-18)


def test_finalize_var_se_from_batches():
    # the standard error of the variance from the batch sums: the scatter of
    # the per-batch variances over sqrt(B)
    import paper_2406_12157_gb300 as S
    rng = np.random.default_rng(0)
    Bn, nb, n = 6, 40, 5
    d = rng.normal(size=(Bn, nb, n))
    raw = {"n_samples": Bn * nb, "batches": Bn, "batch_n": np.full(Bn, nb, dtype=np.int64),
           "batch_sum_d": np.ascontiguousarray(d.sum(1)), "batch_sum_d2": np.ascontiguousarray((d * d).sum(1))}
    p = W.oracle_rod(n=(n, 1, 1), bc="periodic", wall_lo=0.0, wall_hi=0.0)
    fin = S.she_finalize(S.params_from_problem(p), raw)
    allv = d.reshape(-1, n)
    assert np.allclose(fin["var"], allv.var(0), rtol=1e-12)
    vb = d.var(1)
    assert np.allclose(fin["var_se"], vb.std(0, ddof=1) / np.sqrt(Bn), rtol=1e-10)
    # nothing sampled: SHE_ERR_STATE
    with pytest.raises(S.SheError) as e:
        S.she_finalize(S.params_from_problem(p), dict(raw, n_samples=0))
    assert e.value.status == S._abi.SHE_ERR_STATE
