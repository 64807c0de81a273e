"""Merging statistics of independent replicas (one process per GPU).

Realizations are independent and the noise is addressed by the global
realization index (``stream_offset``), so shards of one ensemble run on
different GPUs produce exactly the sample paths of one large run.  Their
statistics combine by summing the raw FP64 accumulators -- the sample count,
sum(delta), sum(delta^2) and, where accumulated, sum(delta delta^T) and the
time correlation's lag sums with their pair counts -- which
is the one exchange the method has (no per-step collective).  This module
does that sum with ``torch.distributed.all_reduce`` (gloo on host memory, or
NCCL), then finalises the statistics exactly as ``she_stats`` does.
"""
import numpy as np


def raw_from_stats(stats, realizations=None):
    """Raw pooled sums from a ``she_stats(..., raw=True[, cov=True][,
    time_corr=True])`` result.  The time correlation needs the handle's
    realization count R: lag l has R (n/R - l) pairs."""
    n = float(stats["n_samples"])
    out = {"n": n, "sum_d": np.asarray(stats["sum_d"], dtype=np.float64),
           "sum_d2": np.asarray(stats["sum_d2"], dtype=np.float64)}
    if "cov" in stats:
        mu = out["sum_d"] / n
        out["sum_dd"] = n * (np.asarray(stats["cov"], dtype=np.float64) + np.outer(mu, mu))
    if "time_corr" in stats:
        R = int(realizations)
        ns = int(round(n / R))
        tc = np.asarray(stats["time_corr"], dtype=np.float64)
        pairs = np.array([R * max(0, ns - l) for l in range(tc.shape[0])], dtype=np.float64)
        out["n_tc"] = pairs
        out["sum_tc"] = np.where(pairs[:, None] > 0, np.nan_to_num(tc) * pairs[:, None], 0.0)
    return out


def allreduce_raw(raw, group=None):
    """Sum the raw accumulators of every rank (in place on a copy)."""
    import torch
    import torch.distributed as dist
    keys = [k for k in ("sum_d", "sum_d2", "sum_dd", "sum_tc", "n_tc") if k in raw]
    flat = np.concatenate([np.array([raw["n"]])] + [np.ravel(raw[k]) for k in keys])
    t = torch.from_numpy(flat.copy())
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    flat = t.numpy()
    out = {"n": float(flat[0])}
    pos = 1
    for k in keys:
        size = np.size(raw[k])
        out[k] = flat[pos:pos + size].reshape(np.shape(raw[k]))
        pos += size
    return out


def finalize(raw, tref):
    """mean = T_ref + sum(delta)/n, var = sum(delta^2)/n - mu^2 (biased, as
    in Sec. 3), cov = sum(delta delta^T)/n - mu mu^T."""
    n = raw["n"]
    mu = raw["sum_d"] / n
    out = {"n": n, "mean": np.asarray(tref) + mu, "var": raw["sum_d2"] / n - mu * mu}
    if "sum_dd" in raw:
        out["cov"] = raw["sum_dd"] / n - np.outer(mu, mu)
    if "sum_tc" in raw:
        # <delta_i(t + l K) delta_i(t)> over the pairs of every rank
        pairs = np.asarray(raw["n_tc"])[:, None]
        out["time_corr"] = np.where(pairs > 0, raw["sum_tc"] / np.maximum(pairs, 1), np.nan)
    return out
