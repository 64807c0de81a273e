"""Merging the statistics of independent replicas (one process per GPU).

Realizations are independent and the noise is addressed by the global
realization index (``stream_offset``), so shards of one ensemble run on
different GPUs produce exactly the sample paths of one large run.  Their
statistics combine by summing the raw FP64 accumulators of she_stats_raw --
per-batch sums of delta and delta^2 with their sample counts, sum of
delta delta^T, the structure factors' sums and the time correlation's lag
sums with their pair counts -- which is the one exchange the method has (no
per-step collective).  This module only does that sum, with one
``torch.distributed.all_reduce`` (gloo on host memory, or NCCL); the
library's host call she_finalize then forms the statistics, exactly as
she_stats does for a single handle.
"""
import numpy as np

from . import she_finalize

_INT_KEYS = ("batch_n", "tc_pairs")
_SUM_KEYS = ("batch_n", "batch_sum_d", "batch_sum_d2", "sum_dd", "sk_sum", "axes_sum", "tc_sum", "tc_pairs")


def allreduce_raw(raw, group=None):
    """Element-wise sum of every rank's raw block (she_stats_raw layout)."""
    import torch
    import torch.distributed as dist
    keys = [k for k in _SUM_KEYS if raw.get(k) is not None]
    flat = np.concatenate([np.array([float(raw["n_samples"])])] +
                          [np.ravel(raw[k]).astype(np.float64) for k in keys])
    t = torch.from_numpy(flat.copy())
    if dist.get_backend(group) == "nccl":      # NCCL reduces device memory
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    flat = t.cpu().numpy()
    out = {"n_samples": int(round(flat[0])), "batches": int(raw["batches"])}
    pos = 1
    for k in keys:
        size = np.size(raw[k])
        v = flat[pos:pos + size].reshape(np.shape(raw[k]))
        out[k] = np.rint(v).astype(np.int64) if k in _INT_KEYS else np.ascontiguousarray(v)
        pos += size
    return out


def finalize(params, raw, **kw):
    """Statistics of the merged ensemble: she_finalize on the summed block."""
    return she_finalize(params, raw, **kw)
