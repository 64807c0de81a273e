"""GPU parity of the batched uneven 1D instances (one CUDA-graph launch per
step batch) against the oracle run of each instance (its own N, kappa,
walls and seed; noise stream = instance index)."""
import numpy as np
import pytest

import she_workloads as W
from oracle import she as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2406_12157_gb300 as S  # noqa: E402


def rel_err(a, b):
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


def _batch(ns, steps=300, relax=40, K=4):
    probs = W.batched_rods(count=len(ns), seed=77)
    out = []
    for i, (q, n) in enumerate(zip(probs, ns)):
        q = dict(q, n=(n, 1, 1), relax_steps=relax, stats_interval=K, kB=2e-3)
        out.append(q)
    return out


# one or more instances of every layout class, full and ragged rows
NS = [2, 5, 16, 17, 32, 33, 64, 100, 128, 129, 170, 200, 255, 256, 300, 350, 420, 512, 513, 600, 700, 740, 800,
      880, 950, 1000, 1024, 1100, 1250, 1400, 1500, 1650, 1700, 1900, 2048]


def test_batch_matches_oracle_per_instance():
    probs = _batch(NS)
    steps = 300
    with S.BatchSimulation(probs) as b:
        st0, _ = b.state()
        b.step(steps)
        st, step = b.state()
        g = b.stats(raw=True)
    assert step == steps
    for i, q in enumerate(probs):
        off, n = b.offsets[i], q["n"][0]
        ic = O.run(q, 1, 0, stream0=i)["state"][0]
        assert rel_err(st0[off:off + n].astype(np.float64), ic) < 1e-6
        ref = O.run(q, 1, steps, stream0=i)
        assert rel_err(st[off:off + n].astype(np.float64), ref["state"][0]) < 2e-4, (i, n)
        fin = O.finalize(q, ref)
        assert g["n_samples"] == ref["n_samples"]
        assert np.max(np.abs(g["mean"][off:off + n] - fin["mean"])) < 1e-4
        assert rel_err(g["var"][off:off + n], fin["var"]) < 5e-2


def test_batch_one_step_fp32_parity():
    probs = _batch([7, 40, 256, 700, 2000])
    rng = np.random.default_rng(3)
    total = sum(q["n"][0] for q in probs)
    x = rng.uniform(1.0, 3.0, size=total).astype(np.float32)
    with S.BatchSimulation(probs) as b:
        b.set_state(x, 999)
        b.step(1)
        got, _ = b.state()
    for i, q in enumerate(probs):
        off, n = b.offsets[i], q["n"][0]
        ref = O.step(q, x[off:off + n].astype(np.float64), 999, i)
        assert rel_err(got[off:off + n].astype(np.float64), ref) < 2e-5


def test_ten_thousand_rods_sampled_one_percent():
    # 10,000 instances, N log-uniform in [16, 2048]; 1 % checked against the oracle
    probs = W.batched_rods(count=10_000, seed=0)
    steps = 200
    with S.BatchSimulation(probs) as b:
        b.step(steps)
        st, _ = b.state()
        assert b.launches() > 0
    for i in range(0, 10_000, 100):
        q = probs[i]
        off, n = b.offsets[i], q["n"][0]
        ref = O.run(q, 1, steps, stream0=i)["state"][0]
        assert rel_err(st[off:off + n].astype(np.float64), ref) < 2e-4
