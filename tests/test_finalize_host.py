"""The host-only finalisation (she_finalize, the code she_stats runs) of the
1D structure factor against its definition, on CPU: S(k) = <|hat T_k|^2>
with hat T the unnormalised DFT of Eq. (3.11) of every sampled field
T = T_ref + delta, and the fluctuation part <|hat delta_k|^2> - |<hat
delta_k>|^2, both evaluated sample by sample with a dense DFT matrix; the
library forms them from the pooled sums only (the wrapped-diagonal sums of
sum delta delta^T)."""
import numpy as np
import pytest

import she_workloads as W

S = pytest.importorskip("paper_2406_12157_gb300")


@pytest.mark.parametrize("N,bc", [(7, "dirichlet"), (37, "periodic"), (64, "dirichlet"), (300, "periodic")])
def test_finalize_1d_structure_factor_matches_its_definition(N, bc):
    rng = np.random.default_rng(N)
    B, nb = 4, 30
    d = rng.normal(size=(B, nb, N)) * 0.1 + rng.normal(size=N) * 0.05
    raw = {"n_samples": B * nb, "batches": B, "batch_n": np.full(B, nb, dtype=np.int64),
           "batch_sum_d": np.ascontiguousarray(d.sum(1)), "batch_sum_d2": np.ascontiguousarray((d * d).sum(1)),
           "sum_dd": np.ascontiguousarray(np.einsum("bsi,bsj->ij", d, d).ravel())}
    walls = (1.0, 2.0) if bc == "dirichlet" else (1.5, 1.5)
    p = W.oracle_rod(n=(N, 1, 1), bc=bc, wall_lo=walls[0], wall_hi=walls[1], want_cov=1, want_sk=1)
    fin = S.she_finalize(S.params_from_problem(p), raw, cov=True, sk=True)
    x = d.reshape(-1, N)
    # the exact steady profile of a uniform rod: linear between the walls
    ref = walls[0] + (walls[1] - walls[0]) * (np.arange(N) + 0.5) / N
    F = np.exp(-2j * np.pi * np.outer(np.arange(N), np.arange(N)) / N)
    that = (ref + x) @ F.T
    dhat = x @ F.T
    sk = np.mean(np.abs(that) ** 2, axis=0)
    sk_fluct = np.mean(np.abs(dhat) ** 2, axis=0) - np.abs(dhat.mean(axis=0)) ** 2
    assert np.allclose(fin["sk"], sk, rtol=1e-10, atol=1e-12 * np.max(sk))
    assert np.allclose(fin["sk_fluct"], sk_fluct, rtol=1e-9, atol=1e-10 * np.max(sk_fluct))
    mu = x.mean(axis=0)
    assert np.allclose(fin["cov"], x.T @ x / x.shape[0] - np.outer(mu, mu), rtol=1e-10, atol=1e-14)
