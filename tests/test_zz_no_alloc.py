"""The entry point that allocates nothing, against the handle path.

she_step_plain_noalloc serves callers that cannot call cudaMalloc (graph
capture, pre-reserved memory budgets, allocation-free real-time loops): the
caller passes its own device input and output rows, and the face fluxes go
to a fixed device array inside the library.  Two consecutive calls must give
the rows the existing plain-form handle path (she_init with kernel =
SHE_KERNEL_PLAIN, she_set_state, she_step_n, she_get_state) gives, within the
FP64 parity tolerance of the other tests (1e-12 relative).  The file is named
to be collected last.
"""
import ctypes

import numpy as np
import pytest

import she_workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2406_12157_gb300 as S  # noqa: E402
from paper_2406_12157_gb300 import _abi  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2406_12157_gb300 import build
    build.build()


@pytest.mark.parametrize("N,bc,eq", [(256, "dirichlet", "heat"), (37, "periodic", "species")])
def test_noalloc_step_matches_handle_path_twice(N, bc, eq):
    walls = (1.0, 2.0) if bc == "dirichlet" else (1.5, 1.5)
    R = 64
    prob = W.oracle_rod(n=(N, 1, 1), bc=bc, equation=eq, wall_lo=walls[0], wall_hi=walls[1],
                        n0=300.0, kB=2e-3, realizations=R, precision="fp64", kernel="plain",
                        want_cov=0, want_sk=0, stream_offset=11)
    x = W.random_states(prob, R, seed=N)
    step0 = 4321
    # existing entry points: a plain-form handle, two steps
    with S.Simulation(prob) as sim:
        sim.set_state(x, step0)
        sim.step(1)
        ref1, _ = sim.state()
        sim.step(1)
        ref2, _ = sim.state()
    # the allocation-free entry point, caller-owned device rows, two calls
    L = S.lib()
    params = S.params_from_problem(prob)
    d_in = torch.from_numpy(x).to("cuda")
    d_mid = torch.empty_like(d_in)
    d_out = torch.empty_like(d_in)
    torch.cuda.synchronize()
    st = L.she_step_plain_noalloc(ctypes.byref(params), d_in.data_ptr(), d_mid.data_ptr(), step0)
    assert st == _abi.SHE_OK
    st = L.she_step_plain_noalloc(ctypes.byref(params), d_mid.data_ptr(), d_out.data_ptr(), step0 + 1)
    assert st == _abi.SHE_OK
    torch.cuda.synchronize()
    got1 = d_mid.cpu().numpy()
    got2 = d_out.cpu().numpy()
    assert np.max(np.abs(got1 - ref1) / np.abs(ref1)) < 1e-12
    assert np.max(np.abs(got2 - ref2) / np.abs(ref2)) < 1e-12


def test_noalloc_accepts_exactly_its_scratch_size():
    # realizations * (N + 1) == the limit: 4096 rows of 255 cells fill the array
    N = 255
    R = _abi.SHE_NOALLOC_MAX_FACES // (N + 1)
    assert R * (N + 1) == _abi.SHE_NOALLOC_MAX_FACES
    prob = W.oracle_rod(n=(N, 1, 1), wall_lo=1.0, wall_hi=2.0, realizations=R, precision="fp64",
                        kernel="plain", want_cov=0, want_sk=0)
    x = W.random_states(prob, R, seed=7)
    with S.Simulation(prob) as sim:
        sim.set_state(x, 99)
        sim.step(1)
        ref, _ = sim.state()
    params = S.params_from_problem(prob)
    d_in = torch.from_numpy(x).to("cuda")
    d_out = torch.empty_like(d_in)
    torch.cuda.synchronize()
    st = S.lib().she_step_plain_noalloc(ctypes.byref(params), d_in.data_ptr(), d_out.data_ptr(), 99)
    assert st == _abi.SHE_OK
    torch.cuda.synchronize()
    got = d_out.cpu().numpy()
    assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-12


def test_noalloc_rejects_sizes_beyond_its_scratch():
    R = (_abi.SHE_NOALLOC_MAX_FACES // 257) + 1     # realizations * (N + 1) just above the limit
    assert R * 257 > _abi.SHE_NOALLOC_MAX_FACES
    prob = W.oracle_rod(n=(256, 1, 1), realizations=R, precision="fp64", want_cov=0, want_sk=0)
    params = S.params_from_problem(prob)
    d = torch.empty(1, dtype=torch.float64, device="cuda")
    e = torch.empty(1, dtype=torch.float64, device="cuda")
    st = S.lib().she_step_plain_noalloc(ctypes.byref(params), d.data_ptr(), e.data_ptr(), 0)
    assert st == _abi.SHE_ERR_INVALID_ARG
