"""Benchmark: SHE cell-updates/s incl. noise on one GB300 (or N, weak scaling).

A bench *step* is one pass of the whole hot path over one batch of input:
``--chunk`` forward-Euler time steps (default 10,000) of the full ensemble,
including the inline Philox noise and the moment (and covariance) sampling
every K steps after relaxation.  The default workload is the 1D
non-equilibrium rod: 256 cells, walls 1 and 2, 4096 realizations, FP32 state,
statistics every 10 steps after 1e5 steps; ``--steps 100`` covers its full
1e6 time steps.

``--impl reference`` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (there is no other reference implementation).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SHE cell-updates/s incl. noise, FP32-batched vs FP64 plain, % of roofline"
UNIT = "cell-updates/s"

# Per-pipe roofline.  Algorithmic lane-operations per cell-update are counted
# from the source algorithm (never from compiled code) and assigned to the
# pipe the CUDA programming guide's throughput table puts them on; rates are
# that table's results per clock per SM (FP32 add/multiply/FMA 128; 32-bit
# integer multiply 64; 32-bit integer add, logic, compare, min/max and
# conversions 64) except the transcendentals (MUFU), which run at 32 per clock
# per SM on GB300 (twice the table's 16: Blackwell Ultra doubled the special
# function units; the XU pipe counters of the covariance kernel's capture
# agree), plus the issue limit of one warp instruction per clock per SM
# sub-partition (4 x 32 lane-ops).  The bound is the slowest resource.
PIPE_RATES = {"issue": 128.0, "fma": 128.0, "alu": 64.0, "imad": 64.0, "xu": 32.0}


def noise_ops(nz):
    """Lane-ops of nz normals.  Philox-4x32-10 per block of 4 normals: 10
    rounds of two 32x32->64 products (hi and lo: 4 integer-multiply ops) and
    four xors (the round keys are precomputed per launch, so the key
    schedule's adds are not per-block work): 10 imad + 10 alu per normal.
    Box-Muller per block: 2 log2, 2 square roots, 2 sin, 2 cos (8 xu), 4
    integer-to-float conversions and 2 sign-flip xors (6 alu), 10 FP32
    multiplies/FMAs (the two uniforms' scale, -2 ln 2 times the logarithm,
    the two angles, the four products): per normal 2 xu, 1.5 alu, 2.5 fma."""
    return {"imad": 10.0 * nz, "alu": 11.5 * nz, "xu": 2.0 * nz, "fma": 2.5 * nz}


def flux_ops(nf, species):
    """Face fluxes: heat, the face sum T_l + T_r and its product with the
    normal that carries the amplitude (2 fma); species, the face sum, its
    clamp at 0 (1 alu), the product with r eps_c (the halving of the mean
    folded into the constant), the square root (1 xu) and the product with
    the normal (3 fma)."""
    if species:
        return {"fma": 3.0 * nf, "alu": 1.0 * nf, "xu": 1.0 * nf}
    return {"fma": 2.0 * nf}


def add_ops(*parts):
    out = {k: 0.0 for k in ("imad", "alu", "xu", "fma")}
    for d in parts:
        for k, v in d.items():
            if k != "issue":
                out[k] += v
    out["issue"] = sum(out[k] for k in ("imad", "alu", "xu", "fma"))
    return out


# cell update: 1D per face q_f = r (T_r - T_l) + G_f (a difference and an FMA)
# and T + (q_hi - q_lo) (two adds): 4 FP32 ops per cell-update beside the
# face flux; 2D 9, 3D 11; the predictor-corrector's trapezoid (T + T* + inc) / 2: 3
OPS_1D = add_ops(noise_ops(257.0 / 256.0), flux_ops(257.0 / 256.0, False), {"fma": 4.0})
OPS_1D_PC = add_ops(noise_ops(257.0 / 256.0), flux_ops(2 * 257.0 / 256.0, False), {"fma": 2 * 4.0 + 3.0})
OPS_2D_SP = add_ops(noise_ops(2.0), flux_ops(2.0, True), {"fma": 9.0})
OPS_2D_SP_PC = add_ops(noise_ops(2.0), flux_ops(4.0, True), {"fma": 2 * 9.0 + 3.0})
OPS_3D = add_ops(noise_ops(3.0), flux_ops(3.0, False), {"fma": 11.0})
# implicit theta scheme: the explicit right-hand side (stencil and flux
# difference 5), the block LU (forward 1, backward 2: FMA and multiply), the
# correction by the neighbouring values (2) and the reduced solve (4 FMAs per
# source lane per lane, LPR / C = 1/4 of a source lane per cell at 32 x 8: 1);
# its factors are read from a shared-memory table
OPS_1D_THETA = add_ops(noise_ops(257.0 / 256.0), flux_ops(257.0 / 256.0, False), {"fma": 4.0 + 6.0})
# a rod of several materials: the update ic (a_hi (T_r - T) + a_lo (T_l - T) + dG) + T,
# 5 FP32 ops beyond the face sums, its coefficients read from a shared-memory table
OPS_1D_VAR = add_ops(noise_ops(257.0 / 256.0), flux_ops(257.0 / 256.0, False), {"fma": 5.0})


def pipe_roofline(ops, cu_per_s, sm_mhz, sms=152):
    """Per-pipe bounds (cell-updates/s) and the binding one."""
    pipes = {}
    for k, rate in PIPE_RATES.items():
        if ops.get(k, 0.0) <= 0.0:
            continue
        bound = sms * sm_mhz * 1e6 * rate / ops[k]
        pipes[k] = {"ops_per_cell_update": round(ops[k], 3), "rate_per_clk_per_sm": rate,
                    "bound_cell_updates_per_s": bound, "frac": round(cu_per_s / bound, 4)}
    binding = min(pipes, key=lambda k: pipes[k]["bound_cell_updates_per_s"])
    return binding, pipes


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="she_clocks_", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu_index)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------- workloads --

# Per workload: problem, description, default time steps per bench step, the
# dominant kernel, and its algorithmic work per cell-update counted from the
# source algorithm: lane-ops per pipe (noise_ops, flux_ops, the update) and
# HBM bytes (state read + write, 8 B, plus the FP32 moment read-modify-write,
# 16 B per sample, on the streaming 2D/3D paths; the 1D path keeps its rows
# on chip for a whole launch).
WORKLOADS = {
    "gradient_rod": dict(
        leg_chunk=10000, leg_steps=10,
        make=lambda W: W.gradient_rod(),
        desc=("1D SHE rod, 256 cells, Dirichlet walls T_L=1 T_R=2, eps=1e-3, r=0.2, 4096 "
              "realizations, FP32 state, moments and full 256x256 equal-time covariance "
              "(tcgen05) every 10 steps after 1e5 steps"),
        chunk=10_000, ops=OPS_1D, bytes=None,
        kernel="k_step1d_cov<16,16,dirichlet,heat>",
        # DRAM read + write of one launch (2560 steps, mostly the per-CTA
        # covariance flush), ncu capture in profiles/k_step1d_cov_gradient_rod.md
        traffic=dict(bytes=100.741376e6 + 41.261312e6, realizations=4096)),
    "gradient_rod_pc": dict(
        leg_chunk=10000, leg_steps=10,
        make=lambda W: W.gradient_rod(scheme="pc"),
        desc=("the gradient_rod configuration (1D SHE rod, 256 cells, walls 1 and 2, eps=1e-3, r=0.2, "
              "4096 realizations, FP32, moments and the 256x256 covariance on tcgen05 every 10 steps "
              "after 1e5) stepped by the predictor-corrector scheme of Sec. 3"),
        # one normal per face as forward Euler, the face flux and update twice
        # (predictor, corrector on T*), and the trapezoid (T + T* + inc) / 2
        chunk=10_000, ops=OPS_1D_PC, bytes=None,
        kernel="k_step1d_cov<16,16,dirichlet,heat,pc>",
        traffic=dict(bytes=100.781824e6 + 41.127168e6, realizations=4096)),   # profiles/k_step1d_cov_pc_gradient_rod_pc.md
    "species_2d": dict(
        leg_chunk=1000, leg_steps=10,
        make=lambda W: W.species_2d(want_sk=1),
        desc=("2D stochastic species diffusion, 256x256 periodic, D=1, r=0.1, eps_c=1e-3, c=1 + "
              "zero-sum perturbation, 256 realizations, FP32, moments and the full 2D S(k) "
              "(two-stage DFT-as-GEMM on tcgen05) every 10 steps after 1e4"),
        chunk=1000, ops=OPS_2D_SP, bytes=8.0 + 16.0 / 10,
        kernel="k_step2d<float,8,32,species>",
        traffic=dict(bytes=72.756736e6 + 21.945344e6, realizations=256),   # profiles/k_step2d_species_2d.md
        # per realization and sample: row DFT (ny x nx x nx MAC) + column DFTs
        # for the 128 rows ky < 128 (2 x 128 x ny x nx MAC; the other rows
        # follow from the real-field symmetry), 3 split products, 2 flop per MAC
        stats_kernel="k_sk2d", stats_flop=lambda p: 3 * 2 * (p["n"][1] * p["n"][0] ** 2
                                                           + 2 * 128 * p["n"][1] * p["n"][0])),
    "gradient_rod_tc": dict(
        leg_chunk=10000, leg_steps=10,
        make=lambda W: W.gradient_rod(want_cov=0, tc_lags=8, tune=1),
        desc=("the gradient_rod configuration without the covariance, with the time correlation "
              "<delta_i(t + l K) delta_i(t)> at 8 lags accumulated every 10 steps after 1e5 (the "
              "exercise on <dT_i^{n+m} dT_i^n>, Sec. 6); layout picked by the autotuner"),
        # forward Euler plus one product and one add per lag and cell at
        # every sample (8 lags / 10 steps); memory per cell and sample: the
        # ring store and L - 1 ring loads (4 B each), every 10 steps (the lag
        # sums are shared-memory partials, flushed once per launch)
        chunk=10_000, ops=add_ops(OPS_1D, {"fma": 2 * 8 / 10.0}), bytes=(4.0 * 8) / 10.0,
        kernel="k_step1d<float,8,32,dirichlet,heat> with the time correlation",
        traffic=dict(bytes=117.473024e6 + 66.203904e6, realizations=4096)),   # profiles/k_step1d_tc_gradient_rod_tc.md
    "species_2d_pc": dict(
        leg_chunk=1000, leg_steps=6,
        make=lambda W: W.species_2d(want_sk=1, scheme="pc"),
        desc=("the species_2d configuration (2D species diffusion 256x256 periodic, 256 realizations, "
              "FP32, moments and the full 2D S(k) every 10 steps after 1e4) stepped by the "
              "predictor-corrector scheme of Sec. 3 in one pass (the predictor state carried one row "
              "ahead of the corrector)"),
        # two normals per cell drawn once, the two face fluxes and the update
        # twice, the trapezoid 3; bytes: the state read and written once plus
        # the moments
        chunk=1000, ops=OPS_2D_SP_PC, bytes=8.0 + 16.0 / 10,
        kernel="k_step2d_pc<float,8,32,species>",
        traffic=dict(bytes=75.952384e6 + 23.411968e6, realizations=256),   # profiles/k_step2d_pc_species_2d_pc.md
        stats_kernel="k_sk2d", stats_flop=lambda p: 3 * 2 * (p["n"][1] * p["n"][0] ** 2
                                                           + 2 * 128 * p["n"][1] * p["n"][0])),
    "cube_3d": dict(
        leg_chunk=100, leg_steps=10,
        make=lambda W: W.cube_3d(want_sk=2),
        desc=("3D SHE 256^3 periodic, T0=1, r=0.1, eps=1e-3, 8 realizations, FP32, HBM-streaming "
              "stencil, moments and S(k) along x, y, z (line covariance on tcgen05) every 10 steps"),
        chunk=100, ops=OPS_3D, bytes=8.0 + 16.0 / 10,
        kernel="k_step3d<float,8,heat>",
        traffic=dict(bytes=574.792192e6 + 494.729216e6, realizations=8),    # profiles/k_step3d_cube_3d.md
        # per realization and sample: for each axis a SYRK over all lines
        # (cells / n_a lines x n_a^2 MAC), 3 split products, 2 flop per MAC
        stats_kernel="k_axes_syrk", stats_flop=lambda p: 3 * 2 * sum(
            (p["n"][0] * p["n"][1] * p["n"][2] // p["n"][a]) * p["n"][a] ** 2 for a in range(3))),
    "batched_rods": dict(
        leg_chunk=2560, leg_steps=10,
        make=lambda W: W.batched_rods(count=10_000, seed=0),
        desc=("10,000 uneven 1D SHE rods, N log-uniform in [16, 2048], kappa U[0.5, 2], walls U[1, 3], "
              "r = 0.2 each, per-instance seeds, FP32, moments every 10 steps after 1e4, one CUDA-graph "
              "launch per step batch"),
        chunk=2560, ops=OPS_1D, bytes=None, kernel="k_step1d_batch<*>",
        traffic=dict(bytes=84.418304e6 + 44.954112e6, realizations=1)),    # profiles/k_step1d_batch_batched_rods.md
    "two_material_rod": dict(
        leg_chunk=10000, leg_steps=10,
        make=lambda W: W.two_material_rod(),
        desc=("1D SHE rod of two materials (the iron / aluminium exercise, Sec. 6): 256 cells, iron "
              "(rho c_V 1, lambda 1) left, aluminium (0.684, 3.386) right, walls 1 and 2, dt 0.08, "
              "k_B 1e-3, 4096 realizations, FP32, moments and the 256x256 covariance (tcgen05) every 10 "
              "steps after 1e5"),
        chunk=10_000, ops=OPS_1D_VAR, bytes=None,
        kernel="k_step1d_cov<16,16,dirichlet,heat,var>",
        traffic=dict(bytes=100.785664e6 + 41.385216e6, realizations=4096)),   # profiles/k_step1d_cov_var_two_material_rod.md
    "gradient_rod_cn": dict(
        leg_chunk=10000, leg_steps=10,
        make=lambda W: W.gradient_rod(scheme="cn", dt=2.0, want_cov=0),
        desc=("the gradient_rod configuration (1D SHE rod, 256 cells, walls 1 and 2, eps=1e-3, 4096 "
              "realizations, FP32, moments every 10 steps after 1e5) stepped by Crank-Nicolson (the implicit "
              "exercise of Sec. 6) at r = 2, ten times forward Euler's stability limit; a partitioned "
              "tridiagonal solve per realization and step"),
        chunk=10_000, ops=OPS_1D_THETA, bytes=None,
        kernel="k_step1d<float,32,8,dirichlet,heat,theta>",
        traffic=dict(bytes=21.046272e6, realizations=4096)),   # profiles/k_step1d_theta_gradient_rod_cn.md
    "oracle_rod": dict(
        leg_chunk=10000, leg_steps=3,
        make=lambda W: W.oracle_rod(want_cov=0, want_sk=0),
        desc="1D SHE rod, 32 cells, walls 1, 16 realizations, FP64",
        chunk=10_000, ops=OPS_1D, bytes=None, kernel="k_step1d<double,4,8>"),
}


# the workloads timed in short legs beside the headline (the `workloads`
# sub-object of the bench line)
LEG_WORKLOADS = ["gradient_rod_pc", "gradient_rod_cn", "gradient_rod_tc", "two_material_rod", "species_2d",
                 "species_2d_pc", "cube_3d", "batched_rods"]


def workload(name):
    import she_workloads as W
    if name not in WORKLOADS:
        raise SystemExit("unknown workload %s" % name)
    w = WORKLOADS[name]
    return w["make"](W), w["desc"]


def _cells(p):
    c = 1
    for v in p["n"][: p["dim"]]:
        c *= v
    return c


# ------------------------------------------------------------ oracle timing --

def oracle_sample_rate(p, seconds_hint=10.0):
    """Time the FP64 oracle, as it stands, on a bounded sample of the workload
    (10-30 s of host work, sampling phase, relax 0); returns (cell-updates/s,
    threads used, sample description).  A list of uneven instances is sampled
    as every k-th instance, run one after the other (one realization each, so
    one thread)."""
    from oracle import she as O
    O.lib()
    if isinstance(p, list):
        pick = p[:: max(1, len(p) // 64)][:64]
        cells = sum(q["n"][0] for q in pick)
        steps = int(max(10, min(10_000, 1.4e8 // cells)))
        t0 = time.perf_counter()
        for i, q in enumerate(pick):
            O.run(dict(q, relax_steps=0), 1, steps, stream0=i)
        dt = time.perf_counter() - t0
        sample = ("%d of the %d instances (every %d-th, %d cells in all) x %d steps each, one after the "
                  "other, FP64 oracle, %.1f s" % (len(pick), len(p), max(1, len(p) // 64), cells, steps, dt))
        return cells * steps / dt, 1, sample
    q = dict(p)
    q["relax_steps"] = 0
    cells = _cells(p)
    R_s = min(p["realizations"], 1024 if cells <= 4096 else 16)
    budget = 1.0e9 if p["dim"] == 3 else 2.6e9
    steps = int(max(10, min(10_000, budget // (R_s * cells))))
    q["want_sk"] = 0 if p["dim"] > 1 else q.get("want_sk", 0)
    t0 = time.perf_counter()
    O.run(q, R_s, steps)
    dt = time.perf_counter() - t0
    rate = R_s * steps * _cells(p) / dt
    sample = ("%d realizations x %d steps of the workload (sampling phase, every %d steps%s), "
              "FP64 oracle, %.1f s" % (R_s, steps, p["stats_interval"],
                                       ", covariance" if q.get("want_cov") else "", dt))
    return rate, O.num_threads(), sample


# --------------------------------------------------------------- our arm ----

def _make_sim(she, args, name, rank, stream, realizations=None):
    """Simulation of a workload (a batch of instances for a list), its
    problem, cells per realization and realizations; every rank runs a full
    ensemble on its own noise streams (weak scaling)."""
    p, desc = workload(name)
    if isinstance(p, list):
        probs = [dict(q, relax_steps=args.relax) if args.relax is not None else q for q in p]
        sim = she.BatchSimulation(probs, stream=stream, stream_offset=rank * len(probs))
        return sim, probs[0], desc, sum(q["n"][0] for q in probs), 1, probs
    if args.relax is not None:
        p["relax_steps"] = args.relax
    if realizations:
        p["realizations"] = realizations
    sim = she.Simulation(p, stream=stream, stream_offset=rank * p["realizations"])
    return sim, p, desc, _cells(p), p["realizations"], None


def _roofline(wl, p, R, batch, cu_per_launch, per_launch_ms, prof, ms, peaks, peak_src, sm_mhz):
    """Per-pipe roofline of the dominant (step) kernel, plus the HBM and the
    tensor-core statistics kernels where the workload has them."""
    cu_rate = cu_per_launch / (per_launch_ms / 1e3)
    ops = wl["ops"]
    binding, pipes = pipe_roofline(ops, cu_rate, sm_mhz)
    rate = PIPE_RATES[binding]
    achieved = cu_rate * ops[binding] / 1e12                    # lane-op Tops/s on the binding pipe
    peak = 152 * sm_mhz * 1e6 * rate / 1e12
    traffic = None
    if wl.get("traffic"):
        traffic = wl["traffic"]["bytes"] * (R / wl["traffic"]["realizations"] if not batch else 1.0)
    roof = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "Tops/s",
            "frac": round(achieved / peak, 4), "traffic": traffic, "kernel": wl["kernel"],
            "binding_pipe": binding, "pipes": pipes,
            "ms_per_launch": round(per_launch_ms, 5), "cell_updates_per_launch": cu_per_launch,
            "launches": prof["step_launches"],
            "share_of_timed_region": round(prof["step_ms"] / ms, 4) if ms > 0 and prof["step_launches"] else None,
            "peak_source": ("min over pipes of (rate per clk per SM x 152 SMs x sampled SM clock %.0f MHz) / "
                            "(lane-ops per cell-update); rates from the CUDA throughput table (%s peaks file "
                            "for the other roofs)" % (sm_mhz, peak_src))}
    if wl["bytes"]:
        gbs = cu_rate * wl["bytes"] / 1e9
        roof["hbm"] = {"achieved": round(gbs, 1), "peak": peaks.get("hbm_gbs", 6800.0), "unit": "GB/s",
                       "frac": round(gbs / peaks.get("hbm_gbs", 6800.0), 4), "bytes_per_cell_update": wl["bytes"],
                       "peak_source": "hbm_gbs (%s)" % peak_src}
    if prof["stats_launches"] and wl.get("stats_flop"):
        flop = wl["stats_flop"](p) * (R if not batch else 1)
        tf = flop / (prof["stats_ms"] / prof["stats_launches"] / 1e3) / 1e12
        bf16 = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1900.0))
        roof["stats"] = {"bound": "tensor", "kernel": wl["stats_kernel"], "achieved": round(tf, 2),
                         "peak": bf16, "unit": "TFLOP/s", "frac": round(tf / bf16, 4),
                         "flop_per_launch": flop, "launches": prof["stats_launches"],
                         "ms_per_launch": round(prof["stats_ms"] / prof["stats_launches"], 5),
                         "share_of_timed_region": round(prof["stats_ms"] / ms, 4) if ms > 0 else None,
                         "peak_source": "bf16_tflops_sustained (%s); the BF16x3 split counts 3 products" % peak_src}
    return roof


def _time_leg(sim, stream, chunk, steps, flush, barrier):
    """K timed bench steps (CUDA events on the simulation's stream, L2 flushed
    between them outside the events) with the library's per-kernel device
    timing; returns (ms, launches, prof)."""
    import torch
    launches0 = sim.launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    sim.profile(True)
    barrier()
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.add_(1.0)                 # L2 flush (256 MB write) outside the timed events
            ev[k][0].record(stream)
        sim.step(chunk)
        with torch.cuda.stream(stream):
            ev[k][1].record(stream)
    barrier()
    prof = sim.profile_read()
    sim.profile(False)
    ms = sum(x.elapsed_time(y) for x, y in ev)
    return ms, sim.launches() - launches0, prof


def _relax(sim, p, chunk):
    """Step past the relaxation so that every timed step is in the sampling
    phase (the phase that holds nine tenths of a full run)."""
    left = int(p.get("relax_steps", 0))
    while left > 0:
        n = min(left, 100 * chunk)
        sim.step(n)
        left -= n


def run_workload_leg(she, args, name, stream, flush, barrier, peaks, peak_src):
    """A short device-timed leg of another workload for the `workloads`
    sub-object: relaxation untimed, one warm-up bench step, then its timed
    bench steps; the per-kernel roofline as for the headline."""
    import torch
    wl = WORKLOADS[name]
    sim, p, desc, cells, R, probs = _make_sim(she, args, name, 0, stream)
    batch = probs is not None
    layout = int(she.she_get_sizes(sim.h).layout)
    chunk = wl["leg_chunk"]
    try:
        _relax(sim, p, chunk)
        sim.step(chunk)
        torch.cuda.synchronize()
        clocks = ClockSampler(0)
        clocks.start()
        ms, launches, prof = _time_leg(sim, stream, chunk, wl["leg_steps"], flush, barrier)
        clk = clocks.stop()
    finally:
        sim.close()
    cu = R * cells * chunk * wl["leg_steps"]
    sm_mhz = (clk or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    step_launches = max(1, prof["step_launches"])
    per_launch_ms = prof["step_ms"] / step_launches if prof["step_launches"] else ms / max(1, launches)
    roof = _roofline(wl, p, R, batch, cu / step_launches, per_launch_ms, prof, ms, peaks, peak_src, sm_mhz)
    return {"value": cu / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / wl["leg_steps"], "layout": layout,
            "steps": wl["leg_steps"], "time_steps_per_bench_step": chunk, "description": desc,
            "phase": "sampling", "roofline": roof, "gpu_launches": int(launches), "clocks": clk}


def run_ours(args):
    import numpy as np
    import torch

    import paper_2406_12157_gb300 as she

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    she.lib()
    stream = torch.cuda.Stream()
    sim, p, desc, cells, R, probs = _make_sim(she, args, args.workload, rank, stream, args.realizations)
    batch = probs is not None
    layout = int(she.she_get_sizes(sim.h).layout)
    wl = WORKLOADS[args.workload]
    chunk = args.chunk if args.chunk else wl["chunk"]
    cu_per_step = R * cells * chunk

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # relaxation untimed, then the warm-up steps: the timed steps are all in
    # the sampling phase
    if args.relax is None:
        _relax(sim, p, chunk)
    for _ in range(args.warmup):
        sim.step(chunk)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    t_wall0 = time.perf_counter()
    ms, launches, prof = _time_leg(sim, stream, chunk, args.steps, flush, barrier)
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    if dist is not None:
        tt = torch.tensor([ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    total_cu = cu_per_step * args.steps * world
    value = total_cu / (ms / 1e3)
    try:
        stats = sim.stats(cov=bool(p.get("want_cov")), sk=bool(p.get("want_sk", 0) & 1),
                          sk_axes=bool(p.get("want_sk", 0) & 2))          # device reduce + D2H
        assert np.all(np.isfinite(stats["var"]))
    except she.SheError as e:
        if e.status != she._abi.SHE_ERR_STATE:   # no sample yet in a short run is fine
            raise

    # ---- replicas: every rank's raw accumulators summed (one all-reduce, the
    # method's only exchange) and finalised by the library on rank 0 ----
    merged = None
    if dist is not None and not batch:
        from paper_2406_12157_gb300 import replica
        try:
            total = replica.allreduce_raw(sim.stats_raw())
            if rank == 0:
                fin = replica.finalize(sim.params, total, cov=bool(p.get("want_cov")))
                merged = {"n_samples": fin["n_samples"], "ranks": world,
                          "mean_var": float(np.mean(fin["var"])),
                          "max_var_se_rel": float(np.nanmax(fin["var_se"] / fin["var"]))}
        except she.SheError as e:
            if e.status != she._abi.SHE_ERR_STATE:
                raise

    # ---- FP64 plain form on the same workload, a bounded number of steps ----
    plain_steps = max(10, min(2000, int(2e8 // (R * cells))))
    p64 = dict(p)
    # 1D: the plain three-launches-per-step FP64 form; 2D/3D (streaming
    # kernels already launch once per step): the same kernel in FP64
    kind64 = ("plain" if p["dim"] == 1 and p.get("scheme", "fe") == "fe" and not p.get("tc_lags")
              and p.get("lambda_cells") is None else "auto")
    if batch:     # same total cells as 256-cell rows in the plain FP64 form
        p64 = dict(p, n=(256, 1, 1), realizations=max(1, cells // 256))
    sim64 = she.Simulation(p64, stream=stream, precision="fp64", kernel=kind64, stream_offset=rank * R,
                           want_cov=0, want_sk=0)
    sim64.step(min(plain_steps, 50))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
    sim64.step(plain_steps)
    with torch.cuda.stream(stream):
        e1.record(stream)
    torch.cuda.synchronize()
    plain_rate = (p64["realizations"] * _cells(p64)) * plain_steps / (e0.elapsed_time(e1) / 1e3)
    sim64.close()

    # ---- e2e through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        state, step = sim.state()
        host = torch.from_numpy(state).pin_memory()
        host_np = host.numpy()
        e2e_steps = max(1, min(args.steps, 10))
        barrier()
        t0 = time.perf_counter()
        d2h = 0
        for _ in range(e2e_steps):
            sim.set_state(host_np, step)            # H2D of the step's input state
            sim.step(chunk)
            try:
                out = sim.stats(cov=bool(p.get("want_cov")), sk=bool(p.get("want_sk", 0) & 1),
                                sk_axes=bool(p.get("want_sk", 0) & 2))      # device reduce + D2H
                d2h = sum(v.nbytes for v in out.values() if hasattr(v, "nbytes"))
                d2h += 2 * min(32, R) * cells * 8 + (cells * cells * 8 if p.get("want_cov") else 0)
            except she.SheError as e:
                if e.status != she._abi.SHE_ERR_STATE:
                    raise
                st_now, _ = sim.state()             # no sample yet: read the state back
                d2h = st_now.nbytes
            step += chunk
        barrier()
        te = time.perf_counter() - t0
        e2e = {"value": cu_per_step * e2e_steps * world / te, "unit": UNIT,
               "h2d_bytes_per_step": int(host_np.nbytes),
               "d2h_bytes_per_step": int(d2h)}
    sim.close()

    peaks, peak_src = _peaks()
    # the other workloads: short device-timed legs, every rank (weak scaling
    # runs them per GPU; rank 0 reports its own)
    legs = {}
    if not args.no_workloads and args.workload == "gradient_rod":
        for name in LEG_WORKLOADS:
            legs[name] = run_workload_leg(she, args, name, stream, flush, barrier, peaks, peak_src)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    # the dominant (step) kernel alone: its launches and their summed device
    # time, from the event pairs the library recorded in the timed region
    step_launches = max(1, prof["step_launches"])
    cu_per_launch = cu_per_step * args.steps / step_launches
    per_launch_ms = prof["step_ms"] / step_launches if prof["step_launches"] else ms / max(1, launches)
    sm_mhz = (clk or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    roof = _roofline(wl, p, R, batch, cu_per_launch, per_launch_ms, prof, ms, peaks, peak_src, sm_mhz)
    cpu = None
    if not args.no_cpu_baseline and world == 1:     # rank 0 at N = 1 only
        rate, cores, sample = oracle_sample_rate(probs if batch else p)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if p["precision"] == "fp32" else "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "cells": cells,
                   "realizations_per_gpu": R, "time_steps_per_bench_step": chunk,
                   "stats_interval": p["stats_interval"], "relax_steps": p["relax_steps"],
                   "fused_1d_layout": layout,
                   "phase": ("sampling: the relaxation steps run untimed before the warm-up"
                             if args.relax is None else "relax overridden to %d" % args.relax),
                   "l2": "flushed between timed steps (256 MB write outside the events)"},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
        "clocks": clk,
        "fp64_plain": {"value": plain_rate, "unit": UNIT, "steps": plain_steps,
                       "form": "plain FP64 (3 launches/step)" if kind64 == "plain" else "same kernel in FP64",
                       "speedup_fp32_batched": value / world / plain_rate},
        "workloads": legs or None,
        "replica_merge": merged,
        "wall_s": t_wall,
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


# --------------------------------------------------------- reference arm ----

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    from oracle import she as O
    p, desc = workload(args.workload)
    q = dict(p)
    q["relax_steps"] = 0
    cells = _cells(p)
    R_s, steps = 32, 2000
    O.lib()
    for _ in range(max(0, args.warmup)):
        O.run(q, R_s, 200)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        O.run(q, R_s, steps, step0=k * steps)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = R_s * steps * cells * args.steps / total
    sample = ("%d realizations x %d steps per bench step (sampling phase), FP64 oracle" % (R_s, steps))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "cells": cells},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="gradient_rod")
    ap.add_argument("--chunk", type=int, default=0,
                    help="time steps per bench step (default: per workload)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the short legs of the other workloads")
    ap.add_argument("--realizations", type=int, default=None,
                    help="override the workload's realizations (small ncu captures)")
    ap.add_argument("--relax", type=int, default=None,
                    help="override the workload's relaxation steps (profiling the sampling phase)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
