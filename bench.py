#!/usr/bin/env python3
"""Benchmark of the adiabatic-evolution hot path on one GB300 (or N replicas).

Headline (one bench step = one pass of the whole hot path over one synthetic instance):
  Exact-Cover-3 instance, n = 28 qubits, seed 3; linear path H = (1-s) H_i + s H_f,
  s = t/T, T = 100; uniform start |S>; fixed-step grid from the step rule (kappa = 0.1).
  Each step: set psi(0) -> 3 RK4 start-up steps -> PEC steps (one fused H*psi per step) up to
  `--pec` grid steps -> P_1 and E(T-window) readback.  State in complex64 (headline) and
  complex128 (reported beside it, against the FP64 FMA rate measured in the same run).
Metric: H*psi GB/s = algorithmic bytes of the hot path / device time (inputs resident in HBM),
with the fused PEC step's achieved bandwidth against the measured HBM copy peak.

Beside it on the same line: the small-state workload (n = 10, T = 20: wall time per solve,
step by step and with CUDA-graph replays), the batched workload (512 instances, n 12-22,
T 10-200, with a one-at-a-time sample), the served request stream (n 10-26 and n = 30,
T 10-500, under a stated time cap, and the same requests one at a time), the XY algorithm's
PEC step, and per-result checks of the complex64 results with n <= 14 against the FP64
oracle (spawned host processes running beside the GPU legs, outside every timed region).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_QUBITS = 28
SEED = 3
T_RUN = 100.0
PEC_DEFAULT = 64
METRIC = "H*psi GB/s (EC3 n=28 fused PEC step, algorithmic bytes)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--pec", type=int, default=PEC_DEFAULT, help="PEC steps per bench step")
    ap.add_argument("--n", type=int, default=N_QUBITS)
    ap.add_argument("--slab-bits", type=int, default=0, help="slab order of the PEC step: 0 off, -1 auto")
    ap.add_argument("--no-c128", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-xy", action="store_true")
    ap.add_argument("--no-small", action="store_true")
    ap.add_argument("--no-ycomp", action="store_true")
    ap.add_argument("--no-oracle-check", action="store_true")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--serve-count", type=int, default=40)
    ap.add_argument("--serve-rate", type=float, default=1.0, help="requests per second (Poisson)")
    ap.add_argument("--serve-cap", type=float, default=120.0, help="time cap of the served stream (s)")
    ap.add_argument("--quick", action="store_true", help="small batched/served legs (not the stated workloads)")
    ap.add_argument("--only-xy", action="store_true", help="run the XY-algorithm leg alone (profiling)")
    ap.add_argument("--xy-n", type=int, default=24)
    ap.add_argument("--xy-start", choices=["ground", "dicke"], default="ground",
                    help="XY start: the sector ground state (Lanczos) or the Dicke state (no Lanczos workspace)")
    a = ap.parse_args()
    if a.quick:
        a.batch_count, a.serve_count, a.serve_cap = 48, 16, 30.0
    return a


# ----------------------------------------------------------------------------- accounting
def alg_bytes(n, amp, pec_steps):
    """Algorithmic bytes of one bench step: the minimum vector traffic of each operation.
    PEC step 7 N b (read y, f_n, f_{n-1}, f_{n-2}, f_{n-3}; write y, f_{n+1}); RK4 step 18 N b;
    f_3 + predictor 8 N b; init 1 N b; energy 1 N b."""
    N = 1 << n
    return N * amp * (7 * pec_steps + 18 * 3 + 8 + 1 + 1)


def pec_flops_c128(n_flip, n_clause_classes=1):
    """Algorithmic FP64 flops per amplitude of one PEC step: flip products 4 each (complex
    amplitude times real coefficient, accumulated), diagonal 4 + 2 per clause class,
    corrector and predictor 16 each, norm and error reductions 10."""
    return 4 * n_flip + 4 + 2 * n_clause_classes + 32 + 10


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def kernel_hash():
    h = hashlib.sha256()
    for f in ("kernels.cu", "xpartial.cu", "api.cu", "aqc_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_1311_3938_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def len_layouts(n, t, c):
    """Number of tile layouts for n qubits (tile bits t, contiguous chunk bits c)."""
    if n <= t:
        return 1
    return 1 + -(-(n - t) // (t - c))


def profiled_traffic(prec_name, n=N_QUBITS):
    """dram bytes per PEC step from the committed ncu summary, if it was taken on the current
    kernel sources and the same state size (else None)."""
    p = os.path.join(ROOT, "profiles", "pec_step_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
    except Exception:
        return None
    e = d.get(prec_name)
    if not e or e.get("kernel_hash") != kernel_hash() or e.get("n", N_QUBITS) != n:
        return None
    return e.get("dram_bytes_per_pec_step")


# ----------------------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no-samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- replicas
def replica_barrier(dist, device):
    """Barrier across replicas (no-op for one process)."""
    if dist is not None:
        if device.type == "cuda":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def replica_max(dist, x, device):
    """Max of a scalar over replicas: the job's time is its slowest replica's."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(bytes_per_step, steps, world, ms_max):
    """Whole-job throughput: every replica processes its own copy of the workload (weak
    scaling), the job ends with the slowest replica."""
    return bytes_per_step * steps * world / (ms_max * 1e-3) / 1e9


# ----------------------------------------------------------------------------- CPU oracle
def cpu_sample(target_s=15.0):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the workload: the same EC3
    family / path / T at n = 22 (vectors far beyond CPU caches), first 3 RK4 + P PEC steps,
    all host cores.  Returns (GB/s of algorithmic bytes, cores, description)."""
    from instances import generate_ec3
    from oracle import oracle as O

    n = 22
    inst = generate_ec3(n, SEED)
    H = O.ec3_hamiltonian(inst)
    sched = O.linear_path(T_RUN)
    N = O.step_count(H, sched)
    cores = os.cpu_count() or 1
    psi0 = O.uniform_state(n)
    t0 = time.perf_counter()
    O.propagate(H, sched, N, psi0, max_steps=4, nthreads=cores)  # 3 RK4 + 1 PEC: 14 evaluations
    t_probe = time.perf_counter() - t0
    per_eval = t_probe / 14.0
    pec = max(1, min(2000, int((target_s - t_probe) / max(per_eval, 1e-6))))
    t0 = time.perf_counter()
    O.propagate(H, sched, N, psi0, max_steps=3 + pec, nthreads=cores)
    dt = time.perf_counter() - t0
    gbs = alg_bytes(n, 16, pec) / dt / 1e9
    desc = (f"FP64 oracle (plain C, {cores} threads) on the EC3 seed-{SEED} linear T={T_RUN:g} workload at n={n}: "
            f"3 RK4 + {pec} PEC steps of its step grid, {dt:.1f} s")
    return gbs, cores, desc, dt


# ----------------------------------------------------------------------------- oracle checks
ORACLE_MAX_N = 14  # results checked against the FP64 oracle (host processes, outside timed regions)


def _nice_worker():
    try:
        os.nice(10)  # below the bench's own host thread, which drives the GPU
    except OSError:
        pass


def oracle_solve(spec):
    """The FP64 CPU oracle on one job (X algorithm, EC3 instance of `seed`, uniform start), in
    a spawned host process: returns (spec, grid steps, P_1, final state)."""
    from instances import generate_ec3, xx_pairs
    from oracle import oracle as O

    n, seed, nonlinear, T, s_kind = spec["n"], spec["seed"], spec["nonlinear"], spec["T"], spec["s_kind"]
    inst = generate_ec3(n, seed)
    H = O.ec3_hamiltonian(inst, pairs=xx_pairs(n, seed) if nonlinear else None)
    sched = (O.nonlinear_path if nonlinear else O.linear_path)(T, s_kind)
    N = O.step_count(H, sched)
    r = O.propagate(H, sched, N, O.uniform_state(n))
    return spec, N, O.fidelity(r.psi, inst.solution), r.psi


class OracleChecks:
    """FP64 oracle solves of the checked jobs on the host cores (spawned processes, niced),
    running while the GPU legs run; `results(timeout)` collects what finished."""

    def __init__(self, workers):
        import multiprocessing as mp

        self.pool = mp.get_context("spawn").Pool(processes=workers, initializer=_nice_worker)
        self.workers = workers
        self.pending = {}

    @staticmethod
    def spec_of(job):
        return {"n": job.n, "seed": job.seed, "nonlinear": bool(job.nonlinear), "T": float(job.T),
                "s_kind": int(job.s_kind)}

    def submit(self, key, spec):
        self.pending[key] = self.pool.apply_async(oracle_solve, (spec,))

    def results(self, timeout):
        t_end = time.perf_counter() + timeout
        out = {}
        for key, r in self.pending.items():
            try:
                out[key] = r.get(timeout=max(0.0, t_end - time.perf_counter()))
            except Exception:
                pass
        self.pool.terminate()
        self.pool.join()
        return out


def oracle_errors(jobs, tag, oracle_results, max_n=ORACLE_MAX_N):
    """Per-result comparison of finished complex64 jobs with n <= max_n against the oracle:
    relative state error, |P_1 - P_1(oracle)|, equal step grids."""
    import numpy as np

    rows = []
    for job in jobs:
        if job.n > max_n or job.state is None:
            continue
        got = oracle_results.get((tag, job.jid))
        if got is None:
            continue
        spec, N, P1_or, psi_or = got
        a = job.state.astype(np.complex128)
        rows.append({"n": job.n, "grid_steps": int(job.steps), "oracle_steps": int(N),
                     "state_err": float(np.linalg.norm(a - psi_or) / np.linalg.norm(psi_or)),
                     "P1_err": abs(job.P1 - P1_or)})
    eligible = sum(1 for j in jobs if j.n <= max_n and j.state is not None)
    return {
        "checked": len(rows),
        "eligible": eligible,
        "max_n": max_n,
        "max_state_err_vs_oracle": max((r["state_err"] for r in rows), default=None),
        "max_P1_err_vs_oracle": max((r["P1_err"] for r in rows), default=None),
        "step_grids_equal": all(r["grid_steps"] == r["oracle_steps"] for r in rows),
        "state_bar": 1e-5,
    }


def quantile_censored(values, q):
    """Nearest-rank quantile of latencies where unfinished requests count as +inf; returns
    (value or None if it falls on an unfinished request, censored flag)."""
    v = sorted(values)
    if not v:
        return None, False
    k = max(0, math.ceil(q * len(v)) - 1)
    return (None, True) if math.isinf(v[k]) else (v[k], False)


# ----------------------------------------------------------------------------- workloads
def batched_jobs(count):
    from paper_1311_3938_gb300 import workloads as W

    return W.random_jobs(count, 1000, n_range=(12, 22), T_range=(10.0, 200.0), nonlinear=True)


def served_jobs(count, rate):
    from paper_1311_3938_gb300 import workloads as W

    return W.random_jobs(count, 2000, n_range=(10, 26), T_range=(10.0, 500.0), rate=rate, big_every=20, big_n=30,
                         path_mix=True)


def measure_batched(a, checks):
    """The batched workload: `count` seeded EC3 instances (seeds from 1000), n ~ U{12..22},
    nonlinear path, T ~ U[10, 200], complex64, all as members of one batch (autotuned shape).
    One-at-a-time solves of all of them would take about 2x the batch time, so every 16th job
    runs one at a time and batched again, for a like-for-like speedup at equal step grids."""
    import copy

    from paper_1311_3938_gb300 import autotune as A
    from paper_1311_3938_gb300 import workloads as W

    jobs = batched_jobs(a.batch_count)
    for j in jobs:
        j.keep = j.n <= ORACLE_MAX_N
    shape, _ = A.autotune(copy.deepcopy(jobs[: min(16, len(jobs))]), rounds=3)
    tile_bits, threads, spr = shape
    t_batch = W.run_batched(jobs, threads=threads, steps_per_round=spr, tile_bits=tile_bits)
    every = 16 if len(jobs) >= 64 else 1
    sample = [copy.deepcopy(j) for j in jobs[::every]]
    for j in sample:
        j.keep, j.state = False, None
    sb = copy.deepcopy(sample)
    t_sb = W.run_batched(sb, threads=threads, steps_per_round=spr, tile_bits=tile_bits)
    t_seq = W.run_sequential(sample)
    dP1 = max(abs(x.P1 - y.P1) for x, y in zip(sb, sample))
    steps = sum(j.steps for j in jobs)
    amp_steps = sum(j.steps * (1 << j.n) for j in jobs)
    return {
        "workload": f"{len(jobs)} EC3 instances, seeds 1000-{999 + len(jobs)}, n~U{{12..22}}, nonlinear path, "
                    "T~U[10,200], complex64 (FP64 reductions), one batch, persistent k_batch under CUDA graphs",
        "count": len(jobs),
        "wall_s": t_batch,
        "solves_per_s_batched": len(jobs) / t_batch,
        "grid_steps_total": steps,
        "alg_GBs": 7 * 8 * amp_steps / t_batch / 1e9,
        "sequential_sample": f"every {every}th job ({len(sample)} jobs) one at a time and batched again",
        "solves_per_s_sequential": len(sample) / t_seq,
        "sample_solves_per_s_batched": len(sample) / t_sb,
        "sample_speedup": t_seq / t_sb,
        "max_abs_dP1_batched_vs_sequential": dP1,
        "autotuned_shape": {"tile_bits": tile_bits, "threads": threads, "steps_per_round": spr},
        "_jobs": jobs,
    }


def measure_serving(a):
    """The serving stream: `count` requests, Poisson arrivals at `rate`/s, n ~ U{10..26} with
    every 20th request n = 30, path linear/nonlinear uniform, T ~ U[10, 500], complex64;
    continuous batching (n <= 16 in the batch; larger states, which fill the GPU alone, on their
    own stream one at a time) under the HBM budget, arrived requests taken in order of estimated work; ended at
    the time cap (requests then unfinished are censored).  The same requests then run one at a
    time in the same order (the arrived request of least work next) under the same cap."""
    import copy

    from paper_1311_3938_gb300 import workloads as W

    jobs = served_jobs(a.serve_count, a.serve_rate)
    for j in jobs:
        j.keep = j.n <= ORACLE_MAX_N
    seq_jobs = copy.deepcopy(jobs)
    for j in seq_jobs:
        j.keep = False
    import torch

    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    large_grid = (3 * sms) // 4
    srv = W.Server(batch_max_n=16, max_members=128, steps_per_round=16, big_chunk=32, policy="shortest", max_large=1,
                   large_grid=large_grid)
    try:
        res = srv.serve(jobs, time_limit=a.serve_cap)
    finally:
        srv.close()
    done = res.pop("jobs")
    cens = res.pop("censored_jobs")
    res.pop("not_admitted")
    offered = [j for j in jobs if j.arrival <= a.serve_cap]
    lat = [j.latency if not math.isnan(j.finished) else math.inf for j in offered]
    p50, c50 = quantile_censored(lat, 0.50)
    p99, c99 = quantile_censored(lat, 0.99)
    s_done, s_cens, s_wall = W.serve_one_at_a_time(seq_jobs, time_limit=a.serve_cap, order="shortest")
    s_lat = [j.latency if not math.isnan(j.finished) else math.inf for j in seq_jobs if j.arrival <= a.serve_cap]
    sp50, sc50 = quantile_censored(s_lat, 0.50)
    sp99, sc99 = quantile_censored(s_lat, 0.99)
    # the n = 15..20 results against the library's own complex128 path (the oracle takes the n <= 14 ones)
    W.attach_c128_errors(done, min_n=ORACLE_MAX_N + 1, max_n=20)
    c128 = [j.P1_err_vs_c128 for j in done if not math.isnan(j.P1_c128)]
    ns = [j.n for j in jobs]
    return {
        "workload": (f"{len(jobs)} requests (seed 2000), Poisson {a.serve_rate:g}/s, n~U{{10..26}} + every 20th n=30, "
                     f"path linear/nonlinear, T~U[10,500], complex64; time cap {a.serve_cap:g} s"),
        "requests": len(jobs),
        "offered_within_cap": len(offered),
        "n_mix": {str(k): ns.count(k) for k in sorted(set(ns))},
        "order": "arrived requests by estimated work T n 2^n, smallest first (both runs)",
        "served": {
            "policy": f"continuous batching of n <= 16; one n > 16 state at a time on its own stream, its launches "
                      f"capped at {large_grid} CTAs ({large_grid} of {sms} SMs) so that batch launches find SMs free",
            "completed": len(done),
            "censored_in_flight": len(cens),
            "wall_s": res["wall_s"],
            "solves_per_s": len(done) / res["wall_s"] if res["wall_s"] > 0 else None,
            "p50_latency_s": p50, "p50_censored": c50,
            "p99_latency_s": p99, "p99_censored": c99,
            "completed_p50_latency_s": res["p50_latency_s"],
            "completed_p99_latency_s": res["p99_latency_s"],
            "hbm_budget_bytes": res["hbm_budget_bytes"],
            "hbm_peak_bytes": res["hbm_peak_bytes"],
            "by_route": res["by_route"],
        },
        "one_at_a_time": {
            "policy": "one context at a time",
            "completed": len(s_done),
            "censored_in_flight": len(s_cens),
            "wall_s": s_wall,
            "solves_per_s": len(s_done) / s_wall if s_wall > 0 else None,
            "p50_latency_s": sp50, "p50_censored": sc50,
            "p99_latency_s": sp99, "p99_censored": sc99,
        },
        "quantiles": "nearest rank over requests that arrived within the cap; unfinished ones count as infinite "
                     "(value null and *_censored true when the quantile falls on one)",
        "c128_checked": len(c128),
        "max_P1_err_vs_c128_gpu_path": max(c128) if c128 else None,
        "_jobs": done,
    }


def measure_xy(a, seed=3, pec=48):
    """PEC step of the XY algorithm with the alpha = 8 catalyst (Eq. Hixy, Eq. nlpath), started
    from the ground state of H^xy in the solution's Hamming-weight sector (Lanczos, complex64):
    Y products run through the general-product loop, pairs across layouts through the remote
    gather, so it moves more than the X-driver step."""
    import torch

    from instances import generate_ec3
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context
    import paper_1311_3938_gb300 as P

    n = a.xy_n
    inst = generate_ec3(n, seed)
    ctx = Context(n, P.AQC_C64)
    sched, k = HB.load_xy(ctx, inst, driver="xy", catalyst_alpha=8.0)
    ctx.set_schedule(20.0, sched)
    ctx.set_integrator(0, 0.0)
    t0 = time.perf_counter()
    if a.xy_start == "ground":
        E0, resid, iters = HB.set_xy_ground_start(ctx, k)
        start = f"ground state of H^xy in the weight-{k} sector"
    else:
        ctx.set_initial_state(("dicke", k))
        E0, resid, iters = None, None, 0
        start = f"Dicke state of weight {k}"
    t_ground = time.perf_counter() - t0
    torch.cuda.empty_cache()  # the Lanczos basis is released before the timed steps
    ctx.propagate(4, stats=False)
    ms = []
    for _ in range(3):
        st = ctx.propagate(pec, stats=True)
        ms.append(st["elapsed_ms"] / pec)
    torch.cuda.synchronize()
    ctx.close()
    step_ms = min(ms)
    gbs = 7 * (1 << n) * 8 / (step_ms * 1e-3) / 1e9
    return {"workload": f"XY algorithm + catalyst, EC3 n={n} seed {seed}, T=20, start: {start}, complex64",
            "ground_state": {"energy": E0, "residual": resid, "lanczos_steps": iters, "seconds": t_ground},
            "pec_step_ms": step_ms, "achieved": gbs, "unit": "GB/s (7 N b per PEC step)",
            "frac": gbs / peaks()[0]}


def measure_ycomp(a, pec=48):
    """The headline PEC step (EC3 n, seed 3, linear, T = 100, complex64) with the compensated
    corrector (aqc_set_y_compensation): what keeping y's low part costs per step."""
    import torch

    from instances import generate_ec3
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context
    import paper_1311_3938_gb300 as P

    n = a.n
    ctx = Context(n, P.AQC_C64, extra_vector=True)
    HB.load_ec3(ctx, generate_ec3(n, SEED))
    ctx.set_schedule(T_RUN, HB.linear_schedule())
    ctx.set_integrator(0, 0.0)
    ctx.set_y_compensation(True)
    ctx.set_initial_state("uniform")
    ctx.propagate(4, stats=False)
    ms = []
    for _ in range(3):
        st = ctx.propagate(pec, stats=True)
        ms.append(st["elapsed_ms"] / pec)
    torch.cuda.synchronize()
    ctx.close()
    torch.cuda.empty_cache()
    step_ms = statistics.median(ms)
    return {"what": "PEC step with the compensated corrector (y's low part read and written: 9 N b algorithmic)",
            "pec_step_ms": step_ms,
            "alg_GBs_9Nb": 9 * (1 << n) * 8 / (step_ms * 1e-3) / 1e9,
            "alg_GBs_7Nb": 7 * (1 << n) * 8 / (step_ms * 1e-3) / 1e9}


def measure_small(a, reps=30):
    """The small-state workload alone: EC3 n = 10 seed 1, linear path, T = 20, uniform start,
    complex128; host wall time per whole solve (initial state, every grid step, P_1 readback),
    step by step, with CUDA-graph replays of 16 PEC steps, and with replays of 64 steps on 8-bit
    tiles (the one-tile step runs on one SM at the FP64 rate; 8-bit tiles spread it over 4)."""
    import statistics as S

    from instances import generate_ec3
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context
    import paper_1311_3938_gb300 as P

    inst = generate_ec3(10, 1)
    out = {"workload": "ec3-n10-seed1-linear-T20-uniform, complex128, one context"}
    for label, k, tb in (("step_by_step", 0, 0), ("graph_replay", 16, 0), ("graph_replay_8bit_tiles", 64, 8)):
        ctx = Context(10, P.AQC_C128)
        ctx.set_graph_steps(k)
        if tb:
            ctx.set_tile_bits(tb)
        HB.load_ec3(ctx, inst)
        ctx.set_schedule(20.0, HB.linear_schedule())
        ctx.set_integrator(0, 0.0)
        walls = []
        for r in range(reps + 3):
            l0 = ctx.launch_count()
            t0 = time.perf_counter()
            ctx.set_initial_state("uniform")
            st = ctx.propagate(-1, stats=False)
            P1 = ctx.fidelity(inst.solution)
            dt = time.perf_counter() - t0
            if r >= 3:
                walls.append(dt)
        steps = ctx.grid()[0]
        out[label] = {"wall_ms_p50": 1e3 * S.median(walls), "wall_ms_min": 1e3 * min(walls),
                      "grid_steps_per_s": steps / S.median(walls), "kernels_per_solve": ctx.launch_count() - l0,
                      "graph_replays": ctx.graph_replays(), "P1": P1}
        out["grid_steps"] = steps
        if k and not tb:
            out["_state"] = ctx.state()
        ctx.close()
    out["speedup"] = out["step_by_step"]["wall_ms_p50"] / min(out["graph_replay"]["wall_ms_p50"],
                                                            out["graph_replay_8bit_tiles"]["wall_ms_p50"])
    return out


def measure_fp64_peak(device):
    """The FP64 FMA rate measured by aqc_measure_fp64_fma (clocks sampled during it)."""
    import torch

    from paper_1311_3938_gb300 import _native as N

    s = torch.cuda.current_stream(device)
    tf, ms = N.aqc_measure_fp64_fma(device, s.cuda_stream, 1 << 12)
    iters = int(min(1 << 24, max(1 << 12, (1 << 12) * 300.0 / max(ms, 1e-3))))  # ~0.3 s
    clk = Clocks(device)
    clk.start()
    tf, ms = N.aqc_measure_fp64_fma(device, s.cuda_stream, iters)
    clocks = clk.stop()
    return {"tflops": tf, "ms": ms, "iters": iters, "kernel": "k_fma64: 4 CTAs x 256 threads per SM, 8 FMA chains",
            "clocks": clocks}


# ----------------------------------------------------------------------------- our arm
def run_xy_only(a):
    import torch

    import paper_1311_3938_gb300 as P

    torch.cuda.set_device(0)
    P.build()
    print(json.dumps({"xy_algorithm": measure_xy(a)}), flush=True)


def run_ours(a):
    import numpy as np
    import torch

    import paper_1311_3938_gb300 as P
    from instances import generate_ec3
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    P.build()
    n = a.n
    inst = generate_ec3(n, SEED)
    hbm_peak, peak_kind = peaks()
    dev = torch.device("cuda", local)

    def barrier():
        replica_barrier(dist, dev)

    def max_over_ranks(x):
        return replica_max(dist, x, dev)

    def measure(prec):
        amp = 16 if prec == P.AQC_C128 else 8
        ctx = Context(n, prec, device=local)
        HB.load_ec3(ctx, inst)
        ctx.set_schedule(T_RUN, HB.linear_schedule())
        ctx.set_integrator(0, 0.0)
        ctx.set_slab_bits(a.slab_bits)
        stream = ctx.stream
        pec_ms = []
        res = {}

        def bench_step(record):
            ctx.set_initial_state("uniform")
            ctx.propagate(4, stats=False)  # 3 RK4 + f_3 + predictor + 1 PEC
            st = ctx.propagate(a.pec - 1, stats=True)  # timed PEC steps (events on ctx stream)
            if record:
                pec_ms.append(st["elapsed_ms"] / (a.pec - 1))
            res["P1"] = ctx.fidelity(inst.solution)
            res["E"] = ctx.energy(P.AQC_GRP_B)
            res["st"] = st

        for _ in range(a.warmup):
            bench_step(False)
        barrier()
        torch.cuda.synchronize()
        clk = Clocks(local)
        clk.start()
        l0 = ctx.launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            bench_step(True)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clocks = clk.stop()
        launches = ctx.launch_count() - l0
        ms = e0.elapsed_time(e1)
        ms = max_over_ranks(ms)
        # matvec only (aqc_hpsi: out = H(t) psi over all layout passes), device buffers
        dt_state = torch.complex64 if amp == 8 else torch.complex128
        mv_in = torch.full((1 << n,), 1.0 / math.sqrt(1 << n), dtype=dt_state, device=dev)
        mv_out = torch.empty_like(mv_in)
        with torch.cuda.stream(stream):
            for _ in range(2):
                ctx.hpsi(0.37 * T_RUN, mv_in, mv_out)
            m0 = torch.cuda.Event(enable_timing=True)
            m1 = torch.cuda.Event(enable_timing=True)
            m0.record(stream)
            reps = 5
            for _ in range(reps):
                ctx.hpsi(0.37 * T_RUN, mv_in, mv_out)
            m1.record(stream)
        torch.cuda.synchronize()
        mv_ms = m0.elapsed_time(m1) / reps
        del mv_in, mv_out
        ab = alg_bytes(n, amp, a.pec)
        value = whole_job_value(ab, a.steps, world, ms)
        pec_step_ms = statistics.mean(pec_ms)
        pec_ach = 7 * (1 << n) * amp / (pec_step_ms * 1e-3) / 1e9
        out = {
            "value": value,
            "ms_per_step": ms / a.steps,
            "pec_step_ms": pec_step_ms,
            "pec_step_gbs": pec_ach,
            "P1": res["P1"],
            "E": res["E"],
            "n_steps_grid": res["st"]["n_steps"],
            "t_end": res["st"]["t"],
            "launches": launches,
            "clocks": clocks,
            "matvec_ms": mv_ms,
        }
        # end-to-end through the public API with pinned host buffers: each step's psi(0) is
        # copied in and its final psi copied out by the staged transfers, so the copies of
        # instance k+1 (in) and k (out) overlap the integration; the first copy in and the last
        # copy out are inside the timed region and not hidden
        if not a.no_e2e:
            tdt = torch.complex64 if amp == 8 else torch.complex128
            host_in = [torch.empty(1 << n, dtype=tdt).pin_memory() for _ in range(2)]
            for h_ in host_in:
                h_.fill_(1.0 / math.sqrt(1 << n))
            host_out = [torch.empty_like(host_in[0]).pin_memory() for _ in range(2)]
            ctx.attach_transfers()
            obs = []

            def e2e_run(k_steps):
                ctx.stage_initial_state(host_in[0])
                for k in range(k_steps):
                    ctx.set_initial_state("staged")
                    if k + 1 < k_steps:
                        ctx.stage_initial_state(host_in[(k + 1) % 2])
                    ctx.propagate(a.pec + 3, stats=False)
                    obs.append((ctx.fidelity(inst.solution), ctx.energy(P.AQC_GRP_B)))  # D2H 16 B
                    ctx.fetch_state(host_out[k % 2])
                ctx.transfer_wait()

            e2e_run(1)
            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
            e2e_run(a.steps)
            torch.cuda.synchronize()
            dt = max_over_ranks(time.perf_counter() - t0)
            out["e2e"] = {
                "value": whole_job_value(ab, a.steps, world, dt * 1e3),
                "unit": "GB/s",
                "h2d_bytes_per_step": (1 << n) * amp,
                "d2h_bytes_per_step": (1 << n) * amp + 16,
                "copies": "staged (copy engines overlap the integration; first in / last out exposed)",
            }
            ctx.transfer_wait()
            del host_in, host_out
        ctx.close()
        del ctx
        torch.cuda.empty_cache()
        return out

    r64 = measure(P.AQC_C64)
    r128 = None if a.no_c128 else measure(P.AQC_C128)
    solo = world == 1
    fp64 = measure_fp64_peak(local) if (r128 is not None and solo) else None
    small = None if (a.no_small or not solo) else measure_small(a)
    # FP64 oracle solves of the checked results on the host cores, beside the GPU legs below
    checks = None
    if solo and not a.no_oracle_check and not (a.no_batch and a.no_serve and small is None):
        checks = OracleChecks(max(1, (os.cpu_count() or 2) - 2))
        if small is not None:
            checks.submit(("small", 0), {"n": 10, "seed": 1, "nonlinear": False, "T": 20.0, "s_kind": 0})
        if not a.no_batch:
            for j in batched_jobs(a.batch_count):
                if j.n <= ORACLE_MAX_N:
                    checks.submit(("batch", j.jid), OracleChecks.spec_of(j))
        if not a.no_serve:
            for j in served_jobs(a.serve_count, a.serve_rate):
                if j.n <= ORACLE_MAX_N:
                    checks.submit(("serve", j.jid), OracleChecks.spec_of(j))
    xy = None if (a.no_xy or not solo) else measure_xy(a)
    ycomp = None if (a.no_ycomp or not solo) else measure_ycomp(a)
    batched = None if (a.no_batch or not solo) else measure_batched(a, checks)
    serving = None if (a.no_serve or not solo) else measure_serving(a)
    if checks is not None:
        t0 = time.perf_counter()
        got = checks.results(timeout=300.0)
        wait_s = time.perf_counter() - t0
        if batched is not None:
            batched["oracle_check"] = oracle_errors(batched["_jobs"], "batch", got)
        if serving is not None:
            serving["oracle_check"] = oracle_errors(serving["_jobs"], "serve", got)
        if small is not None and ("small", 0) in got:
            import numpy as np

            _, N_or, P1_or, psi_or = got[("small", 0)]
            small["oracle_check"] = {
                "state_err": float(np.linalg.norm(small["_state"] - psi_or) / np.linalg.norm(psi_or)),
                "P1_err": abs(small["graph_replay"]["P1"] - P1_or), "grid_steps_equal": N_or == small["grid_steps"],
                "state_bar": 1e-10}
        oracle_note = {"workers": checks.workers, "submitted": len(checks.pending), "finished": len(got),
                       "extra_wait_s": wait_s}
    else:
        oracle_note = None
    for leg in (batched, serving, small):
        if leg is not None:
            leg.pop("_jobs", None)
            leg.pop("_state", None)
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        gbs, cores, desc, _ = cpu_sample()
        cpu = {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": desc}
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    traffic = profiled_traffic("c64", n)
    line = {
        "metric": METRIC,
        "value": r64["value"],
        "unit": "GB/s",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": r64["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "precision": "complex64 state, FP32 arithmetic, FP64 reductions",
        "data": "synthetic (seeded EC3 instance)",
        "config": {
            "workload": f"ec3-n{n}-seed{SEED}-linear-T{T_RUN:g}-uniform",
            "n_qubits": n,
            "path": "linear s=t/T",
            "T": T_RUN,
            "grid_steps": r64["n_steps_grid"],
            "bench_step": f"init + 3 RK4 + {a.pec} PEC grid steps + P1/E readback",
            "parallelism": f"replicas x{world}",
            "l2": f"no flush: each state vector ({(1 << n) * 8 / 2**30:.0f} GiB) is far larger than L2",
        },
        "roofline": {
            "bound": "hbm",
            "kernel": ("fused PEC step, per grid step: k_apply partial pass(es) + k_slab (last partial layout "
                       "and step over L2-sized slabs)" if a.slab_bits != 0 else
                       "fused PEC step, per grid step: k_partial_x (TMA) partial passes + k_apply MODE_STEP"),
            "achieved": r64["pec_step_gbs"],
            "peak": hbm_peak,
            "peak_kind": peak_kind,
            "unit": "GB/s",
            "frac": r64["pec_step_gbs"] / hbm_peak,
            "traffic": traffic,
            "alg_bytes_per_launch": 7 * (1 << n) * 8,
        },
        "matvec": {
            "what": "aqc_hpsi: out = H(t) psi (all layout passes), device buffers",
            "ms": r64["matvec_ms"],
            "alg_bytes": 2 * (1 << n) * 8,
            "achieved": 2 * (1 << n) * 8 / (r64["matvec_ms"] * 1e-3) / 1e9,
            "unit": "GB/s",
            "frac": 2 * (1 << n) * 8 / (r64["matvec_ms"] * 1e-3) / 1e9 / hbm_peak,
            "moved_bytes_as_built": (3 * len_layouts(n, 13, 5) - 1) * (1 << n) * 8,
        },
        "cpu_baseline": cpu,
        "e2e": r64.get("e2e"),
        "gpu_launches": r64["launches"],
        "clocks": r64["clocks"],
        "fidelity_P1_window": r64["P1"],
        "small_state": small,
        "batched": batched,
        "serving": serving,
        "oracle_checks": oracle_note,
        "y_compensation": ycomp,
        "xy_algorithm": xy,
    }
    if r128 is not None:
        flops = pec_flops_c128(n) * (1 << n)
        if fp64 is not None:
            fp64_peak, fp64_kind = fp64["tflops"], "measured in this run (aqc_measure_fp64_fma)"
        else:
            fp64_peak, fp64_kind = 1.25, "nominal FP64 (no measurement in this run)"
        line["c128"] = {
            "dtype": "f64",
            "value": r128["value"],
            "unit": "GB/s",
            "ms_per_step": r128["ms_per_step"],
            "pec_step_ms": r128["pec_step_ms"],
            "roofline": {
                "bound": "alu",
                "achieved": flops / (r128["pec_step_ms"] * 1e-3) / 1e12,
                "peak": fp64_peak,
                "peak_kind": fp64_kind,
                "unit": "TFLOP/s",
                "frac": flops / (r128["pec_step_ms"] * 1e-3) / 1e12 / fp64_peak,
                "hbm_frac": r128["pec_step_gbs"] / hbm_peak,
                "traffic": profiled_traffic("c128", n),
                "fp64_fma_measurement": fp64,
            },
            "e2e": r128.get("e2e"),
            "gpu_launches": r128["launches"],
            "clocks": r128["clocks"],
            "P1_c128_minus_c64": r128["P1"] - r64["P1"],
        }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_reference(a):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per_step = max(5.0, min(20.0, 150.0 / max(1, a.steps + a.warmup)))
    for _ in range(a.warmup):
        cpu_sample(per_step)
    vals, secs, desc, cores = [], [], "", 1
    for _ in range(a.steps):
        gbs, cores, desc, dt = cpu_sample(per_step)
        vals.append(gbs)
        secs.append(dt)
    v = statistics.mean(vals)
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": v,
        "unit": "GB/s",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": 1e3 * statistics.mean(secs),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded EC3 instance)",
        "config": {"workload": f"ec3-n{N_QUBITS}-seed{SEED}-linear-T{T_RUN:g}-uniform",
                   "sample": "n=22 member of the same workload family, bounded step count"},
        "cpu_baseline": {"value": v, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.only_xy:
        run_xy_only(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
