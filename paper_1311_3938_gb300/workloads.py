"""Batched solves and a continuous-batching request server on top of the C ABI.

* `Job`: one Exact-Cover-3 solve (instance seed, n, path, T, precision).
* `solve_single(job)`: the job alone through aqc_propagate (one context, its own stream).
* `run_batched(jobs, ...)`: all jobs as members of one aqc_batch (K PEC steps per graph
  replay), members retired as they reach t = T.
* `Server`: requests arrive over time (Poisson); each is admitted when its workspace fits the
  HBM budget; small states join the running batch between rounds (continuous batching), large
  states run on their own streams concurrently with the batch; finished jobs are retired and
  their memory released.  Reports p50/p99 latency, solves/s and HBM occupancy.

All device work is libaqc.so's; this module only schedules it.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from instances import SplitMix64, generate_ec3, generate_ec3_hard, xx_pairs

from . import _native as N
from . import hamiltonians as HB
from .engine import Batch, Context


@dataclass
class Job:
    jid: int
    n: int
    seed: int
    nonlinear: bool
    T: float
    precision: int = N.AQC_C64
    s_kind: int = N.AQC_S_LINEAR
    arrival: float = 0.0
    driver: str = "x"      # "x" (Eq. Hix, start |S>); "xy" (Eq. Hixy, start: its sector ground
                           # state); "xyz" (Eq. Hixyz, start: the Dicke state, its sector ground state)
    alpha: float = 8.0     # catalyst strength of the XY/XYZ nonlinear path (Eq. nlpath)
    hard: bool = False     # instance by the hard-instance recipe of Sec. I.E
    # filled in when the job is served
    admitted: float = math.nan
    finished: float = math.nan
    P1: float = math.nan
    E: float = math.nan
    norm2: float = math.nan
    steps: int = 0
    route: str = ""
    keep: bool = False         # keep the final state (job.state) when the job finishes
    P1_c128: float = math.nan  # the same job re-solved on the GPU's complex128 path, if checked
    state: np.ndarray = field(default=None, repr=False)

    @property
    def P1_err_vs_c128(self):
        """|P_1 - P_1(complex128 GPU path)|: this result's fidelity against the library's own
        FP64 path (a check of the FP32 state's rounding, not an independent reference)."""
        return abs(self.P1 - self.P1_c128)

    @property
    def latency(self):
        return self.finished - self.arrival

    def workspace_bytes(self):
        return N.aqc_workspace_bytes(self.n, self.precision)


_INSTANCE_CACHE = {}


def _instance(n, seed, hard=False):
    key = (n, seed, hard)
    if key not in _INSTANCE_CACHE:
        _INSTANCE_CACHE[key] = generate_ec3_hard(n, seed) if hard else generate_ec3(n, seed)
    return _INSTANCE_CACHE[key]


def make_context(job: Job, device=0, stream=None, tile_bits=0) -> tuple:
    inst = _instance(job.n, job.seed, job.hard)
    pairs = xx_pairs(job.n, job.seed) if job.nonlinear else None
    ctx = Context(job.n, job.precision, device=device, stream=stream)
    if tile_bits:
        ctx.set_tile_bits(tile_bits)
    if job.driver == "x":
        HB.load_ec3(ctx, inst, pairs=pairs)
        ctx.set_schedule(job.T, HB.nonlinear_schedule() if job.nonlinear else HB.linear_schedule(), job.s_kind)
        ctx.set_integrator(0, 0.0)
        ctx.set_initial_state("uniform")
    else:  # XY / XYZ algorithm; the nonlinear path adds the catalyst alpha s(1-s) H_{m-1}
        sched, k = HB.load_xy(ctx, inst, driver=job.driver, catalyst_alpha=job.alpha if job.nonlinear else 0.0)
        ctx.set_schedule(job.T, sched, job.s_kind)
        ctx.set_integrator(0, 0.0)
        if job.driver == "xy":
            HB.set_xy_ground_start(ctx, k)
        else:
            ctx.set_initial_state(("dicke", k))
    return ctx, inst


def _finish(job: Job, ctx: Context, inst, keep_state: bool):
    job.P1 = ctx.fidelity(inst.solution)
    job.E = ctx.energy(N.AQC_GRP_B)
    job.norm2 = ctx.norm2()
    if keep_state or job.keep:
        job.state = ctx.state()


def solve_single(job: Job, device=0, keep_state=False, stream=None) -> Job:
    """The job alone: one context, aqc_propagate to t = T."""
    ctx, inst = make_context(job, device, stream)
    st = ctx.propagate(-1)
    job.steps = st["steps_done"]
    job.route = "single"
    _finish(job, ctx, inst, keep_state)
    ctx.close()
    return job


def random_jobs(count, seed, n_range=(12, 22), T_range=(10.0, 200.0), nonlinear=True, precision=N.AQC_C64,
                rate=None, big_every=0, big_n=30, s_kind=N.AQC_S_LINEAR, path_mix=False, big_T_range=None):
    """Seeded job list: n ~ U{n_range}, T ~ U[T_range], instance seeds seed..seed+count-1;
    with `rate`, Poisson arrival times (exponential gaps of mean 1/rate seconds); every
    `big_every`-th job has n = big_n (and T ~ U[big_T_range] if given); `path_mix` draws
    linear/nonlinear uniformly."""
    rng = SplitMix64(seed * 7919 + 17)
    jobs = []
    t = 0.0
    for k in range(count):
        n = n_range[0] + rng.below(n_range[1] - n_range[0] + 1)
        T = T_range[0] + (T_range[1] - T_range[0]) * rng.uniform()
        if big_every and (k + 1) % big_every == 0:
            n = big_n
            if big_T_range:
                T = big_T_range[0] + (big_T_range[1] - big_T_range[0]) * (T - T_range[0]) / max(1e-300, T_range[1] - T_range[0])
        nl = (rng.below(2) == 1) if path_mix else nonlinear
        if rate:
            t += -math.log(1.0 - rng.uniform()) / rate
        jobs.append(Job(jid=k, n=n, seed=seed + k, nonlinear=nl, T=T, precision=precision, s_kind=s_kind, arrival=t))
    return jobs


def run_batched(jobs, device=0, threads=256, steps_per_round=16, rounds_per_poll=4, keep_state=False,
                tile_bits=0, max_members=None):
    """Every job a member of one batch; members retire at t = T.  Returns wall seconds."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mm = max_members or len(jobs)
    items = 1
    for j in jobs:
        items += 1 << max(0, j.n - (tile_bits or (13 if j.precision == N.AQC_C64 else 12)) + 3)
    b = Batch(jobs[0].precision, device=device, max_members=mm, max_items=max(items, 1024), threads=threads,
              steps_per_round=steps_per_round)
    live = {}
    queue = list(jobs)
    while queue or live:
        while queue and len(live) < mm:
            job = queue.pop(0)
            ctx, inst = make_context(job, device, tile_bits=tile_bits)
            slot = b.add(ctx)
            live[slot] = (job, ctx, inst)
        b.run(rounds_per_poll)
        steps, active, _ = b.poll()
        for slot in list(live):
            job, ctx, inst = live[slot]
            if steps[slot] >= 0 and b.members.get(slot) is ctx and steps[slot] >= _nsteps(ctx, job):
                b.remove(slot)
                job.steps = steps[slot]
                job.route = "batch"
                _finish(job, ctx, inst, keep_state)
                ctx.close()
                del live[slot]
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    b.close()
    return dt


def _nsteps(ctx, job):
    """N of the context's step grid (asked once from the library)."""
    if getattr(ctx, "_nsteps", None) is None:
        ctx._nsteps = ctx.grid()[0]
    return ctx._nsteps


def attach_c128_errors(jobs, min_n=0, max_n=20, device=0):
    """For complex64 results with min_n <= n <= max_n, solve the same job on the library's
    complex128 path and store its P_1 (job.P1_c128), so each result states how far its FP32
    state's rounding moved the fidelity."""
    import copy

    for job in jobs:
        if job.precision != N.AQC_C64 or not (min_n <= job.n <= max_n) or math.isnan(job.P1):
            continue
        ref = copy.deepcopy(job)
        ref.precision = N.AQC_C128
        ref.state = None
        ref.keep = False
        solve_single(ref, device)
        job.P1_c128 = ref.P1
    return jobs


def run_sweep_n20(seed=2, n=20, Ts=(10.0, 50.0, 200.0), device=0):
    """The n = 20 workload: linear and nonlinear paths x s = t/T and smoothstep x T, in
    complex128 and complex64; per run P_1, E, norm^2 - 1, grid steps, seconds, and the
    complex64 fidelity error against the complex128 (FP64) result."""
    rows = []
    for nonlinear in (False, True):
        for s_kind in (N.AQC_S_LINEAR, N.AQC_S_SMOOTHSTEP):
            for T in Ts:
                res = {}
                for prec in (N.AQC_C128, N.AQC_C64):
                    job = Job(jid=0, n=n, seed=seed, nonlinear=nonlinear, T=T, precision=prec, s_kind=s_kind)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    solve_single(job, device)
                    torch.cuda.synchronize()
                    res[prec] = (job, time.perf_counter() - t0)
                j128, t128 = res[N.AQC_C128]
                j64, t64 = res[N.AQC_C64]
                rows.append({
                    "path": "nonlinear" if nonlinear else "linear",
                    "s": "smoothstep" if s_kind == N.AQC_S_SMOOTHSTEP else "t/T",
                    "T": T,
                    "grid_steps": j128.steps,
                    "P1_c128": j128.P1,
                    "E_c128": j128.E,
                    "norm2_minus_1_c128": j128.norm2 - 1.0,
                    "seconds_c128": t128,
                    "P1_c64": j64.P1,
                    "P1_err_c64_vs_fp64": abs(j64.P1 - j128.P1),
                    "seconds_c64": t64,
                })
    return rows


def serve_one_at_a_time(jobs, device=0, time_limit=None, chunk_amplitude_steps=1 << 26, order="arrival"):
    """The one-at-a-time baseline of a request stream: each job alone on the GPU (one context),
    started once it has arrived and the previous one is done -- the next one in arrival order,
    or (order "shortest") the arrived job of least work_estimate; propagated in chunks of about
    `chunk_amplitude_steps` / 2^n grid steps so that a time limit ends the run between chunks
    (the job then in progress is censored).  Returns (finished jobs, censored jobs, wall
    seconds)."""
    if order not in ("arrival", "shortest"):
        raise ValueError("order must be 'arrival' or 'shortest'")
    pending = sorted(jobs, key=lambda j: j.arrival)
    done, censored = [], []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    now = lambda: time.perf_counter() - t0  # noqa: E731
    while pending:
        if time_limit and now() > time_limit:
            break
        wait = pending[0].arrival - now()
        if wait > 0:
            if time_limit and pending[0].arrival > time_limit:
                break
            time.sleep(wait)
        if order == "shortest":
            t = now()
            job = min((j for j in pending if j.arrival <= t), key=work_estimate)
        else:
            job = pending[0]
        del pending[next(i for i, p in enumerate(pending) if p is job)]
        job.admitted = now()
        ctx, inst = make_context(job, device)
        chunk = max(16, chunk_amplitude_steps >> job.n)
        total = _nsteps(ctx, job)
        steps = 0
        while steps < total and not (time_limit and now() > time_limit):
            ctx.propagate(min(chunk, total - steps), stats=False)
            ctx.stream.synchronize()
            steps = min(total, steps + chunk)
        if steps < total:
            ctx.close()
            censored.append(job)
            break
        job.steps = total
        job.route = "single"
        _finish(job, ctx, inst, False)
        job.finished = now()
        ctx.close()
        done.append(job)
    return done, censored, now()


def run_sequential(jobs, device=0, keep_state=False):
    """Every job alone, one after another (the one-at-a-time baseline).  Returns wall seconds."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for job in jobs:
        solve_single(job, device, keep_state)
    torch.cuda.synchronize()
    return time.perf_counter() - t0


def run_batch512(count=512, seed=1000, device=0, sample_every=16):
    """The batched workload at full size: `count` instances from `seed`, n ~ U{12..22}, nonlinear
    path, T ~ U[10, 200], complex64, all as members of one batch (autotuned shape).  One-at-a-time
    solves of every job would take hours, so the comparison runs on every `sample_every`-th job:
    batched and sequential on that sample, equal step grids."""
    import copy

    from . import autotune as A

    jobs = random_jobs(count, seed, n_range=(12, 22), T_range=(10.0, 200.0), nonlinear=True)
    shape, _ = A.autotune(jobs[:16], rounds=3)
    tile_bits, threads, spr = shape
    t_all = run_batched(jobs, device, threads=threads, steps_per_round=spr, tile_bits=tile_bits)
    sample = [copy.deepcopy(j) for j in jobs[::sample_every]]
    sb = copy.deepcopy(sample)
    t_sb = run_batched(sb, device, threads=threads, steps_per_round=spr, tile_bits=tile_bits)
    t_ss = run_sequential(sample, device)
    amp_steps = sum(j.steps * (1 << j.n) for j in jobs)
    return {"workload": f"{count} EC3 instances, seeds {seed}-{seed + count - 1}, n~U{{12..22}}, nonlinear, "
                        "T~U[10,200], complex64",
            "grid_steps_total": sum(j.steps for j in jobs), "amplitude_steps": amp_steps,
            "wall_s_batched": t_all, "solves_per_s_batched": count / t_all,
            "alg_GBs_batched": 7 * 8 * amp_steps / t_all / 1e9,
            "sample": len(sample), "sample_wall_s_batched": t_sb, "sample_wall_s_sequential": t_ss,
            "sample_speedup": t_ss / t_sb,
            "sample_max_abs_dP1": max(abs(a.P1 - b.P1) for a, b in zip(sb, sample)),
            "autotuned_shape": {"tile_bits": tile_bits, "threads": threads, "steps_per_round": spr}}


def run_algorithms(n=13, seed=3, Ts=(2.0, 5.0, 10.0, 20.0, 50.0), precision=N.AQC_C64, device=0):
    """The algorithms of Sec. III-IV on one instance: X (from |S>), XYZ (from the Dicke state of
    the solution's weight), XY (from the ground state of H^xy in that sector) and XY with the
    alpha = 8 catalyst (Eq. nlpath), each over runtimes T: final P_1, energy E and wall seconds
    per solve (the start-state preparation included)."""
    rows = []
    for driver, nonlinear in (("x", False), ("xyz", False), ("xy", False), ("xy", True)):
        for T in Ts:
            job = Job(jid=0, n=n, seed=seed, nonlinear=nonlinear, T=T, precision=precision, driver=driver)
            t0 = time.perf_counter()
            solve_single(job, device)
            rows.append({"algorithm": driver + ("+catalyst" if nonlinear else ""), "n": n, "T": T,
                         "grid_steps": job.steps, "P1": job.P1, "E": job.E, "norm2_minus_1": job.norm2 - 1.0,
                         "seconds": time.perf_counter() - t0})
    return rows


def run_ts_scaling(ns=(8, 10, 12), count=8, seed=5000, drivers=("x", "xy"), precision=N.AQC_C64,
                   device=0, T_max=512.0, hard=True):
    """Median successful runtime T_s (E(T_s)/Omega = 1/2, Sec. III.B) over `count` seeded hard
    instances (Sec. I.E) per n and algorithm, each T_s found by batched solves (tsearch.find_Ts)."""
    from .tsearch import find_Ts

    rows = []
    for n in ns:
        for driver in drivers:
            ts, evals = [], 0
            t0 = time.perf_counter()
            for k in range(count):
                job = Job(jid=k, n=n, seed=seed + 100 * n + k, nonlinear=False, T=1.0, precision=precision,
                          driver=driver, hard=hard)
                r = find_Ts(job, T_lo=1.0, T_hi=64.0, k=8, rtol=1e-2, device=device, T_max=T_max)
                evals += r["evaluations"]
                if r["Ts"] is not None:
                    ts.append(r["Ts"])
            rows.append({"n": n, "algorithm": driver, "instances": count, "found": len(ts),
                         "median_Ts": float(np.median(ts)) if ts else None,
                         "min_Ts": min(ts) if ts else None, "max_Ts": max(ts) if ts else None,
                         "solves": evals, "seconds": time.perf_counter() - t0})
    return rows


def run_gap_curves(n=13, seed=3, s_points=25, precision=N.AQC_C128, device=0, max_iter=200):
    """Gap between the two lowest eigenvalues of H(s) along the path (Fig. 41N13, bottom) for
    the X algorithm (full space, random start), the XY algorithm and the XY algorithm with the
    alpha = 8 catalyst (solution's Hamming-weight sector, Dicke start), by aqc_lanczos; minimum
    gap, where it sits, and milliseconds per Lanczos solve."""
    from instances import random_state

    inst = _instance(n, seed)
    k = bin(int(inst.solution)).count("1")
    s_grid = [0.02 + 0.96 * i / (s_points - 1) for i in range(s_points)]
    rows = []
    for driver, alpha in (("x", 0.0), ("xy", 0.0), ("xy", 8.0)):
        ctx = Context(n, precision, device=device)
        if driver == "x":
            HB.load_ec3(ctx, inst)
            ctx.set_schedule(1.0, HB.linear_schedule())
            start = torch.from_numpy(random_state(n, seed)).to(ctx.dev)
        else:
            sched, _ = HB.load_xy(ctx, inst, driver=driver, catalyst_alpha=alpha)
            ctx.set_schedule(1.0, sched)
            ctx.set_initial_state(("dicke", k))
            start = ctx.state(device=True)
        gaps, ms = [], []
        for sv in s_grid:
            t0 = time.perf_counter()
            eig, conv, iters = ctx.lanczos(sv, start, max_iter=max_iter, n_eig=2, tol=1e-11)
            ms.append((time.perf_counter() - t0) * 1e3)
            gaps.append(eig[1] - eig[0])
        ctx.close()
        j = int(np.argmin(gaps))
        rows.append({"algorithm": driver + ("+catalyst" if alpha else ""), "n": n, "sector_weight": None if driver == "x" else k,
                     "min_gap": gaps[j], "s_at_min": s_grid[j], "gaps": gaps, "s": s_grid,
                     "ms_per_lanczos": float(np.median(ms))})
    return rows


def _main():
    import argparse
    import json

    ap = argparse.ArgumentParser(description="workload drivers")
    ap.add_argument("what", choices=["sweep20", "algorithms", "ts", "gap", "batch512"])
    ap.add_argument("--n", type=int, default=13)
    a = ap.parse_args()
    if a.what == "sweep20":
        for row in run_sweep_n20():
            print(json.dumps(row), flush=True)
    elif a.what == "algorithms":
        for row in run_algorithms(n=a.n):
            print(json.dumps(row), flush=True)
    elif a.what == "ts":
        for row in run_ts_scaling():
            print(json.dumps(row), flush=True)
    elif a.what == "gap":
        for row in run_gap_curves(n=a.n):
            print(json.dumps(row), flush=True)
    elif a.what == "batch512":
        print(json.dumps(run_batch512()), flush=True)


def admit_ready(pending, now, used, budget, n_members, max_members, batch_max_n, start):
    """Admit arrived jobs from the head of `pending` (sorted by arrival) in FIFO order.

    A job is admitted while its workspace fits the HBM budget (`used` + its bytes <= `budget`)
    and, for a small job (n <= batch_max_n, a batch member), while the batch has fewer than
    `max_members` members (`n_members()`); the first arrived job that does not fit waits and
    blocks the jobs behind it (no overtaking).  Each admitted job leaves `pending` and is passed
    to `start(job, small)`, which creates its context.  `now()` is read for every job, so jobs
    that arrive while earlier ones start are admitted in the same pass.  Returns the new
    `used`."""
    while pending and pending[0].arrival <= now():
        job = pending[0]
        need = job.workspace_bytes()
        small = job.n <= batch_max_n
        if used + need > budget or (small and n_members() >= max_members):
            break
        pending.pop(0)
        used += need
        start(job, small)
    return used


def work_estimate(job):
    """T n 2^n: a solve's grid steps (the step rule's N grows with T times the Hamiltonian's norm
    bound, which grows with n) times its amplitudes, up to a constant; orders jobs by cost."""
    return job.T * job.n * float(1 << job.n)


def admit_shortest_first(pending, now, used, budget, n_members, max_members, batch_max_n, n_large, max_large,
                         start):
    """Admit arrived jobs of `pending` in order of work_estimate: a small job (n <= batch_max_n,
    a batch member) while the batch has fewer than `max_members` members, a large one while fewer
    than `max_large` large jobs run (`n_large()`); a job whose workspace does not fit the HBM
    budget waits without blocking smaller jobs behind it.  Returns the new `used`."""
    t = now()
    arrived = sorted((j for j in pending if j.arrival <= t), key=work_estimate)
    for job in arrived:
        small = job.n <= batch_max_n
        if small and n_members() >= max_members:
            continue
        if not small and n_large() >= max_large:
            continue
        need = job.workspace_bytes()
        if used + need > budget:
            continue
        del pending[next(i for i, p in enumerate(pending) if p is job)]
        used += need
        start(job, small)
    return used


class Server:
    """Continuous-batching request loop (see the module docstring).

    policy "fifo": arrived jobs are admitted in arrival order as memory and the member limit
    allow (admit_ready), every admitted large job runs at once.  policy "shortest": arrived jobs
    are admitted in order of estimated work (admit_shortest_first) and at most `max_large` large
    jobs run at a time; the large jobs' states are bandwidth-bound, so running several at once
    adds no throughput and only delays each of them.  large_grid > 0 caps every launch of a
    large job at that many CTAs (aqc_set_grid_limit): its persistent kernels would otherwise
    hold every SM for their whole duration, and each batch launch would wait for one to end."""

    def __init__(self, precision=N.AQC_C64, device=0, hbm_budget=None, reserve=2 << 30, batch_max_n=22,
                 max_members=256, threads=256, steps_per_round=16, big_chunk=64, keep_state=False,
                 big_first=False, policy="fifo", max_large=1, large_grid=0):
        if policy not in ("fifo", "shortest"):
            raise ValueError("policy must be 'fifo' or 'shortest'")
        self.policy = policy
        self.max_large = max_large
        self.large_grid = large_grid  # CTA limit of a large job's launches (0: none; aqc_set_grid_limit)
        self.precision = precision
        self.device = device
        free, total = torch.cuda.mem_get_info(device)
        self.budget = int(hbm_budget if hbm_budget is not None else free - reserve)
        self.batch_max_n = batch_max_n
        self.max_members = max_members
        self.big_chunk = big_chunk
        self.keep_state = keep_state
        max_items = max_members * (1 << max(0, batch_max_n - 13 + 2)) + 1024
        # the batch (many short jobs) runs on a high-priority stream, large jobs on low-priority
        # streams, so CTAs of batch rounds are scheduled first whenever SMs free up; big_first
        # swaps the two (large jobs finish sooner, the batch yields while they run)
        lo, hi = torch.cuda.Stream.priority_range()
        self.hi_prio, self.lo_prio = (lo, hi) if big_first else (hi, lo)
        self.batch = Batch(precision, device=device, max_members=max_members, max_items=max_items, threads=threads,
                           steps_per_round=steps_per_round,
                           stream=torch.cuda.Stream(device, priority=self.hi_prio))
        self.used = 0
        self.peak_used = 0
        self.occupancy = []

    def serve(self, jobs, time_limit=None):
        """Serve `jobs` (arrival times in seconds from now).  Returns a metrics dict."""
        pending = sorted(jobs, key=lambda j: j.arrival)
        in_batch = {}  # slot -> (job, ctx, inst)
        big = []  # [job, ctx, inst, stream, event, steps_enqueued]
        done = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731
        prof = {"admit_s": 0.0, "advance_s": 0.0, "poll_s": 0.0, "retire_s": 0.0, "rounds": 0}
        while pending or in_batch or big:
            if time_limit and now() > time_limit:
                break
            # admission: FIFO among arrived jobs, as memory allows
            ta = time.perf_counter()

            def start(job, small):
                job.admitted = now()
                if small:
                    ctx, inst = make_context(job, self.device)
                    slot = self.batch.add(ctx)
                    in_batch[slot] = (job, ctx, inst)
                else:
                    stream = torch.cuda.Stream(self.device, priority=self.lo_prio)
                    ctx, inst = make_context(job, self.device, stream=stream)
                    if self.large_grid:
                        ctx.set_grid_limit(self.large_grid)
                    big.append([job, ctx, inst, stream, None, 0, []])

            if self.policy == "fifo":
                self.used = admit_ready(pending, now, self.used, self.budget, lambda: len(in_batch),
                                        self.max_members, self.batch_max_n, start)
            else:
                self.used = admit_shortest_first(pending, now, self.used, self.budget, lambda: len(in_batch),
                                                 self.max_members, self.batch_max_n, lambda: len(big),
                                                 self.max_large, start)
            self.peak_used = max(self.peak_used, self.used)
            prof["admit_s"] += time.perf_counter() - ta
            self.occupancy.append(self.used / max(1, self.budget))
            if not in_batch and not big:
                if pending:
                    time.sleep(min(0.01, max(0.0, pending[0].arrival - now())))
                continue
            # advance: one batch round and one chunk per large job, on different streams
            ta = time.perf_counter()
            prof["rounds"] += 1
            if in_batch:
                self.batch.run(1)
            for entry in big:
                job, ctx, inst, stream, ev, enq, inflight = entry
                # at most two chunks of a large job in flight, so batch rounds interleave
                while inflight and inflight[0].query():
                    inflight.pop(0)
                if ev is None and len(inflight) < 2:
                    ctx.propagate(self.big_chunk, stats=False)
                    entry[5] = enq + self.big_chunk
                    e = torch.cuda.Event()
                    e.record(stream)
                    inflight.append(e)
                    if entry[5] >= _nsteps(ctx, job):
                        entry[4] = e
            prof["advance_s"] += time.perf_counter() - ta
            # retire finished work
            ta = time.perf_counter()
            if in_batch:
                steps, _, _ = self.batch.poll()
            prof["poll_s"] += time.perf_counter() - ta
            ta = time.perf_counter()
            if in_batch:
                for slot in list(in_batch):
                    job, ctx, inst = in_batch[slot]
                    if steps[slot] >= _nsteps(ctx, job):
                        self.batch.remove(slot)
                        job.steps = steps[slot]
                        job.route = "batch"
                        _finish(job, ctx, inst, self.keep_state)
                        job.finished = now()
                        ctx.close()
                        self.used -= job.workspace_bytes()
                        del in_batch[slot]
                        done.append(job)
            for entry in list(big):
                job, ctx, inst, stream, ev, enq, inflight = entry
                if ev is not None and ev.query():
                    job.steps = _nsteps(ctx, job)
                    job.route = "stream"
                    _finish(job, ctx, inst, self.keep_state)
                    job.finished = now()
                    ctx.close()
                    self.used -= job.workspace_bytes()
                    big.remove(entry)
                    done.append(job)
            prof["retire_s"] += time.perf_counter() - ta
            if not in_batch and big and all(len(e[6]) >= 2 or e[4] is not None for e in big):
                time.sleep(2e-4)  # only large jobs in flight: do not spin
        wall = now()
        # a time limit leaves work in flight: release it (those requests are censored)
        censored = []
        for slot in list(in_batch):
            job, ctx, inst = in_batch.pop(slot)
            self.batch.remove(slot)
            ctx.close()
            self.used -= job.workspace_bytes()
            censored.append(job)
        for entry in big:
            job, ctx, inst, stream = entry[0], entry[1], entry[2], entry[3]
            stream.synchronize()
            ctx.close()
            self.used -= job.workspace_bytes()
            censored.append(job)
        big.clear()
        lat = np.array([j.latency for j in done]) if done else np.array([math.nan])
        by_route = {}
        for route in ("batch", "stream"):
            lr = np.array([j.latency for j in done if j.route == route])
            if lr.size:
                by_route[route] = {"count": int(lr.size), "p50_latency_s": float(np.percentile(lr, 50)),
                                   "p99_latency_s": float(np.percentile(lr, 99))}
        return {
            "completed": len(done),
            "wall_s": wall,
            "solves_per_s": len(done) / wall if wall > 0 else math.nan,
            "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)),
            "hbm_budget_bytes": self.budget,
            "hbm_peak_bytes": self.peak_used,
            "hbm_mean_occupancy": float(np.mean(self.occupancy)) if self.occupancy else 0.0,
            "by_route": by_route,
            "loop": prof,
            "jobs": done,
            "censored_jobs": censored,   # admitted, unfinished at the time limit
            "not_admitted": pending,     # arrived (or not yet) and never admitted
        }

    def close(self):
        self.batch.close()


if __name__ == "__main__":
    _main()
