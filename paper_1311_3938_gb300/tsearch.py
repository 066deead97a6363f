"""Successful runtime T_s (Sec. III.B): the runtime T at which the final energy E(T)/Omega
reaches 1/2 (every excited state of H_f costs at least Omega, so E = 1/2 bounds P_1 >= 1/2).

`search_Ts` brackets the first crossing E(T) = target on a geometric grid of k runtimes per
round, evaluated together (one batch of solves on the GPU), and shrinks the bracket until its
ratio is below 1 + rtol; the result interpolates log T linearly in E between the bracket's
ends.  `gpu_energies` turns a job template into such an evaluator: every runtime of a round is
one member of a batch (or one context for large n), all solved by libaqc.so.
"""
from __future__ import annotations

import math
from dataclasses import replace


def _geom(lo, hi, k):
    return [lo * (hi / lo) ** (i / (k - 1)) for i in range(k)]


def search_Ts(energies, T_lo, T_hi, target=0.5, k=8, rtol=1e-3, max_rounds=16, max_expand=8, T_max=1024.0):
    """First crossing of E(T) = target between T_lo and T_hi (widened by factors of 4 if E at
    the ends does not straddle the target, never beyond T_max: a path whose gap closes never
    reaches the target).  energies(list of T) -> list of E.  Returns a dict: Ts (None if no
    crossing was found), bracket, rounds, evaluations."""
    if not (0 < T_lo < T_hi) or k < 3:
        raise ValueError("need 0 < T_lo < T_hi and k >= 3")
    seen = {}

    def ev(Ts):
        need = [T for T in Ts if T not in seen]
        if need:
            for T, E in zip(need, energies(need)):
                seen[T] = float(E)
        return [seen[T] for T in Ts]

    lo, hi = float(T_lo), float(T_hi)
    for _ in range(max_expand):
        e_lo, e_hi = ev([lo, hi])
        if e_lo <= target:  # already adiabatic enough at lo: the crossing lies below
            lo, hi = lo / 4.0, lo
        elif e_hi > target:  # not yet at hi: look further up, up to T_max
            if hi >= T_max:
                return {"Ts": None, "bracket": (lo, hi), "rounds": 0, "evaluations": len(seen)}
            lo, hi = hi, min(hi * 4.0, T_max)
        else:
            break
    else:
        return {"Ts": None, "bracket": (lo, hi), "rounds": 0, "evaluations": len(seen)}
    rounds = 0
    while hi / lo > 1.0 + rtol and rounds < max_rounds:
        grid = _geom(lo, hi, k)
        E = ev(grid)
        i = next(j for j in range(1, k) if E[j] <= target)  # E[0] > target >= E[-1]
        lo, hi = grid[i - 1], grid[i]
        rounds += 1
    e_lo, e_hi = ev([lo, hi])
    f = 0.0 if e_lo == e_hi else (e_lo - target) / (e_lo - e_hi)
    Ts = math.exp(math.log(lo) + f * (math.log(hi) - math.log(lo)))
    return {"Ts": Ts, "bracket": (lo, hi), "rounds": rounds, "evaluations": len(seen)}


def gpu_energies(job, device=0, batch_max_n=22):
    """E(T) evaluator for the instance, algorithm and precision of `job` (workloads.Job): each
    call solves every requested runtime, as one batch when n <= batch_max_n."""
    from . import workloads as W

    def f(Ts):
        jobs = [replace(job, jid=i, T=float(T), state=None) for i, T in enumerate(Ts)]
        if job.n <= batch_max_n and len(jobs) > 1:
            W.run_batched(jobs, device)
        else:
            for j in jobs:
                W.solve_single(j, device)
        return [j.E for j in jobs]

    return f


def find_Ts(job, T_lo=1.0, T_hi=64.0, k=8, rtol=1e-2, device=0, T_max=1024.0):
    """T_s of one job template (its T is ignored)."""
    return search_Ts(gpu_energies(job, device), T_lo, T_hi, k=k, rtol=rtol, T_max=T_max)
