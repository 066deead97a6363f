"""Seeded Exact-Cover-3 instances (Sec. I.C-D of the paper) and random qubit pairs.

An instance is a set of m distinct clauses, each a triple of distinct bits; a clause is
satisfied when exactly one of its three bits is 1 (Eq. 1clause, Eq. sat).  Bits are 0-based
here: bit k is qubit k+1 of the paper and has weight 2**k in the basis index z (Eq. ztensor).

Generation rule (the workload's rule, with the paper's discard/restart steps of Sec. I.D):
clauses are drawn uniformly at random among the distinct triples not drawn yet; a clause that
would leave no satisfying assignment is discarded; drawing stops as soon as exactly one
satisfying assignment is left; if the pool of triples runs dry first, the generator restarts.
Solution counting is exact (a depth-first search with unit propagation that stops at two
solutions); tests check it against brute-force enumeration.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from math import comb

from .rng import SplitMix64


@dataclass(frozen=True)
class EC3Instance:
    n: int
    clauses: tuple  # tuple of (a, b, c) with a < b < c, 0-based bits
    solution: int  # the unique satisfying assignment w
    seed: int
    restarts: int = 0

    @property
    def m(self) -> int:
        return len(self.clauses)

    def clause_counts(self):
        """n_i (clauses touching bit i) and n_ij (clauses touching bits i and j), Eq. final_ham."""
        ni = [0] * self.n
        nij = {}
        for c in self.clauses:
            for a in c:
                ni[a] += 1
            for x in range(3):
                for y in range(x + 1, 3):
                    key = (c[x], c[y])
                    nij[key] = nij.get(key, 0) + 1
        return ni, nij


def _propagate(clause_masks, one, zero):
    """Unit propagation for exactly-one clauses. Returns (one, zero) or None on conflict."""
    changed = True
    while changed:
        changed = False
        for cm in clause_masks:
            ones = bin(cm & one).count("1")
            if ones > 1:
                return None
            if ones == 1:
                rest = cm & ~one
                if rest & one:
                    return None
                if (zero | rest) != zero:
                    zero |= rest
                    changed = True
                continue
            free = cm & ~zero
            nfree = bin(free).count("1")
            if nfree == 0:
                return None
            if nfree == 1:
                one |= free
                changed = True
        if one & zero:
            return None
    return one, zero


def count_solutions(n: int, clauses, cap: int = 2) -> int:
    """Number of bitstrings satisfying every clause, counted exactly up to `cap`."""
    masks = [(1 << a) | (1 << b) | (1 << c) for (a, b, c) in clauses]
    covered = 0
    for cm in masks:
        covered |= cm
    free_bits = n - bin(covered & ((1 << n) - 1)).count("1")

    def rec(one, zero, need):
        r = _propagate(masks, one, zero)
        if r is None:
            return 0
        one, zero = r
        best = None
        best_free = 4
        for cm in masks:
            if cm & one:
                continue
            free = cm & ~zero
            nf = bin(free).count("1")
            if nf < best_free:
                best_free = nf
                best = free
        if best is None:
            return 1
        total = 0
        bits = [k for k in range(n) if (best >> k) & 1]
        for k in bits:
            total += rec(one | (1 << k), zero, need - total)
            if total >= need:
                return total
        return total

    base = rec(0, 0, cap)
    if base == 0:
        return 0
    if free_bits > 0:
        return min(cap, base * (1 << min(free_bits, 62)))
    return min(cap, base)


def _solution(n: int, clauses) -> int:
    masks = [(1 << a) | (1 << b) | (1 << c) for (a, b, c) in clauses]
    # follow the unique branch of the search
    def rec(one, zero):
        r = _propagate(masks, one, zero)
        if r is None:
            return None
        one, zero = r
        for cm in masks:
            if cm & one:
                continue
            free = cm & ~zero
            for k in range(n):
                if (free >> k) & 1:
                    got = rec(one | (1 << k), zero)
                    if got is not None:
                        return got
            return None
        return one

    return rec(0, 0)


def _draw_triple(rng: SplitMix64, n: int):
    while True:
        a, b, c = rng.below(n), rng.below(n), rng.below(n)
        if a != b and b != c and a != c:
            return tuple(sorted((a, b, c)))


def generate_ec3(n: int, seed: int, max_restarts: int = 1000) -> EC3Instance:
    """Seeded EC3 instance with a unique satisfying assignment."""
    if n < 4 or n > 40:
        raise ValueError("n must be in [4, 40] (three bits admit one clause and three solutions)")
    rng = SplitMix64(seed)
    pool = comb(n, 3)
    for restart in range(max_restarts):
        used = set()
        clauses = []
        while len(used) < pool:
            t = _draw_triple(rng, n)
            if t in used:
                continue
            used.add(t)
            cnt = count_solutions(n, clauses + [t], cap=2)
            if cnt == 0:
                continue  # the paper's discard rule
            clauses.append(t)
            if cnt == 1:
                w = _solution(n, clauses)
                return EC3Instance(n=n, clauses=tuple(clauses), solution=w, seed=seed, restarts=restart)
        # pool exhausted without a unique solution: restart (Sec. I.D)
    raise RuntimeError("no unique-solution instance found")


def xx_pairs(n: int, seed: int, count: int | None = None):
    """`count` (default 2n) distinct unordered qubit pairs i<j drawn uniformly without
    replacement, each with a coupling J ~ U[-1, 1].  Returns a list of (i, j, J)."""
    if count is None:
        count = 2 * n
    total = n * (n - 1) // 2
    if count > total:
        raise ValueError("more pairs requested than exist")
    rng = SplitMix64(seed ^ 0x5EEDC0DE5EEDC0DE)
    chosen = []
    seen = set()
    while len(chosen) < count:
        i, j = rng.below(n), rng.below(n)
        if i == j:
            continue
        key = (min(i, j), max(i, j))
        if key in seen:
            continue
        seen.add(key)
        chosen.append(key)
    return [(i, j, 2.0 * rng.uniform() - 1.0) for (i, j) in chosen]


def _pairs(c):
    a, b, d = c
    return ((a, b), (a, d), (b, d))


def generate_ec3_hard(n: int, seed: int, m_max: int | None = None, max_restarts: int = 10000) -> EC3Instance:
    """Seeded hard EC3 instance by the recipe of Sec. I.E (Fig. hardEC3): start from one random
    clause of the full pool; keep drawing at random among the remaining clauses that touch the
    graph built so far and share no bit pair with it (n_ij in {0, 1}); once every bit is in the
    graph, count solutions after each draw and discard a clause that leaves none; stop at a
    unique solution; restart when the pool runs dry or m_max clauses are reached.
    m_max defaults to ceil(2n/3) + 2 (near the phase transition m ~ 2n/3 the paper aims at)."""
    if n < 4 or n > 40:
        raise ValueError("n must be in [4, 40]")
    if m_max is None:
        m_max = -(-2 * n // 3) + 2
    rng = SplitMix64(seed ^ 0x4A5D0C1A55E5)
    triples = [(a, b, c) for a in range(n) for b in range(a + 1, n) for c in range(b + 1, n)]
    for restart in range(max_restarts):
        pool = set(triples)
        first = triples[rng.below(len(triples))]
        pool.discard(first)
        clauses = [first]
        bits = set(first)
        used_pairs = set(_pairs(first))
        while True:
            # clauses that touch the graph and share no edge with it
            cand = sorted(c for c in pool if (set(c) & bits) and not (set(_pairs(c)) & used_pairs))
            if not cand or len(clauses) >= m_max:
                break  # restart
            c = cand[rng.below(len(cand))]
            pool.discard(c)
            if len(bits) == n:
                cnt = count_solutions(n, clauses + [c], cap=2)
                if cnt == 0:
                    continue  # discard
                clauses.append(c)
                used_pairs.update(_pairs(c))
                if cnt == 1:
                    w = _solution(n, clauses)
                    return EC3Instance(n=n, clauses=tuple(clauses), solution=w, seed=seed, restarts=restart)
            else:
                clauses.append(c)
                bits.update(c)
                used_pairs.update(_pairs(c))
                if len(bits) == n:
                    cnt = count_solutions(n, clauses, cap=2)
                    if cnt == 1:
                        w = _solution(n, clauses)
                        return EC3Instance(n=n, clauses=tuple(clauses), solution=w, seed=seed, restarts=restart)
                    if cnt == 0:
                        break  # unsatisfiable before any check could discard: restart
    raise RuntimeError("no hard instance found within the restart limit")
