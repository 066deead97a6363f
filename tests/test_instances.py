"""Seeded input generators: determinism, uniqueness of EC3 solutions (brute force), pairs."""
import numpy as np
import pytest

from instances import SplitMix64, count_solutions, generate_ec3, random_state, xx_pairs


def test_splitmix64_reference_values():
    """First outputs for seed 0 of the published SplitMix64 definition."""
    g = SplitMix64(0)
    assert [g.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


@pytest.mark.parametrize("n,seed", [(6, 1), (8, 2), (10, 1), (12, 7), (14, 3), (16, 9)])
def test_ec3_unique_solution_brute_force(n, seed):
    inst = generate_ec3(n, seed)
    assert len(set(inst.clauses)) == inst.m
    for c in inst.clauses:
        assert len(set(c)) == 3 and all(0 <= b < n for b in c)
    z = np.arange(1 << n)
    sat = np.ones(1 << n, bool)
    for (a, b, c) in inst.clauses:
        sat &= (((z >> a) & 1) + ((z >> b) & 1) + ((z >> c) & 1)) == 1
    assert list(np.nonzero(sat)[0]) == [inst.solution]


def test_ec3_deterministic():
    a = generate_ec3(20, 2)
    b = generate_ec3(20, 2)
    assert a == b


def test_count_solutions_cap_and_free_bits():
    # one clause on 4 bits: 3 choices x 2 for the free bit = 6
    assert count_solutions(4, [(0, 1, 2)], cap=100) == 6
    assert count_solutions(4, [(0, 1, 2)], cap=2) == 2
    # contradictory: (0,1,2) and (0,1,3),(2,3,?)...
    assert count_solutions(3, [(0, 1, 2)], cap=10) == 3


def test_xx_pairs_distinct_and_range():
    p = xx_pairs(10, 5)
    assert len(p) == 20
    keys = {(i, j) for (i, j, _) in p}
    assert len(keys) == 20 and all(i < j for (i, j) in keys)
    assert all(-1.0 <= J < 1.0 for (_, _, J) in p)
    assert p == xx_pairs(10, 5)


def test_random_state_normalised():
    v = random_state(8, 3)
    assert abs(np.vdot(v, v).real - 1) < 1e-14
    assert np.array_equal(v, random_state(8, 3))


@pytest.mark.parametrize("n", [8, 10, 12, 14])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_hard_instances_follow_the_recipe(n, seed):
    """Sec. I.E: unique solution (brute force), n_ij in {0, 1} (clauses share at most one bit),
    a connected clause graph over all n bits, at most m_max clauses; seeded and deterministic."""
    from instances.ec3 import generate_ec3_hard

    inst = generate_ec3_hard(n, seed)
    assert inst == generate_ec3_hard(n, seed)
    assert inst.m <= -(-2 * n // 3) + 2
    masks = [(1 << a) | (1 << b) | (1 << c) for (a, b, c) in inst.clauses]
    sols = [z for z in range(1 << n) if all(bin(z & m).count("1") == 1 for m in masks)]
    assert sols == [inst.solution]
    for i in range(len(masks)):
        for j in range(i + 1, len(masks)):
            assert bin(masks[i] & masks[j]).count("1") <= 1
    # connectivity over all bits
    reach, frontier = set(inst.clauses[0]), True
    while frontier:
        frontier = False
        for c in inst.clauses:
            if set(c) & reach and not set(c) <= reach:
                reach |= set(c)
                frontier = True
    assert reach == set(range(n))
