"""Batched stepping (aqc_batch_*): many contexts per launch, K steps per CUDA-graph replay.

Checks: every member's final state equals the same context propagated alone through
aqc_propagate (tolerance of the precision) and the FP64 oracle; a member's result is bitwise
the same alone in a batch and in a mix; members can join while others are running.
"""
import numpy as np
import pytest

from instances import generate_ec3, xx_pairs
from oracle import oracle as O

from _helpers import C64, C128, TOL_STATE, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_3938_gb300 as P

    P.build()
    yield


SPECS = [  # (n, seed, T, nonlinear, s_kind)
    (6, 11, 1.0, True, 0),
    (9, 12, 2.0, False, 1),
    (12, 13, 1.5, True, 1),
    (14, 14, 0.8, True, 0),
    (16, 15, 0.4, False, 0),
    (10, 16, 3.0, True, 0),
    (13, 17, 1.0, False, 1),
    (8, 18, 0.7, True, 1),
    (5, 19, 0.5, False, 0),
]


def _member(spec, prec):
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context

    n, seed, T, nonlinear, s_kind = spec
    inst = generate_ec3(n, seed)
    pairs = xx_pairs(n, seed) if nonlinear else None
    ctx = Context(n, prec)
    HB.load_ec3(ctx, inst, pairs=pairs)
    ctx.set_schedule(T, HB.nonlinear_schedule() if nonlinear else HB.linear_schedule(), s_kind)
    ctx.set_integrator(0, 0.0)
    ctx.set_initial_state("uniform")
    H = O.ec3_hamiltonian(inst, pairs=pairs)
    sched = (O.nonlinear_path if nonlinear else O.linear_path)(T, s_kind)
    return inst, ctx, H, sched


@pytest.mark.parametrize("prec", [C128, C64])
def test_batch_members_match_single_and_oracle(prec):
    from paper_1311_3938_gb300.engine import Batch

    members = [_member(s, prec) for s in SPECS]
    with Batch(prec, max_members=16, steps_per_round=8) as b:
        slots = [b.add(m[1]) for m in members]
        b.run_to_completion(rounds_per_poll=4)
        steps, active, launches = b.poll()
        assert active == 0 and launches > 0
        for (inst, ctx, H, sched), slot in zip(members, slots):
            assert steps[slot] == O.step_count(H, sched)
            b.remove(slot)
    for spec, (inst, ctx, H, sched) in zip(SPECS, members):
        got = ctx.state()
        # the same context alone through aqc_propagate
        single = _member(spec, prec)[1]
        single.propagate(-1)
        ref_single = single.state()
        assert rel_err(got, ref_single) < (1e-12 if prec == C128 else 2e-6), spec
        if spec[0] <= 13:
            ref = O.propagate(H, sched, O.step_count(H, sched), O.uniform_state(spec[0]), nthreads=8)
            assert rel_err(got, ref.psi) < TOL_STATE[prec], spec
        assert abs(ctx.norm2() - single.norm2()) < (1e-12 if prec == C128 else 1e-6)
        single.close()
        ctx.close()


def test_alone_and_in_the_mix_are_identical():
    from paper_1311_3938_gb300.engine import Batch

    probe = SPECS[2]
    with Batch(C64, max_members=16, steps_per_round=8) as b:
        _, ctx, _, _ = _member(probe, C64)
        slot = b.add(ctx)
        b.run_to_completion()
        b.remove(slot)
        alone = ctx.state()
        ctx.close()
    with Batch(C64, max_members=16, steps_per_round=8) as b:
        mix = [_member(s, C64) for s in SPECS]
        slots = [b.add(m[1]) for m in mix]
        b.run_to_completion()
        for s in slots:
            b.remove(s)
        in_mix = mix[2][1].state()
        for m in mix:
            m[1].close()
    assert np.array_equal(alone, in_mix)


def test_members_join_while_others_run():
    from paper_1311_3938_gb300.engine import Batch

    with Batch(C64, max_members=8, steps_per_round=4) as b:
        first = [_member(s, C64) for s in SPECS[:3]]
        slots = {b.add(m[1]): m for m in first}
        b.run(3)
        late = [_member(s, C64) for s in SPECS[3:6]]
        for m in late:
            slots[b.add(m[1])] = m
        b.run_to_completion()
        for slot, m in list(slots.items()):
            b.remove(slot)
    for spec, m in zip(SPECS[:6], first + late):
        single = _member(spec, C64)[1]
        single.propagate(-1)
        assert rel_err(m[1].state(), single.state()) < 2e-6
        single.close()
        m[1].close()
