"""Batches: one graph launch steps many independent problems.  Each member
must compute exactly what it computes when stepped alone (bitwise), across
different orders, mode sizes, ranks (rank buckets) and precisions.  GPU only."""
import numpy as np
import pytest

from paper_2501_13385_gb300 import ttc
from paper_2501_13385_gb300 import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2501_13385_gb300 import build
    build.build()
    ttc.lib()


MEMBERS = [
    (dict(n=[10, 10, 10, 10], r=[1, 2, 2, 2, 1], count=3000), ttc.PREC_FP64),
    (dict(n=[30, 20, 25], r=[1, 4, 3, 1], count=3000), ttc.PREC_FP32),
    (dict(n=[60, 8], r=[1, 2, 1], count=400), ttc.PREC_FP32),
    (dict(n=[6, 300, 5], r=[1, 3, 3, 1], count=8000), ttc.PREC_FP32),   # a mode > 256
    (dict(n=[4, 4, 4, 4, 4, 4], r=[1, 4, 6, 8, 6, 4, 1], count=2500), ttc.PREC_FP64),
    (dict(n=[30, 28, 26], r=[1, 9, 10, 1], count=15000), ttc.PREC_FP32),  # rank bucket 16
]


def make(spec, prec, seed):
    P = w.random_problem(seed, spec["n"], spec["r"], spec["count"], init_rel=0.05)
    c = ttc.Context(P.n, P.r, precision=prec)
    c.set_observations(P.idx, P.y)
    c.set_cores(P.init)
    return P, c


def test_batch_members_bitwise_equal_to_alone():
    steps = 4
    alone = []
    for i, (spec, prec) in enumerate(MEMBERS):
        P, c = make(spec, prec, 100 + i)
        for _ in range(steps):
            c.step()
        alone.append(c.get_cores())
        c.close()
    ctxs = [make(spec, prec, 100 + i)[1] for i, (spec, prec) in enumerate(MEMBERS)]
    with ttc.Batch(ctxs) as b:
        for _ in range(steps):
            b.step()
        b.sync()
        assert b.launch_count() > 0
    for c, ref in zip(ctxs, alone):
        got = c.get_cores()
        for a, r in zip(got, ref):
            assert np.array_equal(a, r)
        c.close()


@pytest.mark.parametrize("lanes", [2, 3])
def test_batch_lanes_bitwise_equal_to_alone(lanes):
    # lanes: each group of members on its own graph and stream, running ahead
    # between joins; every member still computes what it computes alone
    steps = 4
    alone = []
    for i, (spec, prec) in enumerate(MEMBERS):
        P, c = make(spec, prec, 300 + i)
        for _ in range(steps):
            c.step()
        alone.append(c.get_cores())
        c.close()
    ctxs = [make(spec, prec, 300 + i)[1] for i, (spec, prec) in enumerate(MEMBERS)]
    with ttc.Batch(ctxs, lanes=lanes) as b:
        for s in range(steps):
            b.step()
            if s == 1:
                b.join()       # a join in the middle: the next step forks the lanes again
        b.profile_enable(True)
        b.profile_enable(False)
        b.sync()
        assert b.launch_count() > 0
        with pytest.raises(ttc.TTCError):
            lib_lanes = ttc.lib().ttc_batch_set_lanes(b._h, 2)   # after the first step
            ttc._check(lib_lanes, "ttc_batch_set_lanes")
    for c, ref in zip(ctxs, alone):
        got = c.get_cores()
        for a, r in zip(got, ref):
            assert np.array_equal(a, r)
        c.close()


def test_batch_profile_and_member_reuse():
    specs = [MEMBERS[1], MEMBERS[3]]
    ctxs = [make(spec, prec, 200 + i)[1] for i, (spec, prec) in enumerate(specs)]
    with ttc.Batch(ctxs) as b:
        b.profile_enable(True)
        for _ in range(3):
            b.step()
        ms, cnt = b.profile_read()
        assert cnt == 3 and ms > 0
    # members remain usable on their own after the batch is gone
    for c in ctxs:
        c.step()
        c.close()


def test_batch_rejects_bad_members():
    P, c = make(MEMBERS[1][0], ttc.PREC_FP32, 7)
    with pytest.raises(ttc.TTCError):
        ttc.Batch([c, c])
    empty = ttc.Context([5, 6, 7], [1, 2, 2, 1])
    with pytest.raises(ttc.TTCError):
        ttc.Batch([c, empty])
    empty.close()
    c.close()


def test_contexts_of_different_ranks_coexist():
    # a context needing less shared memory, created later, must not break
    # the launches of an earlier one that needs more
    P_big, big = make(MEMBERS[5][0], ttc.PREC_FP32, 400)
    P_small, small = make(MEMBERS[2][0], ttc.PREC_FP32, 401)
    ref = make(MEMBERS[5][0], ttc.PREC_FP32, 400)[1]
    for c in (big, small, ref):
        c.step()
    for a, b in zip(big.get_cores(), ref.get_cores()):
        assert np.array_equal(a, b)
    for c in (big, small, ref):
        c.close()


def test_chunked_dense_stages_bitwise_equal_to_alone():
    # 18 members of order 3 and 9 of order 4 on the warp-per-slice dense path:
    # order 3 runs its dense stages as two concurrent chunks of 9 members,
    # order 4 as one chunk; ranks, mode sizes and precisions differ inside
    # each chunk
    specs = []
    for i in range(18):
        specs.append((dict(n=[12 + i % 5, 9 + i % 3, 11], r=[1, 1 + i % 4, 2 + i % 3, 1], count=600 + 37 * i),
                      ttc.PREC_FP32 if i % 2 else ttc.PREC_FP64))
    for i in range(9):
        specs.append((dict(n=[7, 6 + i % 2, 8, 5], r=[1, 2, 1 + i % 3, 2, 1], count=900 + 11 * i), ttc.PREC_FP32))
    steps = 3
    alone = []
    for i, (spec, prec) in enumerate(specs):
        P, c = make(spec, prec, 500 + i)
        for _ in range(steps):
            c.step()
        alone.append(c.get_cores())
        c.close()
    ctxs = [make(spec, prec, 500 + i)[1] for i, (spec, prec) in enumerate(specs)]
    with ttc.Batch(ctxs) as b:
        for _ in range(steps):
            b.step()
        b.sync()
    for c, ref in zip(ctxs, alone):
        for a, r in zip(c.get_cores(), ref):
            assert np.array_equal(a, r)
        c.close()
