"""Serving (ttc_server_*): continuous batching of solve requests.  A request
served together with others, admitted and retired at different ticks, must
end exactly where ttc_solve takes it alone (bitwise cores, same iteration
count and status).  GPU only."""
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


# (shape, options): orders 2-6, rank buckets 4/8/16, every stop rule and precision
SPECS = [
    (dict(n=[10, 10, 10, 10], r=[1, 2, 2, 2, 1], count=3000),
     dict(precision=ttc.PREC_FP64, stop_rule=ttc.STOP_RESID, tol=1e-11, max_iter=60)),
    (dict(n=[30, 20, 25], r=[1, 4, 3, 1], count=3000),
     dict(precision=ttc.PREC_MIXED, stop_rule=ttc.STOP_RESID, tol=1e-11, max_iter=60, polish_below=1e-5)),
    (dict(n=[60, 8], r=[1, 2, 1], count=400),
     dict(precision=ttc.PREC_FP32, stop_rule=ttc.STOP_NONE, max_iter=7)),
    (dict(n=[6, 300, 5], r=[1, 3, 3, 1], count=8000),
     dict(precision=ttc.PREC_MIXED, stop_rule=ttc.STOP_RELERR, tol=1e-9, max_iter=60, check_every=3,
          polish_below=1e-5)),
    (dict(n=[4, 4, 4, 4, 4, 4], r=[1, 4, 6, 8, 6, 4, 1], count=2500),
     dict(precision=ttc.PREC_FP64, stop_rule=ttc.STOP_STEP, tol=1e-10, max_iter=25, check_every=2)),
    (dict(n=[30, 28, 26], r=[1, 9, 10, 1], count=15000),
     dict(precision=ttc.PREC_FP32, stop_rule=ttc.STOP_RESID, tol=1e-4, max_iter=30)),
]


def problem(i):
    spec, _ = SPECS[i]
    return w.random_problem(300 + i, spec["n"], spec["r"], spec["count"], init_rel=0.05)


def solve_alone(i):
    P = problem(i)
    with ttc.Context(P.n, P.r, options=ttc.default_options(**SPECS[i][1])) as c:
        c.set_observations(P.idx, P.y)
        c.set_cores(P.init)
        if P.truth is not None:
            c.set_truth(P.truth)
        info = c.solve()
        return info, c.get_cores()


def submit(srv, i):
    P = problem(i)
    return srv.submit(P.n, P.r, P.idx, P.y, P.init, truth=P.truth, options=ttc.default_options(**SPECS[i][1]))


@pytest.fixture(scope="module")
def alone():
    return [solve_alone(i) for i in range(len(SPECS))]


def check_same(res, ref):
    info, cores = ref
    assert res["status"] == info["status"]
    assert res["iters"] == info["iters"]
    assert res["converged"] == info["converged"]
    for a, b in zip(res["cores"], cores):
        assert np.array_equal(a, b)


def test_serving_matches_solve_alone(alone):
    with ttc.Server(max_slots=16) as srv:
        tickets = [submit(srv, i) for i in range(len(SPECS))]
        results = [srv.poll(t) for t in tickets]
        st = srv.stats()
    for res, ref in zip(results, alone):
        check_same(res, ref)
        assert res["latency_ms"] >= res["queue_ms"] >= 0.0
    assert st["completed"] == len(SPECS) and st["failed"] == 0 and st["queued"] == 0
    assert st["iterations"] == sum(r["iters"] for r in results)
    assert st["launches"] > 0
    assert 0.0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]


def test_serving_admits_as_slots_free(alone):
    # two slots for six requests: later requests wait in the queue and join
    # the running batch as earlier ones retire
    order = [5, 0, 3, 2, 4, 1, 2, 0]
    with ttc.Server(max_slots=2) as srv:
        tickets = [submit(srv, i) for i in order[:4]]
        first = srv.poll(tickets[0])
        tickets += [submit(srv, i) for i in order[4:]]
        results = [first] + [srv.poll(t) for t in tickets[1:]]
        st = srv.stats()
    for i, res in zip(order, results):
        check_same(res, alone[i])
    assert max(r["queue_ms"] for r in results) > 0.0
    assert st["completed"] == len(order)


def test_serving_request_errors():
    with ttc.Server(max_slots=4) as srv:
        P = problem(1)
        # a repeated index is found at admission and ends only that request
        idx = P.idx.copy()
        idx[5] = idx[9]
        bad = srv.submit(P.n, P.r, idx, P.y, P.init)
        good = submit(srv, 2)
        assert srv.poll(bad)["status"] == "TTC_EDUP"
        assert srv.poll(good)["status"] == "TTC_OK"
        # shape errors are rejected at submission: by the library (r_0 != 1)
        init = [np.zeros((2, P.n[0], P.r[1]))] + list(P.init[1:])
        with pytest.raises(ttc.TTCError) as e:
            srv.submit(P.n, [2] + P.r[1:], P.idx, P.y, init)
        assert e.value.status == -1
        # and by the binding (cores that do not match the ranks)
        with pytest.raises(ValueError):
            srv.submit(P.n, [1, 2] + P.r[2:], P.idx, P.y, P.init)
        with pytest.raises(ttc.TTCError):
            srv.poll(123456789)
        st = srv.stats()
        assert st["failed"] == 1 and st["completed"] == 1


def test_serving_budget_limits():
    # a request larger than the whole budget is refused up front
    with ttc.Server(budget_bytes=1 << 20, max_slots=4) as srv:
        with pytest.raises(ttc.TTCError) as e:
            submit(srv, 5)
        assert e.value.status == -2


def test_serving_poll_timeout_and_shutdown():
    srv = ttc.Server(max_slots=4)
    t = submit(srv, 4)
    r = srv.poll(t, timeout_s=0.0)
    assert r is None or r["status"] == "TTC_OK"
    t2 = submit(srv, 1)
    srv.close()   # finishes queued and running requests before returning


def test_serving_mixed_stream_matches_solve_alone():
    # requests of the mixed stream (orders 3-12, modes 4-256, ranks 2-16):
    # different rank buckets and code widths share the engine
    reqs = [w.random_request(2000 + i, max_entries=20_000) for i in range(6)]
    opt = dict(precision=ttc.PREC_MIXED, stop_rule=ttc.STOP_RESID, tol=1e-8, max_iter=40,
               step_rule=ttc.STEP_STEEPEST)
    alone = []
    for Q in reqs:
        with ttc.Context(Q.n, Q.r, options=ttc.default_options(**opt)) as c:
            c.set_observations(Q.idx, Q.y)
            c.set_cores(Q.init)
            try:
                alone.append((c.solve(), c.get_cores()))
            except ttc.TTCError as e:          # a request may fail; the server must report the same
                alone.append(({"status": ttc.STATUS[e.status]}, None))
    with ttc.Server(max_slots=3) as srv:
        tickets = [srv.submit(Q.n, Q.r, Q.idx, Q.y, Q.init, options=ttc.default_options(**opt)) for Q in reqs]
        results = [srv.poll(t) for t in tickets]
    for res, ref in zip(results, alone):
        if ref[1] is None:
            assert res["status"] == ref[0]["status"]
        else:
            check_same(res, ref)
