"""Parity of the step variants on the GPU with the oracle: the steepest step of
Eq. (PRGD stepsize), the uniform metric (RGD, Section 3.1) and Remark 3.6's
weighted retraction, alone and combined, in FP64 (iterates within 1e-10 of
the oracle's, step sizes within 1e-10); several steps; batches; a mixed
precision solve.  GPU only."""
import numpy as np
import pytest

import oracle as o
from paper_2501_13385_gb300 import ttc
from paper_2501_13385_gb300 import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2501_13385_gb300 import build
    build.build()
    ttc.lib()


VARIANTS = [
    dict(step_rule=ttc.STEP_STEEPEST),
    dict(metric=ttc.METRIC_UNIFORM),
    dict(metric=ttc.METRIC_UNIFORM, step_rule=ttc.STEP_STEEPEST),
    dict(retraction=ttc.RETRACT_WEIGHTED),
    dict(step_rule=ttc.STEP_STEEPEST, retraction=ttc.RETRACT_WEIGHTED),
]

SHAPES = [
    ([10, 10, 10, 10], [1, 2, 2, 2, 1], 3000),
    ([7, 13, 5], [1, 3, 4, 1], 300),
    ([6, 300, 5], [1, 5, 5, 1], 4000),
    ([4, 4, 4, 4, 4, 4], [1, 4, 6, 8, 6, 4, 1], 2500),
    ([30, 28, 26], [1, 9, 10, 1], 15000),     # rank bucket 16: block-per-slice dense kernels
]


def oracle_kw(v):
    return dict(step="adaptive" if v.get("step_rule") == ttc.STEP_STEEPEST else "constant",
                metric="uniform" if v.get("metric") == ttc.METRIC_UNIFORM else "precond",
                retraction="weighted" if v.get("retraction") == ttc.RETRACT_WEIGHTED else "plain")


def ctx_for(P, **kw):
    c = ttc.Context(P.n, P.r, **kw)
    c.set_observations(P.idx, P.y)
    c.set_cores(P.init)
    return c


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s[0])))
@pytest.mark.parametrize("variant", VARIANTS, ids=lambda v: "-".join(f"{k}{x}" for k, x in v.items()))
def test_one_fp64_step_matches_oracle(shape, variant):
    n, r, cnt = shape
    P = w.random_problem(31, n, r, cnt, init_rel=0.2)
    with ctx_for(P, precision=ttc.PREC_FP64, **variant) as c:
        info = c.step()
        got = c.get_cores()
    ref, oi = o.prgd_step(P.init, P.idx, P.y, P.n, P.r, eps_rel=1.0, alpha_scale=1.5, **oracle_kw(variant))
    assert info["eps"] == pytest.approx(oi.eps, rel=1e-12)
    assert info["alpha"] == pytest.approx(oi.alpha, rel=1e-10)
    assert o.tt_dist(got, ref) <= 1e-10 * o.tt_norm(ref)


@pytest.mark.parametrize("variant", VARIANTS, ids=lambda v: "-".join(f"{k}{x}" for k, x in v.items()))
def test_four_fp64_steps_track_oracle(variant):
    P = w.planted_small(3)
    cur = P.init
    with ctx_for(P, precision=ttc.PREC_FP64, **variant) as c:
        for _ in range(4):
            info = c.step()
            cur, oi = o.prgd_step(cur, P.idx, P.y, P.n, P.r, eps_rel=1.0, alpha_scale=1.5, **oracle_kw(variant))
            assert info["alpha"] == pytest.approx(oi.alpha, rel=1e-9)
            assert o.tt_dist(c.get_cores(), cur) <= 1e-9 * o.tt_norm(cur)


def test_explicit_step_size_overrides_the_steepest_step():
    P = w.planted_small(4)
    with ctx_for(P, precision=ttc.PREC_FP64, step_rule=ttc.STEP_STEEPEST) as c:
        info = c.step(alpha=0.21)
        assert info["alpha"] == 0.21
        ref, _ = o.prgd_step(P.init, P.idx, P.y, P.n, P.r, alpha=0.21, eps_rel=1.0)
        assert o.tt_dist(c.get_cores(), ref) <= 1e-10 * o.tt_norm(ref)


def test_variants_in_a_batch_are_bitwise_alone():
    specs = [(dict(n=[7, 13, 5], r=[1, 3, 4, 1], count=300), VARIANTS[0]),
             (dict(n=[10, 10, 10, 10], r=[1, 2, 2, 2, 1], count=3000), VARIANTS[2]),
             (dict(n=[6, 300, 5], r=[1, 5, 5, 1], count=4000), VARIANTS[4])]
    alone = []
    for i, (sp, v) in enumerate(specs):
        P = w.random_problem(40 + i, sp["n"], sp["r"], sp["count"], init_rel=0.05)
        with ctx_for(P, precision=ttc.PREC_FP32, **v) as c:
            for _ in range(3):
                c.step()
            alone.append(c.get_cores())
    ctxs = []
    for i, (sp, v) in enumerate(specs):
        P = w.random_problem(40 + i, sp["n"], sp["r"], sp["count"], init_rel=0.05)
        ctxs.append(ctx_for(P, precision=ttc.PREC_FP32, **v))
    with ttc.Batch(ctxs) as b:
        for _ in range(3):
            b.step()
        b.sync()
    for c, ref in zip(ctxs, alone):
        for a, r in zip(c.get_cores(), ref):
            assert np.array_equal(a, r)
        c.close()


def test_steepest_mixed_solve_recovers_orthogonal_cubic():
    P = w.orthogonal_cubic(5)
    with ctx_for(P, precision=ttc.PREC_MIXED, step_rule=ttc.STEP_STEEPEST, stop_rule=ttc.STOP_RELERR,
                 tol=1e-6, max_iter=200) as c:
        c.set_truth(P.truth)
        res = c.solve()
        assert res["converged"]
        assert c.relerr() <= 1e-6


def test_qst_workload_fp64_steps_match_oracle():
    # order 10, mode 4, TT-ranks 4 (the tomography experiment's shape, Section 5)
    P = w.qst_like(1, init_rel=0.1)
    cur = P.init
    with ctx_for(P, precision=ttc.PREC_FP64) as c:
        for _ in range(2):
            c.step()
            cur, _ = o.prgd_step(cur, P.idx, P.y, P.n, P.r, eps_rel=1.0, alpha_scale=1.5)
            assert o.tt_dist(c.get_cores(), cur) <= 1e-9 * o.tt_norm(cur)


def test_qst_workload_mixed_solve_converges():
    P = w.qst_like(2)
    with ctx_for(P, precision=ttc.PREC_MIXED, stop_rule=ttc.STOP_RELERR, tol=1e-6, max_iter=400) as c:
        c.set_truth(P.truth)
        res = c.solve()
        assert res["converged"], res


def _oracle_with_fallback(P, alpha_scale, iters):
    """The oracle's iterates under the divergence fallback: constant steps of
    Theorem 4.1's form until the relative residual more than doubles from one
    iteration to the next, the steepest step of Eq. (PRGD stepsize) from the
    following iteration on.  Returns (cores, the first steepest iteration or
    -1)."""
    yn = np.linalg.norm(P.y)
    cur, prev, steep, fb = P.init, -1.0, False, -1
    for it in range(1, iters + 1):
        rel = float(np.linalg.norm(o.residual(cur, P.idx, P.y))) / yn
        cur, _ = o.prgd_step(cur, P.idx, P.y, P.n, P.r, eps_rel=1.0, alpha_scale=alpha_scale,
                             step="adaptive" if steep else "constant")
        if not steep and prev > 0 and rel > 2 * prev:
            steep, fb = True, it + 1
        prev = rel
    return cur, fb


def test_diverging_constant_step_falls_back_to_the_steepest_step():
    # alpha_scale 5 on this planted problem: the relative residual goes
    # 0.58, 0.84, 2.2 (more than doubling at iteration 3), so iterations from
    # 4 on take the steepest step, which recovers the tensor
    P = w.planted_small(6)
    ref, fb = _oracle_with_fallback(P, 5.0, 12)
    assert fb == 4
    with ctx_for(P, precision=ttc.PREC_FP64, alpha_scale=5.0, stop_rule=ttc.STOP_NONE, max_iter=12) as c:
        res = c.solve()
        assert res["fallback_iter"] == fb
        assert o.tt_dist(c.get_cores(), ref) <= 1e-9 * o.tt_norm(ref)
    with ctx_for(P, precision=ttc.PREC_FP64, alpha_scale=5.0, stop_rule=ttc.STOP_RELERR, tol=1e-9,
                 max_iter=200) as c:
        c.set_truth(P.truth)
        res = c.solve()
        assert res["converged"] and res["fallback_iter"] == fb
        assert c.relerr() <= 1e-9
        # a second solve starts again from the configured constant step
        c.set_cores(P.init)
        again = c.solve()
        assert again["fallback_iter"] == fb and again["iters"] == res["iters"]
    # with the fallback off the same iteration keeps diverging
    with ctx_for(P, precision=ttc.PREC_FP64, alpha_scale=5.0, step_fallback=0, stop_rule=ttc.STOP_NONE,
                 max_iter=6) as c:
        res = c.solve()
        assert res["fallback_iter"] == -1
        assert o.tt_dist(c.get_cores(), P.truth) > o.tt_norm(P.truth)


def test_fallback_in_the_server_matches_solve_alone():
    P = w.planted_small(6)
    opts = dict(precision=ttc.PREC_FP64, alpha_scale=5.0, stop_rule=ttc.STOP_RELERR, tol=1e-9, max_iter=200)
    with ctx_for(P, **opts) as c:
        c.set_truth(P.truth)
        alone = c.solve()
        cores = c.get_cores()
    Q = w.planted_small(7)
    with ttc.Server(max_slots=4) as srv:
        t0 = srv.submit(Q.n, Q.r, Q.idx, Q.y, Q.init, truth=Q.truth,
                        options=ttc.default_options(precision=ttc.PREC_FP64, stop_rule=ttc.STOP_RELERR, tol=1e-9))
        t1 = srv.submit(P.n, P.r, P.idx, P.y, P.init, truth=P.truth, options=ttc.default_options(**opts))
        other, res = srv.poll(t0), srv.poll(t1)
    assert other["converged"]
    assert res["converged"] and res["iters"] == alone["iters"]
    for a, b in zip(res["cores"], cores):
        assert np.array_equal(a, b)
