"""Edge cases of the CUDA path against the oracle: a single observation, the
largest order (16), a mode of size 1 (a zero-bit code field), the largest
rank (32), two-word packed codes, all ranks 1, and empty or oversized inputs
rejected.  FP64 steps within 1e-10 of the oracle.  GPU only."""
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


def fp64_step_matches(P, steps=1, tol=1e-10):
    cur = P.init
    with ttc.Context(P.n, P.r, precision=ttc.PREC_FP64) as c:
        c.set_observations(P.idx, P.y)
        c.set_cores(P.init)
        for _ in range(steps):
            info = c.step()
            cur, oi = o.prgd_step(cur, P.idx, P.y, P.n, P.r, eps_rel=1.0, alpha_scale=1.5)
            assert info["alpha"] == pytest.approx(oi.alpha, rel=1e-12)
            assert o.tt_dist(c.get_cores(), cur) <= tol * o.tt_norm(cur)
        # the sampled values agree too (FP64 evaluation at Omega)
        v = c.eval(P.idx, ttc.PREC_FP64)
        assert np.max(np.abs(v - o.tt_eval(cur, P.idx))) <= 1e-12 * max(1.0, np.max(np.abs(v)))


@pytest.mark.parametrize("case", [
    ("single_entry", dict(n=[3, 4, 5], r=[1, 1, 1, 1], count=1)),
    ("all_ranks_one", dict(n=[20, 30, 25], r=[1, 1, 1, 1], count=400)),
    ("order_16", dict(n=[2] * 16, r=[1, 2, 3] + [4] * 11 + [3, 2, 1], count=6000)),
    ("mode_of_size_one", dict(n=[9, 1, 8, 7], r=[1, 3, 3, 3, 1], count=300)),
    ("two_word_codes", dict(n=[5000, 4000, 3000], r=[1, 3, 3, 1], count=20000)),
    ("rank_32", dict(n=[64, 64, 64], r=[1, 32, 32, 1], count=100000)),
    ("order_2_matrix", dict(n=[120, 90], r=[1, 6, 1], count=4000)),
], ids=lambda c: c[0])
def test_edge_shapes_fp64_step(case):
    _, spec = case
    P = w.random_problem(77, spec["n"], spec["r"], spec["count"], init_rel=0.1)
    fp64_step_matches(P, steps=2 if spec["count"] > 1 else 1)


def test_empty_and_oversized_inputs_are_rejected():
    with ttc.Context([5, 6, 7], [1, 2, 2, 1]) as c:
        with pytest.raises(ttc.TTCError) as e:
            c.set_observations(np.zeros((0, 3), dtype=np.int32), np.zeros(0))
        assert e.value.status == -1
    with pytest.raises(ttc.TTCError) as e:                 # order above 16
        ttc.Context([2] * 17, [1] + [2] * 16 + [1])
    assert e.value.status == -10
    with pytest.raises(ttc.TTCError) as e:                 # rank above 32
        ttc.Context([64, 64, 64], [1, 33, 33, 1])
    assert e.value.status == -10
    with pytest.raises(ttc.TTCError) as e:                 # codes wider than 128 bits
        ttc.Context([1 << 17] * 7, [1] + [2] * 6 + [1]).set_observations(
            np.zeros((1, 7), dtype=np.int32), np.zeros(1))
    assert e.value.status in (-10, -1)


@pytest.mark.parametrize("spec", [
    dict(n=[30, 28, 26], r=[1, 9, 10, 1], count=15000),
    dict(n=[40, 40, 40], r=[1, 20, 20, 1], count=48000),
    dict(n=[12, 10, 11, 13], r=[1, 12, 17, 11, 1], count=9000),
    dict(n=[64, 64, 64], r=[1, 32, 32, 1], count=100000),
    dict(n=[200, 30, 20], r=[1, 9, 10, 1], count=20000),   # 128-row groups of the two-mode prefix table
], ids=lambda s: "r" + "-".join(map(str, s["r"][1:-1])) + "-n" + str(s["n"][0]))
@pytest.mark.parametrize("steepest", [False, True], ids=["constant", "steepest"])
def test_float_float_dense_stages_match_oracle(spec, steepest):
    # FP64 steps whose slice products (the Grams, the new cores and, with the
    # steepest step, the unit-step update cores B1 and ||Z||_W^2) run in
    # float-float, as every FP32 step's do: the products are accurate to
    # ~1e-11 relative to sum |a_i b_i| (compensated dot products of 48-bit
    # operands), so the step stays within 1e-8 of the oracle's (an FP32
    # product would miss by ~1e-6, a wrong index by O(1)); two steps, so
    # that the second starts from iterates the float-float path made
    P = w.random_problem(78, spec["n"], spec["r"], spec["count"], init_rel=0.1)
    cur = P.init
    rule = ttc.STEP_STEEPEST if steepest else ttc.STEP_CONSTANT
    with ttc.Context(P.n, P.r, precision=ttc.PREC_FP64, dense_mode=ttc.DENSE_FF, step_rule=rule) as c:
        c.set_observations(P.idx, P.y)
        c.set_cores(P.init)
        for _ in range(2):
            info = c.step()
            cur, oi = o.prgd_step(cur, P.idx, P.y, P.n, P.r, eps_rel=1.0, alpha_scale=1.5,
                                  step="adaptive" if steepest else "constant")
            assert info["alpha"] == pytest.approx(oi.alpha, rel=1e-8)
            assert o.tt_dist(c.get_cores(), cur) <= 1e-8 * o.tt_norm(cur)


def test_dense_mode_fp64_keeps_fp32_steps_in_fp64():
    # TTC_DENSE_FP64: an FP32 step's slice products in FP64; the step still
    # carries the FP32 pass's error, so it is compared within 2e-5 (as the
    # mixed steps of the full-size tests), and against the default
    # (float-float) FP32 step, which must agree to the same bound
    P = w.random_problem(79, [40, 40, 40], [1, 20, 20, 1], 48000, init_rel=0.1)
    ref, _ = o.prgd_step(P.init, P.idx, P.y, P.n, P.r, eps_rel=1.0, alpha_scale=1.5)
    got = {}
    for mode in (ttc.DENSE_FP64, ttc.DENSE_AUTO):
        with ttc.Context(P.n, P.r, precision=ttc.PREC_FP32, dense_mode=mode) as c:
            c.set_observations(P.idx, P.y)
            c.set_cores(P.init)
            c.step()
            got[mode] = c.get_cores()
        assert o.tt_dist(got[mode], ref) <= 2e-5 * o.tt_norm(ref)
    assert o.tt_dist(got[ttc.DENSE_FP64], got[ttc.DENSE_AUTO]) <= 2e-5 * o.tt_norm(ref)
    with pytest.raises(ttc.TTCError) as e:
        ttc.Context(P.n, P.r, dense_mode=3)
    assert e.value.status == -1
