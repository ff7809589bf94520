"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle on the
same seeded inputs: layout bit-exact, sampled values, residual, slice
energies, tangent scatter, one and several PRGD steps, solves.  GPU only.

Tolerances:
  * FP64 pass: 1e-12 relative (both sides FP64; only the summation order differs).
  * FP32 pass: sampled entries within 1e-5 of max(|v64|, rms(v64)) (the stated
    FP32 bound); reductions within 1e-5 of the sum of absolute terms.
  * full FP64 steps: 1e-10 relative Frobenius distance of the iterates (the
    retraction is a truncated SVD; the two sides take it by different but
    exact-in-exact-arithmetic routes).
"""
import math

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


SHAPES = [
    # (n, r, count): several chunks per slice, ragged tails, small and odd modes
    ([10, 10, 10, 10], [1, 2, 2, 2, 1], 3000),
    ([7, 13, 5], [1, 3, 4, 1], 300),
    ([40, 3], [1, 3, 1], 100),
    ([6, 300, 5], [1, 5, 5, 1], 4000),        # a mode > 256 needs two radix digits
    ([4, 4, 4, 4, 4, 4], [1, 4, 6, 8, 6, 4, 1], 2500),
    ([9, 8, 7], [1, 1, 2, 1], 200),           # rank-1 bond
    ([30, 28, 26], [1, 9, 10, 1], 15000),     # rank bucket 16 (shared-memory outer products)
    ([40, 40, 40], [1, 20, 20, 1], 48000),    # rank bucket 32
]


def ctx_for(P, **kw):
    c = ttc.Context(P.n, P.r, **kw)
    c.set_observations(P.idx, P.y)
    c.set_cores(P.init)
    return c


def scatter_definition(cores, idx, g, k, d, mag=None):
    """E_k(x) = sum over entries with x_k = x of g * l^T r^T (plain definition),
    and the error scale sum of mag * |l^T r^T| (mag = |g| by default).  For an
    FP32 pass the residual g = v - y carries an error relative to |v| + |y|,
    so its bound uses mag = |v| + |y|."""
    left, right = o.interface_rows(cores, idx, k)
    E = np.zeros((d, left.shape[1] * right.shape[1]))
    A = np.zeros_like(E)
    outer = left[:, :, None] * right[:, None, :]
    np.add.at(E, idx[:, k], (g[:, None, None] * outer).reshape(len(g), -1))
    mag = np.abs(g) if mag is None else mag
    np.add.at(A, idx[:, k], (mag[:, None, None] * np.abs(outer)).reshape(len(g), -1))
    return E.reshape(d, left.shape[1], right.shape[1]), A.reshape(d, left.shape[1], right.shape[1])


@pytest.mark.parametrize("shape", SHAPES)
def test_layout_bit_exact(shape):
    n, r, cnt = shape
    P = w.random_problem(11, n, r, cnt)
    with ctx_for(P) as c:
        prev = np.arange(cnt)
        for k in range(P.m):
            perm, seg = c.layout(k)
            # mode k's order: the stable sort by x_k of mode k-1's order, so
            # lexicographic in (x_k, ..., x_0, input position)
            ref_perm = prev[np.argsort(P.idx[prev, k], kind="stable")]
            assert np.array_equal(perm, ref_perm)
            assert np.array_equal(perm, np.lexsort([np.arange(cnt)] + [P.idx[:, j] for j in range(k + 1)]))
            prev = ref_perm
            ref = np.concatenate([[0], np.cumsum(np.bincount(P.idx[:, k], minlength=n[k]))])
            assert np.array_equal(seg, ref)


def test_invalid_inputs_are_rejected():
    P = w.random_problem(3, [5, 6, 7], [1, 2, 2, 1], 50)
    with ttc.Context(P.n, P.r) as c:
        bad = P.idx.copy()
        bad[17, 1] = 6
        with pytest.raises(ttc.TTCError) as e:
            c.set_observations(bad, P.y)
        assert e.value.status == -3
        bad = P.idx.copy()
        bad[3, 0] = -1
        with pytest.raises(ttc.TTCError) as e:
            c.set_observations(bad, P.y)
        assert e.value.status == -3
        dup = P.idx.copy()
        dup[40] = dup[2]
        with pytest.raises(ttc.TTCError) as e:
            c.set_observations(dup, P.y)
        assert e.value.status == -4
        y = P.y.copy()
        y[5] = np.nan
        with pytest.raises(ttc.TTCError) as e:
            c.set_observations(P.idx, y)
        assert e.value.status == -5
        with pytest.raises(ttc.TTCError) as e:
            c.step()            # no cores, no observations yet
        assert e.value.status == -1
        c.set_observations(P.idx, P.y)   # a valid call still works afterwards
        c.set_cores(P.init)
        c.step()
    with pytest.raises(ttc.TTCError):
        ttc.Context([5, 6], [1, 40, 1])
    with pytest.raises(ttc.TTCError):
        ttc.Context([5, 6], [2, 2, 1])


@pytest.mark.parametrize("shape", SHAPES)
def test_eval_fp64_and_fp32(shape):
    n, r, cnt = shape
    P = w.random_problem(5, n, r, cnt)
    with ctx_for(P) as c:
        v64 = c.eval(P.idx, ttc.PREC_FP64)
        ref = o.tt_eval(P.init, P.idx)
        assert np.max(np.abs(v64 - ref)) <= 1e-12 * max(np.max(np.abs(ref)), 1e-300)
        v32 = c.eval(P.idx, ttc.PREC_FP32)
        floor = np.maximum(np.abs(ref), np.sqrt(np.mean(ref ** 2)))
        assert np.max(np.abs(v32 - ref) / floor) <= 1e-5


@pytest.mark.parametrize("prec", [ttc.PREC_FP64, ttc.PREC_FP32])
@pytest.mark.parametrize("shape", SHAPES)
def test_pass_outputs_match_definitions(shape, prec):
    n, r, cnt = shape
    P = w.random_problem(7, n, r, cnt, init_rel=0.3)
    with ctx_for(P, precision=prec) as c:
        g_ref = o.residual(P.init, P.idx, P.y)
        g = c.residual()                 # evaluated at the cores just set
        scale = np.maximum(np.abs(o.tt_eval(P.init, P.idx)), np.sqrt(np.mean(P.y ** 2)))
        tol = 1e-12 if prec == ttc.PREC_FP64 else 1e-5
        assert np.max(np.abs(g - g_ref) / scale) <= tol
        c.step()
        v_ref = o.tt_eval(P.init, P.idx)
        mag = np.abs(g_ref) if prec == ttc.PREC_FP64 else np.abs(v_ref) + np.abs(P.y)
        for k in range(P.m):
            s = c.slice_energy(k)
            s_ref = o.slice_energy(g_ref, P.idx[:, k], n[k])
            s_err = o.slice_energy(np.sqrt(2 * np.abs(g_ref) * mag), P.idx[:, k], n[k])  # sum 2|g| mag
            assert np.all(np.abs(s - s_ref) <= tol * (s_err + s_ref) + 1e-300)
            E = c.scatter(k)
            E_ref, E_abs = scatter_definition(P.init, P.idx, g_ref, k, n[k], mag)
            assert np.all(np.abs(E - E_ref) <= tol * (E_abs + 1e-300) + 1e-300)


@pytest.mark.parametrize("shape", SHAPES)
def test_one_fp64_step_matches_oracle(shape):
    n, r, cnt = shape
    P = w.random_problem(9, n, r, cnt, init_rel=0.2)
    with ctx_for(P, precision=ttc.PREC_FP64) as c:
        info = c.step()
        got = c.get_cores()
    ref, oi = o.prgd_step(P.init, P.idx, P.y, P.n, P.r, eps_rel=1.0, alpha_scale=1.5)
    assert info["eps"] == pytest.approx(oi.eps, rel=1e-12)
    assert info["alpha"] == pytest.approx(oi.alpha, rel=1e-12)
    assert o.tt_dist(got, ref) <= 1e-10 * o.tt_norm(ref)
    # the retraction's output is left-orthogonal
    for k in range(P.m - 1):
        L = got[k].reshape(-1, got[k].shape[2])
        assert np.allclose(L.T @ L, np.eye(L.shape[1]), atol=1e-11)


def test_explicit_step_size_and_frozen_eps():
    P = w.planted_small(1)
    with ctx_for(P, precision=ttc.PREC_FP64, eps_frozen=1) as c:
        i1 = c.step(alpha=0.37)
        assert i1["alpha"] == 0.37
        ref1, oi1 = o.prgd_step(P.init, P.idx, P.y, P.n, P.r, alpha=0.37, eps_rel=1.0)
        assert o.tt_dist(c.get_cores(), ref1) <= 1e-10 * o.tt_norm(ref1)
        i2 = c.step()
        assert i2["eps"] == pytest.approx(oi1.eps, rel=1e-12)      # frozen at iteration 0
        ref2, _ = o.prgd_step(ref1, P.idx, P.y, P.n, P.r, eps=oi1.eps, alpha_scale=1.5)
        assert o.tt_dist(c.get_cores(), ref2) <= 1e-10 * o.tt_norm(ref2)


def test_five_fp64_steps_track_oracle():
    P = w.planted_small(2)
    cur = P.init
    with ctx_for(P, precision=ttc.PREC_FP64) as c:
        for _ in range(5):
            c.step()
            cur, _ = o.prgd_step(cur, P.idx, P.y, P.n, P.r, eps_rel=1.0, alpha_scale=1.5)
            assert o.tt_dist(c.get_cores(), cur) <= 1e-9 * o.tt_norm(cur)


def test_planted_recovery_fp64_to_1e_10():
    P = w.planted_small(0)
    with ctx_for(P, precision=ttc.PREC_FP64, stop_rule=ttc.STOP_RELERR, tol=1e-10, max_iter=300) as c:
        c.set_truth(P.truth)
        res = c.solve()
        got = c.get_cores()
        assert res["converged"], res
        assert c.relerr() <= 1e-10
    assert o.tt_dist(got, P.truth) <= 1e-10 * o.tt_norm(P.truth)


def test_orthogonal_cubic_full_size_fp64_step():
    P = w.orthogonal_cubic(0)
    with ctx_for(P, precision=ttc.PREC_FP64) as c:
        c.step()
        got = c.get_cores()
    ref, _ = o.prgd_step(P.init, P.idx, P.y, P.n, P.r, eps_rel=1.0, alpha_scale=1.5)
    assert o.tt_dist(got, ref) <= 1e-10 * o.tt_norm(ref)


def test_orthogonal_cubic_mixed_solve_matches_oracle_solution():
    P = w.orthogonal_cubic(1)
    with ctx_for(P, precision=ttc.PREC_MIXED, stop_rule=ttc.STOP_RELERR, tol=1e-6, max_iter=100) as c:
        c.set_truth(P.truth)
        res = c.solve()
        got = c.get_cores()
    assert res["converged"], res
    ref = o.solve(P.init, P.idx, P.y, P.n, P.r, truth=P.truth, eps_rel=1.0, alpha_scale=1.5,
                  max_iter=100, tol=1e-12).cores
    assert o.tt_dist(got, P.truth) <= 1e-6 * o.tt_norm(P.truth)
    assert o.tt_dist(got, ref) <= 1e-6 * o.tt_norm(ref)


def test_bitwise_reproducible_and_graph_equals_eager():
    P = w.random_problem(21, [30, 20, 25], [1, 4, 3, 1], 3000, init_rel=0.3)
    outs = []
    for graph in (1, 1, 0):
        with ctx_for(P, precision=ttc.PREC_MIXED, use_graph=graph) as c:
            for _ in range(3):
                c.step()
            outs.append(c.get_cores())
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)
    for a, b in zip(outs[0], outs[2]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("maker", ["hyperspectral_like", "tomography_like"])
def test_full_size_sampled_slices(maker):
    """Full-size configurations: the scatter and slice energies of sampled
    slices, each recomputed by the oracle from that slice's entries only."""
    P = getattr(w, maker)(0)
    rng = np.random.default_rng(0)
    for prec, tol in ((ttc.PREC_FP64, 1e-12), (ttc.PREC_FP32, 1e-5)):
        with ctx_for(P, precision=prec) as c:
            c.step()
            for k in range(P.m):
                for x in rng.choice(P.n[k], size=min(3, P.n[k]), replace=False):
                    sel = np.nonzero(P.idx[:, k] == x)[0]
                    g = o.residual(P.init, P.idx[sel], P.y[sel])
                    v = o.tt_eval(P.init, P.idx[sel])
                    mag = np.abs(g) if prec == ttc.PREC_FP64 else np.abs(v) + np.abs(P.y[sel])
                    E_ref, E_abs = scatter_definition(P.init, P.idx[sel], g, k, P.n[k], mag)
                    E = c.scatter(k)[x]
                    assert np.all(np.abs(E - E_ref[x]) <= tol * (E_abs[x] + 1e-300) + 1e-300)
                    s = c.slice_energy(k)[x]
                    assert abs(s - (g @ g)) <= tol * ((g @ g) + 2 * np.abs(g) @ mag)


def test_diverging_solve_never_reports_convergence():
    # an absurd step scale, with the divergence fallback off, makes the
    # iteration diverge: the solver must end with TTC_ENOTCONV or
    # TTC_ENONFINITE (a non-finite metric is never read as converged),
    # whichever comes first
    P = w.planted_small(6)
    for rule in (ttc.STOP_RELERR, ttc.STOP_STEP):
        with ctx_for(P, precision=ttc.PREC_FP64, alpha_scale=1e4, step_fallback=0, stop_rule=rule, tol=1e-6,
                     max_iter=200) as c:
            c.set_truth(P.truth)
            try:
                res = c.solve()
            except ttc.TTCError as e:
                assert e.status == -5
            else:
                assert not res["converged"] and res["status"] == "TTC_ENOTCONV"


@pytest.mark.parametrize("e2", [-80, 72])
def test_extreme_value_scales_fp64(e2):
    # data scaled by 2^e2 (Grams far outside FP32's range): the FP32
    # factorizations inside the dense stage scale exactly by powers of two, so
    # the FP64 step still matches the oracle on the same scaled data
    P = w.planted_small(2)
    s = 2.0 ** e2
    y = P.y * s
    init = [c * 2.0 ** (e2 // 4) for c in P.init]
    with ttc.Context(P.n, P.r, precision=ttc.PREC_FP64) as c:
        c.set_observations(P.idx, y)
        c.set_cores(init)
        c.step()
        got = c.get_cores()
    ref, _ = o.prgd_step(init, P.idx, y, P.n, P.r, eps_rel=1.0, alpha_scale=1.5)
    assert o.tt_dist(got, ref) <= 1e-10 * o.tt_norm(ref)
