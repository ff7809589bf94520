"""Pins for the oracle's step variants on tiny tensors, each against an
independent computation: the steepest step of Eq. (PRGD stepsize) against
the exact line search of the sampled objective and against dense weighted
norms; the uniform metric (RGD, Section 3.1) against the dense Jacobian
projector; Remark 3.6's weighted retraction against a dense TT-SVD of the
weighted tensor.  CPU only."""
import itertools

import numpy as np

import oracle as o

from test_oracle_prgd import dense_weight, grad_dense, jacobian, setup_case


def test_tangent_tt_is_the_sum_of_components():
    n, r, cores, idx, y = setup_case(21)
    grad, G, U, A, g = grad_dense(cores, idx, y, n, 0.7)
    Z = o.tangent_tt(U, A)
    assert [c.shape[0] for c in Z] == [1, 4, 4] and [c.shape[2] for c in Z] == [4, 4, 1]
    assert np.allclose(o.tt_full(Z), o.tangent_to_full(U, A), rtol=1e-12, atol=1e-13)


def test_adaptive_step_is_the_exact_line_search():
    # alpha = ||Z||_W^2 / ||P_Omega Z||^2 must minimise 1/2 ||P_Omega(T - alpha Z) - y||^2
    # = 1/2 ||g - alpha z||^2, i.e. equal <g, z> / <z, z> (Z in the tangent space)
    n, r, cores, idx, y = setup_case(22)
    m = len(n)
    eps = 0.3
    grad, G, U, A, g = grad_dense(cores, idx, y, n, eps)
    alpha = o.adaptive_step(U, A, G, idx)
    z = grad[tuple(idx.T)]
    assert alpha == np.float64(alpha) and alpha > 0
    assert abs(alpha - float(g @ z) / float(z @ z)) <= 1e-10 * alpha
    # dense: ||Z||_W^2 = sum W Z^2 with W = prod_k G_k^{1/(2m)}
    num = float(np.sum(dense_weight(n, G, 1.0 / (2 * m)) * grad * grad))
    assert abs(alpha - num / float(z @ z)) <= 1e-10 * alpha
    f = lambda a: 0.5 * float(np.sum((g - a * z) ** 2))
    assert f(alpha) < f(alpha * 1.01) and f(alpha) < f(alpha * 0.99)


def test_adaptive_step_through_prgd_step():
    n, r, cores, idx, y = setup_case(23)
    new, info = o.prgd_step(cores, idx, y, n, r, eps=0.4, step="adaptive")
    grad, G, U, A, g = grad_dense(cores, idx, y, n, 0.4)
    z = grad[tuple(idx.T)]
    assert abs(info.alpha - float(g @ z) / float(z @ z)) <= 1e-10 * info.alpha
    ref = o.tt_full(o.tt_svd_dense(o.tt_full(cores) - info.alpha * grad, r))
    assert np.allclose(o.tt_full(new), ref, rtol=1e-9, atol=1e-10)


def rgd_direction(cores, idx, y, n):
    """P_T(P_Omega(T - T*)) with the dense Jacobian projector."""
    Gt = np.zeros(n)
    Gt[tuple(idx.T)] = o.tt_eval(cores, idx) - y
    J = jacobian(cores)
    return (J @ np.linalg.lstsq(J, Gt.reshape(-1), rcond=None)[0]).reshape(n)


def test_uniform_metric_is_rgd_with_constant_step():
    n, r, cores, idx, y = setup_case(24)
    c = 0.8
    p = idx.shape[0] / float(np.prod(n))
    new, info = o.prgd_step(cores, idx, y, n, r, alpha_scale=c, metric="uniform")
    assert abs(info.alpha - c / p) <= 1e-15 * info.alpha
    PG = rgd_direction(cores, idx, y, n)
    ref = o.tt_full(o.tt_svd_dense(o.tt_full(cores) - (c / p) * PG, r))
    assert np.allclose(o.tt_full(new), ref, rtol=1e-9, atol=1e-10)


def test_uniform_metric_adaptive_is_rgd_line_search():
    # RGD with the steepest step: alpha = ||P_T G||^2 / ||P_Omega P_T G||^2
    n, r, cores, idx, y = setup_case(25)
    new, info = o.prgd_step(cores, idx, y, n, r, metric="uniform", step="adaptive")
    PG = rgd_direction(cores, idx, y, n)
    zz = PG[tuple(idx.T)]
    alpha = float(np.sum(PG * PG)) / float(zz @ zz)
    assert abs(info.alpha - alpha) <= 1e-9 * alpha
    ref = o.tt_full(o.tt_svd_dense(o.tt_full(cores) - alpha * PG, r))
    assert np.allclose(o.tt_full(new), ref, rtol=1e-8, atol=1e-9)


def test_weighted_retraction_remark_3_6():
    # T_{l+1} = W^{-1/2} SVD^tt_r(W^{1/2} W_l): dense weighted TT-SVD, unweighted
    n, r, cores, idx, y = setup_case(26)
    m = len(n)
    eps, alpha = 0.5, 0.6
    new, _ = o.prgd_step(cores, idx, y, n, r, eps=eps, alpha=alpha, retraction="weighted")
    grad, G, U, A, g = grad_dense(cores, idx, y, n, eps)
    Wl = o.tt_full(cores) - alpha * grad
    w4 = dense_weight(n, G, 1.0 / (4 * m))
    ref = o.tt_full(o.tt_svd_dense(w4 * Wl, r)) / w4
    assert np.allclose(o.tt_full(new), ref, rtol=1e-9, atol=1e-10)
    # the weighted cores of the result are left-orthogonal (they come out of Algorithm 1)
    hat = o.scale_cores(new, G, 1.0 / (4 * m))
    for c in hat[:-1]:
        L = c.reshape(-1, c.shape[2])
        assert np.allclose(L.T @ L, np.eye(L.shape[1]), atol=1e-11)


def test_weighted_retraction_with_constant_weights_is_plain():
    # W = c I commutes with SVD^tt_r: both retractions agree
    n, r, cores, idx, y = setup_case(27)
    a, _ = o.prgd_step(cores, idx, y, n, r, eps=0.5, alpha=0.3, metric="uniform")
    b, _ = o.prgd_step(cores, idx, y, n, r, eps=0.5, alpha=0.3, metric="uniform", retraction="weighted")
    assert o.tt_dist(a, b) <= 1e-12 * o.tt_norm(a)


def test_variants_solve_recover_planted():
    n, r = (8, 7, 6), (1, 2, 2, 1)
    rng = np.random.default_rng(28)
    truth = [rng.standard_normal((r[k], n[k], r[k + 1])) for k in range(3)]
    allidx = np.array(list(itertools.product(*[range(d) for d in n])))
    idx = allidx[rng.choice(len(allidx), 200, replace=False)]
    y = o.tt_eval(truth, idx)
    init = [t + 0.05 * rng.standard_normal(t.shape) for t in truth]
    for kw in ({"step": "adaptive"}, {"metric": "uniform", "step": "adaptive"}, {"retraction": "weighted"}):
        res = o.solve(init, idx, y, list(n), list(r), truth=truth, alpha_scale=1.0, max_iter=300, tol=1e-8, **kw)
        assert res.converged, kw
