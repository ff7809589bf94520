"""Pins for the oracle's PRGD pieces (Section 3, Algorithm 2, Lemmas 3.3-3.5,
Lemma 4.2) against brute force on tiny tensors: a dense Jacobian of the TT
parameterisation, finite differences, closed forms and a hand-worked step.
CPU only."""
import itertools
import math
import os

import numpy as np
import pytest

import oracle as o
from paper_2501_13385_gb300 import workloads as w


def rand_tt(rng, n, r):
    return [rng.standard_normal((r[k], n[k], r[k + 1])) for k in range(len(n))]


def all_indices(n):
    return np.array(list(itertools.product(*[range(d) for d in n])), dtype=np.int64)


def jacobian(cores):
    """Dense Jacobian of cores -> full tensor (the tensor is linear in each core,
    so a column is the TT with one core replaced by a unit tensor)."""
    cols = []
    for k, c in enumerate(cores):
        for flat in range(c.size):
            e = np.zeros(c.size)
            e[flat] = 1.0
            cs = list(cores)
            cs[k] = e.reshape(c.shape)
            cols.append(o.tt_full(cs).reshape(-1))
    return np.stack(cols, axis=1)


def dense_weight(n, G, power):
    """prod_k G_k(x_k)^power over the full grid, C order."""
    out = np.ones(n)
    for k in range(len(n)):
        shape = [1] * len(n)
        shape[k] = n[k]
        out = out * (G[k] ** power).reshape(shape)
    return out


def setup_case(seed=0, n=(3, 4, 3), r=(1, 2, 2, 1), frac=0.6):
    rng = np.random.default_rng(seed)
    n, r = list(n), list(r)
    cores = rand_tt(rng, n, r)
    truth = rand_tt(rng, n, r)
    allidx = all_indices(n)
    sel = rng.choice(len(allidx), int(frac * len(allidx)), replace=False)
    idx = allidx[sel]
    y = o.tt_eval(truth, idx)
    return n, r, cores, idx, y


def grad_dense(cores, idx, y, n, eps):
    """The oracle's Riemannian gradient tilde P_T W^{-1} G_l as a dense tensor,
    assembled from its own pieces."""
    m = len(n)
    g = o.residual(cores, idx, y)
    G = o.metric_diagonals(g, idx, n, eps)
    U, _ = o.left_orthogonalize(o.scale_cores(cores, G, 1.0 / (4 * m)))
    A = o.tangent_project_hat(U, idx, g * o.weight_entries(idx, G, -1.0 / (4 * m)))
    return o.tangent_to_full(U, A) * dense_weight(n, G, -1.0 / (4 * m)), G, U, A, g


def weighted_proj_dense(cores, G, n, Z):
    m = len(n)
    allidx = all_indices(n)
    U, A = o.weighted_projection_components(cores, G, allidx, Z.reshape(-1))
    return o.tangent_to_full(U, A) * dense_weight(n, G, -1.0 / (4 * m))


def test_residual_and_slice_energy_bruteforce():
    n, r, cores, idx, y = setup_case(1)
    X = o.tt_full(cores)
    g = o.residual(cores, idx, y)
    gd = np.array([X[tuple(i)] - yy for i, yy in zip(idx, y)])
    assert np.allclose(g, gd, rtol=1e-13, atol=1e-14)
    for i in range(3):
        s = o.slice_energy(g, idx[:, i], n[i])
        sd = np.zeros(n[i])
        for e, gv in zip(idx, g):
            sd[e[i]] += gv * gv
        assert np.allclose(s, sd, rtol=1e-13)
        # it is diag(M_i(G) M_i(G)^T) of the dense sparse-residual tensor
        Gt = np.zeros(n)
        Gt[tuple(idx.T)] = g
        Mi = np.moveaxis(Gt, i, 0).reshape(n[i], -1)
        assert np.allclose(s, np.diag(Mi @ Mi.T), rtol=1e-13)


def test_component_weight_property():
    # Proposition 3.1: W T has cores T_i x_2 G_i^{1/(2m)}
    rng = np.random.default_rng(2)
    n, r = [3, 4, 2], [1, 2, 2, 1]
    cores = rand_tt(rng, n, r)
    G = [rng.uniform(0.5, 3.0, d) for d in n]
    lhs = o.tt_full(o.scale_cores(cores, G, 1.0 / 6))
    rhs = o.tt_full(cores) * dense_weight(n, G, 1.0 / 6)
    assert np.allclose(lhs, rhs, rtol=1e-13)


def test_euclidean_projection_equals_jacobian_projector():
    rng = np.random.default_rng(3)
    n, r = [3, 4, 3], [1, 2, 2, 1]
    cores = rand_tt(rng, n, r)
    U, _ = o.left_orthogonalize(cores)
    Z = rng.standard_normal(n)
    A = o.tangent_project_hat(U, all_indices(n), Z.reshape(-1))
    P = o.tangent_to_full(U, A)
    J = jacobian(U)
    Pd = J @ np.linalg.lstsq(J, Z.reshape(-1), rcond=None)[0]
    assert np.allclose(P.reshape(-1), Pd, rtol=1e-9, atol=1e-10)


def test_weighted_projection_equals_weighted_jacobian_projector():
    # tilde P_T minimises ||A - J theta||_W : J (J^T W J)^+ J^T W a (Lemma 3.5)
    rng = np.random.default_rng(4)
    n, r = [3, 3, 4], [1, 2, 2, 1]
    cores = rand_tt(rng, n, r)
    G = [rng.uniform(0.2, 5.0, d) for d in n]
    Z = rng.standard_normal(n)
    P = weighted_proj_dense(cores, G, n, Z)
    J = jacobian(cores)
    Wd = dense_weight(n, G, 1.0 / 6).reshape(-1)
    M = J.T @ (Wd[:, None] * J)
    Pd = J @ (np.linalg.pinv(M, rcond=1e-12) @ (J.T @ (Wd * Z.reshape(-1))))
    assert np.allclose(P.reshape(-1), Pd, rtol=1e-8, atol=1e-9)
    # and it differs from the Euclidean projector when weights are not uniform
    Pe = J @ np.linalg.lstsq(J, Z.reshape(-1), rcond=None)[0]
    assert np.linalg.norm(Pe - Pd) > 1e-3


def test_projection_idempotent_and_w_orthogonal():
    rng = np.random.default_rng(5)
    n, r = [4, 3, 3], [1, 2, 3, 1]
    cores = rand_tt(rng, n, r)
    G = [rng.uniform(0.2, 5.0, d) for d in n]
    Z = rng.standard_normal(n)
    P = weighted_proj_dense(cores, G, n, Z)
    PP = weighted_proj_dense(cores, G, n, P)
    assert np.allclose(PP, P, rtol=1e-9, atol=1e-10)
    Wd = dense_weight(n, G, 1.0 / 6)
    assert abs(((Z - P) * Wd * P).sum()) < 1e-9 * np.linalg.norm(Z) ** 2
    # in the hat frame the projection is Euclidean-orthogonal
    m = 3
    U, A = o.weighted_projection_components(cores, G, all_indices(n), Z.reshape(-1))
    Ph = o.tangent_to_full(U, A)
    Zh = Z * dense_weight(n, G, 1 / 12)
    assert abs(((Zh - Ph) * Ph).sum()) < 1e-9 * np.linalg.norm(Zh) ** 2


def test_components_are_w_orthogonal_lemma_3_4():
    rng = np.random.default_rng(6)
    n, r = [3, 4, 3, 2], [1, 2, 2, 2, 1]
    m = 4
    cores = rand_tt(rng, n, r)
    G = [rng.uniform(0.3, 4.0, d) for d in n]
    Z = rng.standard_normal(n)
    U, A = o.weighted_projection_components(cores, G, all_indices(n), (Z * dense_weight(n, G, 1 / (4 * m))).reshape(-1))
    Wm = dense_weight(n, G, -1.0 / (4 * m))
    Wd = dense_weight(n, G, 1.0 / (2 * m))
    comps = []
    for i in range(m):
        cs = list(U)
        cs[i] = A[i]
        comps.append(o.tt_full(cs) * Wm)
    for i in range(m):
        for j in range(i + 1, m):
            ip = (comps[i] * Wd * comps[j]).sum()
            assert abs(ip) < 1e-10 * np.linalg.norm(Z) ** 2


def test_new_left_orthogonal_lemma_3_3():
    # tilde T_i = U_i x_2 G_i^{-1/(4m)} satisfies
    # tilde T^{<=i T} (G_1^{1/2m} (x) ... (x) G_i^{1/2m}) tilde T^{<=i} = I
    rng = np.random.default_rng(7)
    n, r = [3, 4, 3], [1, 2, 3, 1]
    m = 3
    cores = rand_tt(rng, n, r)
    G = [rng.uniform(0.3, 4.0, d) for d in n]
    U, _ = o.left_orthogonalize(o.scale_cores(cores, G, 1.0 / (4 * m)))
    Tt = o.scale_cores(U, G, -1.0 / (4 * m))
    assert np.allclose(o.tt_full(Tt), o.tt_full(cores), rtol=1e-12)
    for i in range(1, m):
        L = o.left_part(Tt, i)
        wk = np.ones(1)
        for k in range(i):
            wk = np.kron(wk, G[k] ** (1.0 / (2 * m)))
        assert np.allclose(L.T @ (wk[:, None] * L), np.eye(r[i]), atol=1e-12)


def test_gradient_by_finite_differences():
    # d/dt f(T + tZ) = <Z, G> = <Z, grad f>_W for tangent Z (Section 3.2)
    n, r, cores, idx, y = setup_case(8)
    m = 3
    eps = 0.7
    grad, G, U, A, g = grad_dense(cores, idx, y, n, eps)
    rng = np.random.default_rng(18)
    J = jacobian(cores)
    Z = (J @ rng.standard_normal(J.shape[1])).reshape(n)
    X = o.tt_full(cores)

    def f(Xt):
        return 0.5 * sum((Xt[tuple(i)] - yy) ** 2 for i, yy in zip(idx, y))

    h = 1e-6
    fd = (f(X + h * Z) - f(X - h * Z)) / (2 * h)
    Wd = dense_weight(n, G, 1.0 / (2 * m))
    assert fd == pytest.approx(float((Z * Wd * grad).sum()), rel=1e-7)
    # grad lies in the tangent space
    Pg = J @ np.linalg.lstsq(J, grad.reshape(-1), rcond=None)[0]
    assert np.allclose(Pg, grad.reshape(-1), atol=1e-10)


def test_assembled_rank_2r_cores_and_step():
    n, r, cores, idx, y = setup_case(9)
    eps, alpha = 0.5, 0.8
    grad, G, U, A, g = grad_dense(cores, idx, y, n, eps)
    C = o.assemble_2r(U, A, alpha, G)
    X = o.tt_full(cores)
    assert np.allclose(o.tt_full(C), X - alpha * grad, rtol=1e-11, atol=1e-12)
    assert [c.shape[0] for c in C] == [1, 4, 4] and [c.shape[2] for c in C] == [4, 4, 1]
    new, info = o.prgd_step(cores, idx, y, n, r, eps=eps, alpha=alpha)
    ref = o.tt_full(o.tt_svd_dense(X - alpha * grad, r))
    assert np.allclose(o.tt_full(new), ref, rtol=1e-10, atol=1e-11)


def test_zero_tangent_retraction_returns_point():
    n, r, cores, idx, y = setup_case(10)
    grad, G, U, A, g = grad_dense(cores, idx, y, n, 1.0)
    new = o.tt_round(o.assemble_2r(U, A, 0.0, G), r)
    assert np.allclose(o.tt_full(new), o.tt_full(cores), rtol=1e-11, atol=1e-12)


def test_uniform_weights_reduce_to_rgd():
    # eps -> infinity: G_i -> eps I, grad -> eps^{-1/2} P_T(G), alpha eps^{-1/2} = c/p:
    # RGD of Section 3.1 with step c/p, written here with the dense Jacobian projector
    n, r, cores, idx, y = setup_case(11)
    c = 0.9
    p = idx.shape[0] / float(np.prod(n))
    eps = 1e24
    new, _ = o.prgd_step(cores, idx, y, n, r, eps=eps, alpha=c * math.sqrt(eps) / p)
    X = o.tt_full(cores)
    Gt = np.zeros(n)
    Gt[tuple(idx.T)] = o.tt_eval(cores, idx) - y
    J = jacobian(cores)
    PG = (J @ np.linalg.lstsq(J, Gt.reshape(-1), rcond=None)[0]).reshape(n)
    ref = o.tt_full(o.tt_svd_dense(X - (c / p) * PG, r))
    assert np.allclose(o.tt_full(new), ref, rtol=1e-8, atol=1e-9)


def test_matrix_case_projection_formula():
    # m = 2: P_T(Z) = UU^T Z + Z VV^T - UU^T Z VV^T
    rng = np.random.default_rng(12)
    cores = rand_tt(rng, [5, 6], [1, 2, 1])
    U, _ = o.left_orthogonalize(cores)
    Z = rng.standard_normal((5, 6))
    A = o.tangent_project_hat(U, all_indices([5, 6]), Z.reshape(-1))
    P = o.tangent_to_full(U, A)
    X = o.tt_full(cores)
    u, s, vt = np.linalg.svd(X)
    Uu, Vv = u[:, :2], vt[:2].T
    ref = Uu @ Uu.T @ Z + Z @ Vv @ Vv.T - Uu @ Uu.T @ Z @ Vv @ Vv.T
    assert np.allclose(P, ref, rtol=1e-10, atol=1e-11)


def test_norm_equivalence_lemma_4_2():
    n, r, cores, idx, y = setup_case(13)
    m = 3
    g = o.residual(cores, idx, y)
    eps = 0.3
    G = o.metric_diagonals(g, idx, n, eps)
    gvee = max(math.sqrt(s.max()) for s in (Gi - eps for Gi in G))
    nu, mu = math.sqrt(eps), math.sqrt(eps + gvee ** 2)
    rng = np.random.default_rng(13)
    for _ in range(5):
        Z = rng.standard_normal(n)
        zw = (Z * Z * dense_weight(n, G, 1.0 / (2 * m))).sum()
        z2 = (Z * Z).sum()
        assert nu * z2 <= zw * (1 + 1e-12) and zw <= mu * z2 * (1 + 1e-12)


def test_tt_svd_perturbation_bound_lemma_26():
    # ||SVD^tt_r(T* + D) - T*||^2 <= ||D||^2 + 600 m ||D||^3 / sigma_min(T*)
    rng = np.random.default_rng(14)
    n, r = [4, 5, 4], [1, 2, 2, 1]
    T = o.tt_full(rand_tt(rng, n, r))
    smin = min(np.linalg.svd(o.separation(T, i), compute_uv=False)[r[i] - 1] for i in (1, 2))
    for scale in (1e-3, 1e-2):
        D = scale * rng.standard_normal(n)
        err = np.linalg.norm(o.tt_full(o.tt_svd_dense(T + D, r)) - T)
        dn = np.linalg.norm(D)
        assert err ** 2 <= dn ** 2 + 600 * 3 * dn ** 3 / smin


def test_hand_worked_rank1_step_golden():
    path = os.path.join(os.path.dirname(__file__), "golden", "rank1_matrix_step.txt")
    rows = [l.strip() for l in open(path) if l.strip() and not l.startswith("#")]
    W0 = np.array([eval(x, {"sqrt": math.sqrt}) for x in rows]).reshape(2, 2)
    cores = [np.array([1.0, 2.0]).reshape(1, 2, 1), np.array([3.0, 4.0]).reshape(1, 2, 1)]
    idx = np.array([[0, 0], [1, 1]])
    y = np.array([4.0, 7.0])
    n, r = [2, 2], [1, 1, 1]
    g = o.residual(cores, idx, y)
    eps = o.eps_from_residual(g, n, 1.0)
    alpha = o.alpha_from_eps(eps, 0.5, 1.0)
    assert eps == 1.0 and alpha == 2.0
    G = o.metric_diagonals(g, idx, n, eps)
    U, A = o.weighted_projection_components(cores, G, idx, g * o.weight_entries(idx, G, -1.0 / 4))  # W^{-1} G
    C = o.assemble_2r(U, A, alpha, G)
    assert np.allclose(o.tt_full(C), W0, rtol=1e-14, atol=1e-14)
    new, _ = o.prgd_step(cores, idx, y, n, r, eps_rel=1.0, alpha_scale=1.0)
    u, s, vt = np.linalg.svd(W0)
    assert np.allclose(o.tt_full(new), s[0] * np.outer(u[:, 0], vt[0]), rtol=1e-13)


def test_planted_recovery_to_1e_10():
    P = w.planted_small(0)
    res = o.solve(P.init, P.idx, P.y, P.n, P.r, truth=P.truth, eps_rel=1.0, alpha_scale=1.5,
                  max_iter=200, tol=1e-10)
    assert res.converged and res.history[-1] <= 1e-10
    h = np.array(res.history)
    # linear convergence: the error shrinks over every block of 5 iterations after the start
    assert all(h[i + 5] < h[i] for i in range(5, len(h) - 5))
