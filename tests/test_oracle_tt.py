"""Pins for the oracle's TT algebra (Section 2) against brute force, closed
forms and library special cases.  CPU only."""
import itertools
import math

import numpy as np
import pytest

import oracle as o
from paper_2501_13385_gb300 import workloads as w


def rand_tt(rng, n, r):
    return [rng.standard_normal((r[k], n[k], r[k + 1])) for k in range(len(n))]


def brute_full(cores):
    """Entry by entry, with explicit matrix products in a Python loop."""
    n = [c.shape[1] for c in cores]
    out = np.zeros(n)
    for x in itertools.product(*[range(d) for d in n]):
        v = np.eye(1)
        for k, c in enumerate(cores):
            v = v @ c[:, x[k], :]
        out[x] = v[0, 0]
    return out


def test_eval_matches_bruteforce():
    rng = np.random.default_rng(1)
    n, r = [3, 4, 2, 3], [1, 2, 3, 2, 1]
    cores = rand_tt(rng, n, r)
    full = brute_full(cores)
    assert np.allclose(o.tt_full(cores), full, rtol=1e-13, atol=1e-13)
    idx = np.array([[0, 0, 0, 0], [2, 3, 1, 2], [1, 2, 0, 1]])
    assert np.allclose(o.tt_eval(cores, idx), full[tuple(idx.T)], rtol=1e-13)


def test_rank_one_closed_form():
    # rank-1 TT is the outer product of the core vectors
    rng = np.random.default_rng(2)
    vecs = [rng.standard_normal(d) for d in (3, 5, 4)]
    cores = [v.reshape(1, -1, 1) for v in vecs]
    assert np.allclose(o.tt_full(cores), np.einsum("a,b,c->abc", *vecs), rtol=1e-14)


def test_separation_factorises_into_parts():
    # T^{<i>} = T^{<=i} T^{>=i+1}  (Section 2, left and right parts)
    rng = np.random.default_rng(3)
    n, r = [3, 2, 4, 2], [1, 2, 3, 2, 1]
    cores = rand_tt(rng, n, r)
    X = brute_full(cores)
    for i in range(1, 4):
        assert np.allclose(o.left_part(cores, i) @ o.right_part(cores, i + 1),
                           o.separation(X, i), rtol=1e-12, atol=1e-12)


def test_tt_svd_reconstructs_exact_low_rank():
    rng = np.random.default_rng(4)
    n, r = [4, 3, 5, 3], [1, 2, 3, 2, 1]
    cores = rand_tt(rng, n, r)
    X = brute_full(cores)
    out = o.tt_svd_dense(X, r)
    assert np.allclose(o.tt_full(out), X, rtol=1e-11, atol=1e-11)
    for k in range(3):
        L = out[k].reshape(-1, out[k].shape[2])
        assert np.allclose(L.T @ L, np.eye(L.shape[1]), atol=1e-12)


def test_tt_svd_matrix_case_is_eckart_young():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((7, 6))
    out = o.tt_svd_dense(X, [1, 2, 1])
    s = np.linalg.svd(X, compute_uv=False)
    err = np.linalg.norm(o.tt_full(out) - X)
    assert err == pytest.approx(math.sqrt((s[2:] ** 2).sum()), rel=1e-12)


def test_tt_svd_oseledets_error_bound():
    # ||X - TT-SVD(X)||^2 <= sum_i (tail energy of the i-th separation)
    rng = np.random.default_rng(6)
    X = rng.standard_normal((3, 4, 3, 4))
    r = [1, 2, 3, 2, 1]
    out = o.tt_svd_dense(X, r)
    err2 = np.linalg.norm(o.tt_full(out) - X) ** 2
    bound = 0.0
    for i in range(1, 4):
        s = np.linalg.svd(o.separation(X, i), compute_uv=False)
        bound += (s[r[i]:] ** 2).sum()
    assert err2 <= bound * (1 + 1e-12)
    assert err2 > 0


def test_round_equals_dense_tt_svd():
    # TT-rounding of a TT is Algorithm 1 on its full tensor (compare full tensors)
    rng = np.random.default_rng(7)
    n, q = [4, 3, 5, 4], [1, 4, 5, 4, 1]
    C = rand_tt(rng, n, q)
    r = [1, 2, 3, 2, 1]
    a = o.tt_full(o.tt_round(C, r))
    b = o.tt_full(o.tt_svd_dense(brute_full(C), r))
    assert np.allclose(a, b, rtol=1e-10, atol=1e-10)


def test_inner_norm_dist_against_dense():
    rng = np.random.default_rng(8)
    n = [3, 4, 3]
    a = rand_tt(rng, n, [1, 2, 2, 1])
    b = rand_tt(rng, n, [1, 3, 2, 1])
    A, B = brute_full(a), brute_full(b)
    assert o.tt_inner(a, b) == pytest.approx(float((A * B).sum()), rel=1e-12)
    assert o.tt_norm(a) == pytest.approx(np.linalg.norm(A), rel=1e-12)
    assert o.tt_dist(a, b) == pytest.approx(np.linalg.norm(A - B), rel=1e-12)
    # distance of nearly equal tensors keeps its relative accuracy (no squared cancellation)
    c = [x.copy() for x in a]
    c[1] = c[1] + 1e-9 * rng.standard_normal(c[1].shape)
    d_dense = np.linalg.norm(brute_full(c) - A)
    assert o.tt_dist(a, c) == pytest.approx(d_dense, rel=1e-5)


def test_left_orthogonalize():
    rng = np.random.default_rng(9)
    n, r = [4, 3, 5], [1, 2, 3, 1]
    cores = rand_tt(rng, n, r)
    U, Rs = o.left_orthogonalize(cores)
    assert np.allclose(o.tt_full(U), o.tt_full(cores), rtol=1e-12, atol=1e-12)
    for k in range(2):
        L = U[k].reshape(-1, U[k].shape[2])
        assert np.allclose(L.T @ L, np.eye(L.shape[1]), atol=1e-13)
        # T^{<=k} = U^{<=k} R_k
        assert np.allclose(o.left_part(cores, k + 1), o.left_part(U, k + 1) @ Rs[k], atol=1e-12)


def test_philox_known_answers():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        v = [int(x, 16) for x in row]
        out = w.philox4x32_10(np.array([v[:4]], dtype=np.uint32), v[4:6])[0]
        assert [int(x) for x in out] == v[6:10]


def test_oversampling_dimensions_golden():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "os_dimensions.txt")
    rows = [l for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) >= 5
    for row in rows:
        ns, rs, dim = [p.strip() for p in row.split("|")]
        n = [int(x) for x in ns.split(",")]
        r = [int(x) for x in rs.split(",")]
        assert w.oversampling_dim(n, r) == int(dim)


def test_generators_shapes_and_spectrum():
    P = w.orthogonal_cubic(0, n1=20, rank=5, frac=0.2)
    assert P.idx.shape == (1600, 3)
    assert len(np.unique(P.idx[:, 0] * 400 + P.idx[:, 1] * 20 + P.idx[:, 2])) == 1600
    X = o.tt_full(P.truth)
    s = np.linalg.svd(o.separation(X, 2), compute_uv=False)
    assert np.allclose(s[:5], np.linspace(10, 1, 5), rtol=1e-12)
    assert np.allclose(P.y, X[tuple(P.idx.T)], rtol=1e-12)
    Q = w.planted_small(3)
    assert o.tt_norm(Q.truth) == pytest.approx(1.0, rel=1e-12)
    assert Q.N == 3000 and Q.r == [1, 2, 2, 2, 1]
    # determinism
    Q2 = w.planted_small(3)
    assert np.array_equal(Q.idx, Q2.idx) and np.array_equal(Q.y, Q2.y)
    assert w.feasible_ranks([4] * 12, 8) == [1, 4] + [8] * 9 + [4, 1]


def test_tt_add_is_the_dense_sum():
    # block cores of A + beta B (ranks add) against the dense sum
    rng = np.random.default_rng(11)
    for n, ra, rb in (([3, 4, 2], [1, 2, 3, 1], [1, 3, 1, 1]), ([5], [1, 1], [1, 1]), ([2, 3, 2, 2], [1, 2, 2, 2, 1], [1, 1, 2, 3, 1])):
        a, b = rand_tt(rng, n, ra), rand_tt(rng, n, rb)
        s = o.tt_add(a, b, -0.75)
        assert [c.shape[0] for c in s[1:]] == [ra[k] + rb[k] for k in range(1, len(n))]
        assert np.allclose(brute_full(s), brute_full(a) - 0.75 * brute_full(b), rtol=1e-13, atol=1e-13)


def test_interface_rows_against_explicit_products():
    # left and right interfaces of mode i for every entry, by explicit slice
    # products in a Python loop; their sandwich of core i is the entry value
    rng = np.random.default_rng(12)
    n, r = [3, 2, 4, 3], [1, 2, 3, 2, 1]
    cores = rand_tt(rng, n, r)
    idx = np.array(list(itertools.product(*[range(d) for d in n])))[::5]
    full = brute_full(cores)
    for i in range(len(n)):
        left, right = o.interface_rows(cores, idx, i)
        for e, x in enumerate(idx):
            lv = np.eye(1)
            for k in range(i):
                lv = lv @ cores[k][:, x[k], :]
            rv = np.eye(1)
            for k in range(len(n) - 1, i, -1):
                rv = cores[k][:, x[k], :] @ rv
            assert np.allclose(left[e], lv[0], rtol=1e-13, atol=1e-14)
            assert np.allclose(right[e], rv[:, 0], rtol=1e-13, atol=1e-14)
            assert math.isclose(left[e] @ cores[i][:, x[i], :] @ right[e], full[tuple(x)], rel_tol=1e-12, abs_tol=1e-13)


def test_right_grams_are_sums_over_all_suffixes():
    # Gam[k] = sum over every suffix multi-index x_{>k} of U^{>=k+1}(x) U^{>=k+1}(x)^T,
    # enumerated by brute force (no recursion)
    rng = np.random.default_rng(13)
    n, r = [2, 3, 2, 3], [1, 2, 3, 2, 1]
    cores = rand_tt(rng, n, r)
    gam = o.right_grams(cores)
    m = len(n)
    assert np.array_equal(gam[m - 1], np.ones((1, 1)))
    for k in range(m - 1):
        G = np.zeros((r[k + 1], r[k + 1]))
        for x in itertools.product(*[range(d) for d in n[k + 1:]]):
            v = np.eye(r[k + 1])
            for j, xj in enumerate(x):
                v = v @ cores[k + 1 + j][:, xj, :]
            G += v @ v.T
        assert np.allclose(gam[k], G, rtol=1e-12, atol=1e-13)
