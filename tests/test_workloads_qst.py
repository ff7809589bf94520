"""The quantum-state-tomography workload (Section 5): the real TT built from a
random MPS must equal the Pauli measurements Tr(rho W_a) of rho = u u^dagger,
computed by brute force with dense Kronecker products.  CPU only."""
import itertools

import numpy as np

import oracle as o
from paper_2501_13385_gb300 import workloads as w


def dense_state(mps):
    u = mps[0]
    for U in mps[1:]:
        u = np.einsum("...a,aib->...ib", u, U)
    return u.reshape(-1)


def test_pauli_measurement_tt_equals_traces():
    mps = w.random_mps(w.Rng(3, 8), 4, 2)
    u = dense_state(mps)
    rho = np.outer(u, u.conj())
    assert abs(np.trace(rho) - 1.0) < 1e-12                       # unit trace
    assert np.min(np.linalg.eigvalsh(rho)) > -1e-12                # positive semidefinite
    cores = w.pauli_measurement_cores(mps)
    assert [c.shape for c in cores] == [(1, 4, 4), (4, 4, 4), (4, 4, 4), (4, 4, 1)]
    T = o.tt_full(cores)
    for a in itertools.product(range(4), repeat=4):
        W = w.PAULI[a[0]]
        for k in a[1:]:
            W = np.kron(W, w.PAULI[k])
        v = np.trace(rho @ W)
        assert abs(v.imag) < 1e-14 and abs(v.real - T[a]) < 1e-13
    # the identity measurement is the trace
    assert abs(T[(0, 0, 0, 0)] - 1.0) < 1e-13


def test_hermitian_basis_is_orthonormal():
    for s in (1, 2, 3):
        H = w.hermitian_basis(s)
        assert H.shape == (s * s, s, s)
        G = np.einsum("aij,bij->ab", H.conj(), H).real
        assert np.allclose(G, np.eye(s * s), atol=1e-15)
        assert all(np.allclose(h, h.conj().T) for h in H)


def test_qst_workload_shape_and_sampling():
    P = w.qst_like(0)
    assert P.n == [4] * 10 and P.r == [1] + [4] * 9 + [1]
    assert P.N == 80000                                # OS 200 x dimension 400 (7.6% of 4^10)
    assert abs(P.N / 4 ** 10 - 0.0763) < 1e-3
    assert np.allclose(o.tt_eval(P.truth, P.idx), P.y, atol=1e-15)
    assert len(np.unique(P.idx.astype(np.int64) @ (4 ** np.arange(9, -1, -1)))) == P.N


def test_huge_tensor_sampling_is_a_set_in_range():
    # tensors with more than 2^53 entries are sampled coordinate by coordinate
    n = [200] * 8
    idx = w.sample_multi_without_replacement(w.Rng(5, 9), n, 5000)
    assert idx.shape == (5000, 8) and idx.min() >= 0 and idx.max() < 200
    assert len(np.unique(idx, axis=0)) == 5000
    P = w.random_request(5)            # order 12, mode 148: about 1e26 entries
    assert P.N == len(np.unique(P.idx, axis=0)) and np.all(P.idx < np.array(P.n))
