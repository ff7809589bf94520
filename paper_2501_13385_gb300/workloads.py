"""Seeded synthetic workloads for TT-format tensor completion.

This module is the single source of inputs for both the CUDA library and the
FP64 CPU oracle.  It draws random numbers and builds problem instances
(ground-truth TT cores, the observed index set Omega, the observed values and
a starting point); it contains none of the PRGD iteration's arithmetic.

Random numbers come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11), written out here from
its published definition, and Gaussians from the Box-Muller transform in FP64.

Core layout everywhere on the host: core k is a C-ordered array of shape
(r_{k-1}, n_k, r_k), the paper's T_k in R^{r_{k-1} x d_k x r_k} (Section 2,
Eq. (TT Core)).  Indices are 0-based.

Workload shapes follow the paper's experiments (Section 5): synthetic
Gaussian/orthogonal-core tensors, a hyperspectral-shaped smooth tensor (in
place of the image data set, which is not available) and a high-order
small-mode tensor shaped like the quantum-state-tomography experiment.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

# --------------------------------------------------------------------------
# Philox4x32-10
# --------------------------------------------------------------------------
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint32(0x9E3779B9)
_W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr: np.ndarray, key: Sequence[int]) -> np.ndarray:
    """Philox4x32 with 10 rounds.

    ctr: uint32 array of shape (K, 4); key: two 32-bit words.
    Returns uint32 array (K, 4).  Each round multiplies words 0 and 2 by the
    two Philox constants, mixes the high halves with words 1, 3 and the key,
    and the key is bumped by the Weyl constants between rounds.
    """
    c = np.asarray(ctr, dtype=np.uint32).reshape(-1, 4)
    x0 = c[:, 0].astype(np.uint64)
    x1 = c[:, 1].astype(np.uint64)
    x2 = c[:, 2].astype(np.uint64)
    x3 = c[:, 3].astype(np.uint64)
    k0 = np.uint32(key[0] & 0xFFFFFFFF)
    k1 = np.uint32(key[1] & 0xFFFFFFFF)
    for rnd in range(10):
        if rnd > 0:
            k0 = np.uint32((int(k0) + int(_W0)) & 0xFFFFFFFF)
            k1 = np.uint32((int(k1) + int(_W1)) & 0xFFFFFFFF)
        p0 = _M0 * x0
        p1 = _M1 * x2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        x0, x1, x2, x3 = (hi1 ^ x1 ^ np.uint64(k0), lo1,
                          hi0 ^ x3 ^ np.uint64(k1), lo0)
    return np.stack([x0, x1, x2, x3], axis=1).astype(np.uint32)


class Rng:
    """Counter-based stream: (seed, stream) select the key / counter word 2;
    successive draws advance a 64-bit block counter held in words 0-1."""

    def __init__(self, seed: int, stream: int = 0):
        self.key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
        self.stream = stream & 0xFFFFFFFF
        self.block = 0

    def u32(self, n: int) -> np.ndarray:
        nb = (n + 3) // 4
        idx = np.arange(self.block, self.block + nb, dtype=np.uint64)
        ctr = np.zeros((nb, 4), dtype=np.uint32)
        ctr[:, 0] = (idx & _MASK32).astype(np.uint32)
        ctr[:, 1] = (idx >> np.uint64(32)).astype(np.uint32)
        ctr[:, 2] = self.stream
        self.block += nb
        return philox4x32_10(ctr, self.key).reshape(-1)[:n]

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in the open interval (0, 1) with 53 random bits."""
        w = self.u32(2 * n).astype(np.uint64).reshape(n, 2)
        a = (w[:, 0] >> np.uint64(5)).astype(np.float64)
        b = (w[:, 1] >> np.uint64(6)).astype(np.float64)
        return (a * 67108864.0 + b + 0.5) / 9007199254740992.0

    def normal(self, n: int) -> np.ndarray:
        """Standard normals by Box-Muller on pairs of uniforms."""
        h = (n + 1) // 2
        u1 = self.uniform(h)
        u2 = self.uniform(h)
        rad = np.sqrt(-2.0 * np.log(u1))
        z = np.empty(2 * h)
        z[0::2] = rad * np.cos(2.0 * math.pi * u2)
        z[1::2] = rad * np.sin(2.0 * math.pi * u2)
        return z[:n]


# --------------------------------------------------------------------------
# Index sets
# --------------------------------------------------------------------------
def sample_linear_without_replacement(rng: Rng, total: int, count: int) -> np.ndarray:
    """`count` distinct linear indices from [0, total), uniform over subsets,
    in draw order (first occurrence kept when a draw repeats)."""
    if count > total:
        raise ValueError("cannot draw more indices than the tensor has")
    out = np.empty(0, dtype=np.int64)
    while out.size < count:
        need = count - out.size
        cand = np.floor(rng.uniform(need + need // 4 + 16) * total).astype(np.int64)
        cand = np.minimum(cand, total - 1)
        allv = np.concatenate([out, cand])
        _, first = np.unique(allv, return_index=True)
        out = allv[np.sort(first)][:count]
    return out


def sample_multi_without_replacement(rng: Rng, n: Sequence[int], count: int) -> np.ndarray:
    """`count` distinct multi-indices drawn uniformly coordinate by coordinate,
    in draw order (first occurrence kept when a draw repeats): the sampler for
    tensors whose entry count does not fit a linear index in double precision
    (above 2^53 entries)."""
    m = len(n)
    nn = np.asarray(n, dtype=np.float64)
    out = np.empty((0, m), dtype=np.int64)
    while out.shape[0] < count:
        need = count - out.shape[0]
        rows = need + need // 4 + 16
        u = rng.uniform(rows * m).reshape(rows, m)
        cand = np.minimum(np.floor(u * nn).astype(np.int64), np.asarray(n, dtype=np.int64) - 1)
        allv = np.concatenate([out, cand])
        _, first = np.unique(allv, axis=0, return_index=True)
        out = allv[np.sort(first)][:count]
    return out.astype(np.int32)


def linear_to_multi(lin: np.ndarray, n: Sequence[int]) -> np.ndarray:
    """Row-major mixed radix: x_1 is the most significant digit."""
    lin = np.asarray(lin, dtype=np.int64).copy()
    m = len(n)
    idx = np.empty((lin.size, m), dtype=np.int32)
    for k in range(m - 1, -1, -1):
        idx[:, k] = (lin % n[k]).astype(np.int32)
        lin //= n[k]
    return idx


def oversampling_dim(n: Sequence[int], r: Sequence[int]) -> int:
    """Dimension of the fixed-TT-rank manifold used by the OS ratio
    (Section 5): sum_k r_{k-1} d_k r_k - sum_{k<m} r_k^2."""
    m = len(n)
    return int(sum(r[k] * n[k] * r[k + 1] for k in range(m)) - sum(r[k] ** 2 for k in range(1, m)))


def feasible_ranks(n: Sequence[int], interior: int) -> List[int]:
    """Clamp a uniform interior rank to the largest separation ranks a
    tensor of these mode sizes can have: r_k <= min(prod_{j<=k} n_j, prod_{j>k} n_j)."""
    m = len(n)
    r = [1]
    for k in range(1, m):
        left = math.prod(n[:k])
        right = math.prod(n[k:])
        r.append(int(min(interior, left, right)))
    r.append(1)
    return r


# --------------------------------------------------------------------------
# Problem container
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Problem:
    name: str
    n: List[int]
    r: List[int]
    idx: np.ndarray               # (N, m) int32, 0-based
    y: np.ndarray                 # (N,) float64 observed values (noise included)
    truth: Optional[List[np.ndarray]]  # ground-truth cores, or None
    init: List[np.ndarray]        # starting cores T_0 (rank r)
    noise_std: float = 0.0
    seed: int = 0

    @property
    def m(self) -> int:
        return len(self.n)

    @property
    def N(self) -> int:
        return int(self.idx.shape[0])

    @property
    def dstar(self) -> int:
        return int(math.prod(self.n))

    @property
    def p(self) -> float:
        return self.N / float(self.dstar)


def _gather_values(cores: Sequence[np.ndarray], idx: np.ndarray, block: int = 1 << 16) -> np.ndarray:
    """Observed values T*(omega) of a ground truth given by cores.

    Small tensors are materialised densely (one Kronecker contraction) and
    indexed; large ones are contracted over gathered slices in blocks.  This
    defines the observation data; it is not part of the PRGD iteration."""
    n = [c.shape[1] for c in cores]
    dstar = math.prod(n)
    if dstar <= (1 << 25):
        full = cores[0].reshape(n[0], -1)
        for c in cores[1:]:
            full = (full @ c.reshape(c.shape[0], -1)).reshape(-1, c.shape[2])
        full = full.reshape(-1)
        lin = np.zeros(idx.shape[0], dtype=np.int64)
        for k in range(len(n)):
            lin = lin * n[k] + idx[:, k]
        return full[lin].copy()
    out = np.empty(idx.shape[0])
    for s in range(0, idx.shape[0], block):
        e = min(idx.shape[0], s + block)
        v = cores[0][0, idx[s:e, 0], :]
        for k in range(1, len(cores)):
            v = np.einsum("ea,aeb->eb", v, cores[k][:, idx[s:e, k], :])
        out[s:e] = v[:, 0]
    return out


def _gaussian_cores(rng: Rng, n, r) -> List[np.ndarray]:
    return [rng.normal(r[k] * n[k] * r[k + 1]).reshape(r[k], n[k], r[k + 1]) for k in range(len(n))]


def _frob_norm_dense(cores) -> float:
    n = [c.shape[1] for c in cores]
    full = cores[0].reshape(n[0], -1)
    for c in cores[1:]:
        full = (full @ c.reshape(c.shape[0], -1)).reshape(-1, c.shape[2])
    return float(np.linalg.norm(full))


def _perturbed_init(rng: Rng, truth, rel: float) -> List[np.ndarray]:
    """T_0 = truth cores plus i.i.d. Gaussian perturbations of relative size
    `rel` per core (Frobenius).  Rank stays r; the start is close to T* as
    the local convergence theory asks (Theorem 4.1)."""
    out = []
    for c in truth:
        e = rng.normal(c.size).reshape(c.shape)
        e *= rel * np.linalg.norm(c) / max(np.linalg.norm(e), 1e-300)
        out.append(c + e)
    return out


def _finish(name, n, r, truth, rng, count, noise_std, noise_mode, init_rel, seed,
            truth_values=None):
    total = math.prod(n)
    if total <= (1 << 53):
        idx = linear_to_multi(sample_linear_without_replacement(rng, total, count), n)
    else:
        idx = sample_multi_without_replacement(rng, n, count)
    y = truth_values(idx) if truth_values is not None else _gather_values(truth, idx)
    if noise_std > 0.0:
        e = rng.normal(y.size)
        if noise_mode == "abs":
            y = y + noise_std * e
        else:   # relative to ||P_Omega T*|| as in the paper's noise experiment
            y = y + noise_std * np.linalg.norm(y) / np.linalg.norm(e) * e
    init = _perturbed_init(Rng(seed, 7), truth, init_rel)
    return Problem(name, list(n), list(r), idx.astype(np.int32), y, truth, init, noise_std, seed)


# --------------------------------------------------------------------------
# The five workload families
# --------------------------------------------------------------------------
def planted_small(seed: int = 0) -> Problem:
    """d=4, n=10 per mode, TT-ranks (1,2,2,2,1); Gaussian cores normalised to
    unit Frobenius norm; 3000 of 10^4 entries observed; noiseless."""
    n, r = [10] * 4, [1, 2, 2, 2, 1]
    rng = Rng(seed, 1)
    cores = _gaussian_cores(rng, n, r)
    s = _frob_norm_dense(cores) ** (1.0 / 4)
    cores = [c / s for c in cores]
    return _finish("planted_small", n, r, cores, rng, 3000, 0.0, "abs", 0.3, seed)


def orthogonal_cubic(seed: int = 0, n1: int = 200, rank: int = 5, frac: float = 0.05) -> Problem:
    """d=3, n=200 per mode, TT-ranks (1,5,5,1).  Cores 1-2 have orthonormal
    left unfoldings (QR of Gaussian matrices); core 3 is diag(10..1) times a
    matrix with orthonormal rows, so the second separation has singular values
    exactly linspace(10, 1, 5).  5% of entries observed; noiseless."""
    n, r = [n1] * 3, [1, rank, rank, 1]
    rng = Rng(seed, 2)
    q1, _ = np.linalg.qr(rng.normal(n1 * rank).reshape(n1, rank))
    q2, _ = np.linalg.qr(rng.normal(rank * n1 * rank).reshape(rank * n1, rank))
    q3, _ = np.linalg.qr(rng.normal(n1 * rank).reshape(n1, rank))
    sig = np.linspace(10.0, 1.0, rank)
    cores = [q1.reshape(1, n1, rank), q2.reshape(rank, n1, rank),
             (sig[:, None] * q3.T).reshape(rank, n1, 1)]
    count = int(round(frac * n1 ** 3))
    return _finish("orthogonal_cubic", n, r, cores, rng, count, 0.0, "abs", 0.1, seed)


def hyperspectral_like(seed: int = 0, shape=(256, 256, 128), terms: int = 20,
                       frac: float = 0.10, noise_std: float = 1e-3) -> Problem:
    """Sum of `terms` separable smooth terms: a 2-D Gaussian bump in the two
    spatial modes (random centre, width 8-32 px) times a smooth spectral curve
    (sum of 2-3 Gaussians over the bands), plus N(0, noise_std^2) noise.  This
    is CP-rank `terms`, hence TT-rank (1, terms, terms, 1); its exact TT form
    is T_1(x1)=[a_q], T_2(x2)=diag(b_q), T_3(x3)=[c_q]^T."""
    n1, n2, n3 = shape
    rng = Rng(seed, 3)
    u = rng.uniform(8 * terms).reshape(terms, 8)
    x1 = np.arange(n1)[None, :]
    x2 = np.arange(n2)[None, :]
    x3 = np.arange(n3)[None, :]
    c1 = (u[:, 0] * n1)[:, None]
    c2 = (u[:, 1] * n2)[:, None]
    w = (8.0 + 24.0 * u[:, 2])[:, None]
    a = np.exp(-0.5 * ((x1 - c1) / w) ** 2)
    b = np.exp(-0.5 * ((x2 - c2) / w) ** 2)
    nb = 2 + (u[:, 3] > 0.5).astype(int)
    spec = np.zeros((terms, n3))
    v = rng.uniform(9 * terms).reshape(terms, 9)
    for q in range(terms):
        for j in range(nb[q]):
            mu = v[q, 3 * j] * n3
            sd = 4.0 + 20.0 * v[q, 3 * j + 1]
            amp = 0.3 + 0.7 * v[q, 3 * j + 2]
            spec[q] += amp * np.exp(-0.5 * ((np.arange(n3) - mu) / sd) ** 2)
    cores = [a.T.reshape(1, n1, terms),
             np.einsum("qx,qs->qxs", b, np.eye(terms)),
             spec.reshape(terms, n3, 1)]
    count = int(round(frac * n1 * n2 * n3))

    def values(idx):
        return np.einsum("eq,eq,eq->e", a.T[idx[:, 0]], b.T[idx[:, 1]], spec.T[idx[:, 2]])

    return _finish("hyperspectral_like", [n1, n2, n3], [1, terms, terms, 1], cores, rng,
                   count, noise_std, "abs", 0.05, seed, truth_values=values)


def tomography_like(seed: int = 0, order: int = 12, mode: int = 4, interior: int = 8,
                    count: int = 200_000, noise_std: float = 1e-4) -> Problem:
    """Order 12, mode size 4 (the Pauli-index shape of the tomography
    experiment), interior TT-rank 8 clamped to the feasible separation ranks,
    Gaussian cores scaled to unit Frobenius norm, 2e5 uniform entries,
    additive N(0, noise_std^2) noise."""
    n = [mode] * order
    r = feasible_ranks(n, interior)
    rng = Rng(seed, 4)
    cores = _gaussian_cores(rng, n, r)
    nrm = _frob_norm_dense(cores) if math.prod(n) <= (1 << 25) else None
    if nrm is None:
        raise ValueError("tomography_like expects a tensor small enough to normalise densely")
    s = nrm ** (1.0 / order)
    cores = [c / s for c in cores]
    return _finish("tomography_like", n, r, cores, rng, count, noise_std, "abs", 0.05, seed)


# Pauli matrices sigma_1..sigma_4 = I, X, Y, Z (Section 5, quantum state tomography)
PAULI = np.array([[[1, 0], [0, 1]], [[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]], dtype=np.complex128)


def hermitian_basis(s: int) -> np.ndarray:
    """An orthonormal basis (Frobenius inner product) of the s x s Hermitian
    matrices over the reals: E_ii, (E_ij + E_ji)/sqrt2, i(E_ij - E_ji)/sqrt2."""
    out = []
    for i in range(s):
        e = np.zeros((s, s), dtype=np.complex128)
        e[i, i] = 1.0
        out.append(e)
    for i in range(s):
        for j in range(i + 1, s):
            e = np.zeros((s, s), dtype=np.complex128)
            e[i, j] = e[j, i] = 1.0 / math.sqrt(2.0)
            out.append(e)
            f = np.zeros((s, s), dtype=np.complex128)
            f[i, j] = -1j / math.sqrt(2.0)
            f[j, i] = 1j / math.sqrt(2.0)
            out.append(f)
    return np.stack(out)


def random_mps(rng: Rng, qubits: int, bond: int) -> List[np.ndarray]:
    """Random matrix product state u = [U_1..U_n], U_k in C^{s_{k-1} x 2 x s_k}
    (s_0 = s_n = 1, interior s = bond), complex Gaussian entries, scaled to
    ||u|| = 1 (so rho = u u^dagger has unit trace)."""
    s = [1] + [bond] * (qubits - 1) + [1]
    cores = []
    for k in range(qubits):
        sz = s[k] * 2 * s[k + 1]
        re, im = rng.normal(sz), rng.normal(sz)
        cores.append((re + 1j * im).reshape(s[k], 2, s[k + 1]))
    # ||u||^2 by the transfer-matrix recursion
    env = np.ones((1, 1), dtype=np.complex128)
    for U in cores:
        env = np.einsum("ab,aic,bid->cd", env, U, U.conj())
    nrm = math.sqrt(float(env.real[0, 0]))
    return [U / nrm ** (1.0 / qubits) for U in cores]


def pauli_measurement_cores(mps: Sequence[np.ndarray]) -> List[np.ndarray]:
    """Real TT cores of T*(a) = Tr(rho W_a), rho = u u^dagger, W_a = sigma_{a_1}
    (x) ... (x) sigma_{a_n} (Section 5).  The left partial products of the
    MPO rho (bond pairs (beta, beta') of the MPS) are Hermitian s x s matrices,
    transported by M -> sum_{i,j} sigma(j, i) U_i^T M conj(U_j); expanding
    them in a real orthonormal basis of the Hermitian matrices gives real
    cores of TT-rank s_k^2."""
    n = len(mps)
    out = []
    bases = [hermitian_basis(U.shape[0]) for U in mps] + [hermitian_basis(1)]
    for k, U in enumerate(mps):
        Hin, Hout = bases[k], bases[k + 1]
        core = np.zeros((len(Hin), 4, len(Hout)))
        for alpha in range(4):
            sig = PAULI[alpha]
            for c, Hc in enumerate(Hin):
                # T_alpha(H_c) = sum_{i,j} sigma(j, i) U_i^T H_c conj(U_j)
                M = np.zeros((U.shape[2], U.shape[2]), dtype=np.complex128)
                for i in range(2):
                    for j in range(2):
                        if sig[j, i] != 0:
                            M += sig[j, i] * (U[:, i, :].T @ Hc @ U[:, j, :].conj())
                for c2, Hd in enumerate(Hout):
                    core[c, alpha, c2] = float(np.real(np.trace(Hd.conj().T @ M)))
        out.append(core)
    return out


def qst_like(seed: int = 0, qubits: int = 10, bond: int = 2, oversampling: float = 200.0,
             init_rel: float = 0.05) -> Problem:
    """Quantum state tomography workload (Section 5): a random MPS with bond
    dimension `bond`, rho = u u^dagger (an MPO of bond dimension bond^2), and
    its Pauli-measurement tensor T*(a) = Tr(rho W_a), an order-`qubits` real
    tensor with mode size 4 and TT-ranks (1, bond^2, ..., bond^2, 1).
    |Omega| = oversampling x (manifold dimension): 80 000 entries (7.6%) for
    10 qubits and bond 2, as in the paper's experiment.  Noiseless."""
    rng = Rng(seed, 8)
    mps = random_mps(rng, qubits, bond)
    truth = pauli_measurement_cores(mps)
    n = [4] * qubits
    r = [1] + [c.shape[2] for c in truth[:-1]] + [1]
    count = min(int(round(oversampling * oversampling_dim(n, r))), math.prod(n))
    return _finish("qst_like", n, r, truth, rng, count, 0.0, "abs", init_rel, seed)


def random_request(seed: int, max_entries: int = 1_000_000) -> Problem:
    """One request of the mixed serving stream: order in [3, 12], mode size in
    [4, 256], interior rank in [2, 16], |Omega| log-uniform in [1e3, 1e6].
    Draws with oversampling below 8 or |Omega| above half the tensor are
    redrawn (such problems are not recoverable)."""
    rng = Rng(seed, 5)
    for _ in range(1000):
        u = rng.uniform(4)
        m = 3 + int(u[0] * 10)
        nn = 4 + int(u[1] * 253)
        rr = 2 + int(u[2] * 15)
        cnt = int(round(10 ** (3 + 3 * u[3])))
        cnt = min(cnt, max_entries)
        n = [nn] * m
        r = feasible_ranks(n, rr)
        dim = oversampling_dim(n, r)
        total = math.prod(n)
        if cnt >= 8 * dim and cnt <= total // 2:
            break
    else:  # pragma: no cover
        raise RuntimeError("no admissible request drawn")
    cores = _gaussian_cores(rng, n, r)
    # unit-scale entries: scale each core so a typical entry is O(1)
    for k in range(m):
        cores[k] /= math.sqrt(r[k])
    return _finish(f"request{seed}", n, r, cores, rng, cnt, 0.0, "abs", 0.05, seed)


CONFIGS = {
    "planted_small": planted_small,
    "orthogonal_cubic": orthogonal_cubic,
    "hyperspectral_like": hyperspectral_like,
    "tomography_like": tomography_like,
}


def random_problem(seed: int, n: Sequence[int], r: Sequence[int], count: int, noise_std: float = 0.0,
                   init_rel: float = 0.1) -> Problem:
    """Small generic instance for edge cases: Gaussian truth cores of ranks r
    scaled to unit-size entries, `count` uniform entries without replacement,
    optional additive noise, start = truth perturbed by `init_rel`."""
    n, r = list(n), list(r)
    rng = Rng(seed, 6)
    cores = _gaussian_cores(rng, n, r)
    for k in range(len(n)):
        cores[k] /= math.sqrt(r[k])
    return _finish(f"random{seed}", n, r, cores, rng, count, noise_std, "abs", init_rel, seed)
