"""Plain FP64 CPU oracle of Preconditioned Riemannian Gradient Descent (PRGD)
for low-TT-rank tensor completion, following the paper step by step.

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and
by bench.py's CPU-baseline leg; never by the product path.  It shares no code
with the CUDA library.

Conventions: core k is an array of shape (r_{k-1}, n_k, r_k) (the paper's T_k
in R^{r_{k-1} x d_k x r_k}); indices are 0-based; `idx` is (N, m) int.
Vectorisation over the observed entries is plain numpy broadcasting; there is
no blocking, fusion or reordering beyond what each cited definition states.

Readings of points the paper leaves open (each is a documented choice):
  * epsilon (Section 3.2, the constant in G_{l,i}) is not given a value.  Here
    eps_l = eps_rel * ||G_l||_F^2 / min_i d_i (the mean mode-slice energy of
    the residual of the most finely divided mode), recomputed every iteration
    (the theory indexes it by l, Theorem 4.1); `eps_mode="frozen"` keeps the
    value of iteration 0.
  * the step size is the constant-in-form choice of Theorem 4.1,
    alpha_l = alpha_scale * eps_l^{1/2} / p with p = |Omega| / d*; the
    steepest step of Eq. (PRGD stepsize) is the "adaptive" variant.
  * the Trim step of Algorithm 2 is skipped, which Section 3.2 allows.
  * the left-orthogonal decomposition of W^{1/2} T is taken by Householder QR
    (any left-orthogonal decomposition spans the same tangent space).
Parity pins for every function live in tests/test_oracle_*.py.  The eps/alpha
policy values themselves are tuned, not derived: parity unpinned for them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

Cores = List[np.ndarray]


# ---------------------------------------------------------------------------
# TT algebra (Section 2)
# ---------------------------------------------------------------------------
def tt_eval(cores: Sequence[np.ndarray], idx: np.ndarray) -> np.ndarray:
    """Entries T(x) = T_1(x_1,:) T_2(:,x_2,:) ... T_m(:,x_m)  (Eq. (TT Core)),
    evaluated left to right for every row of idx."""
    idx = np.asarray(idx)
    v = cores[0][0, idx[:, 0], :]                       # (N, r_1)
    for k in range(1, len(cores)):
        slices = np.transpose(cores[k][:, idx[:, k], :], (1, 0, 2))   # (N, r_{k-1}, r_k)
        v = np.einsum("ea,eab->eb", v, slices)
    return v[:, 0].copy()


def tt_full(cores: Sequence[np.ndarray]) -> np.ndarray:
    """Dense tensor of a TT (brute force over all d* entries)."""
    n = [c.shape[1] for c in cores]
    grids = np.indices(n).reshape(len(n), -1).T
    return tt_eval(cores, grids).reshape(n)


def left_part(cores: Sequence[np.ndarray], i: int) -> np.ndarray:
    """T^{<=i}: matrix (d_1...d_i) x r_i (Section 2, left parts), i >= 1."""
    M = cores[0].reshape(cores[0].shape[1], cores[0].shape[2])
    for k in range(1, i):
        c = cores[k]
        M = (M @ c.reshape(c.shape[0], -1)).reshape(-1, c.shape[2])
    return M


def right_part(cores: Sequence[np.ndarray], i: int) -> np.ndarray:
    """T^{>=i}: matrix r_{i-1} x (d_i...d_m) (Section 2, right parts), 1-based i."""
    m = len(cores)
    c = cores[m - 1]
    M = c.reshape(c.shape[0], -1)
    for k in range(m - 2, i - 2, -1):
        c = cores[k]
        M = (c.reshape(-1, c.shape[2]) @ M).reshape(c.shape[0], -1)
    return M


def separation(X: np.ndarray, i: int) -> np.ndarray:
    """X^{<i>}: reshape to (d_1...d_i) x (d_{i+1}...d_m)."""
    n = X.shape
    return X.reshape(int(np.prod(n[:i])), -1)


def tt_svd_dense(X: np.ndarray, r: Sequence[int]) -> Cores:
    """Algorithm 1 (TT-SVD) on a full tensor, literally:
    L(T_i) <- top r_i left singular vectors of (T^{<=i-1} (x) I_{d_i})^T X^{<i>},
    T^{<=i} = (T^{<=i-1} (x) I) L(T_i);  T_m = (T^{<=m-1})^T X^{<m-1>}."""
    n = X.shape
    m = len(n)
    cores = []
    left = np.ones((1, 1))                               # T^{<=0} = [1]
    for i in range(1, m):
        Xi = separation(X, i)                             # (d_1..d_i) x rest
        K = np.kron(left, np.eye(n[i - 1]))               # (d_1..d_i) x (r_{i-1} d_i)
        M = K.T @ Xi
        U, _, _ = np.linalg.svd(M, full_matrices=False)
        Li = U[:, : r[i]]
        cores.append(Li.reshape(left.shape[1], n[i - 1], r[i]))
        left = K @ Li
    Tm = left.T @ separation(X, m - 1)
    cores.append(Tm.reshape(left.shape[1], n[m - 1], 1))
    return cores


def tt_inner(a: Sequence[np.ndarray], b: Sequence[np.ndarray]) -> float:
    """<A, B> by the left Gram sweep  Lam_k = sum_x A_k(x)^T Lam_{k-1} B_k(x)."""
    lam = np.ones((1, 1))
    for ca, cb in zip(a, b):
        lam = np.einsum("ij,ixk,jxl->kl", lam, ca, cb)
    return float(lam[0, 0])


def tt_add(a: Sequence[np.ndarray], b: Sequence[np.ndarray], beta: float = 1.0) -> Cores:
    """Cores of A + beta*B in block form (rank adds)."""
    m = len(a)
    out = []
    for k in range(m):
        ca, cb = a[k], b[k]
        if m == 1:
            out.append(ca + beta * cb)
        elif k == 0:
            out.append(np.concatenate([ca, beta * cb], axis=2))
        elif k == m - 1:
            out.append(np.concatenate([ca, cb], axis=0))
        else:
            ra, n, sa = ca.shape
            rb, _, sb = cb.shape
            c = np.zeros((ra + rb, n, sa + sb))
            c[:ra, :, :sa] = ca
            c[ra:, :, sa:] = cb
            out.append(c)
    return out


def tt_norm(cores: Sequence[np.ndarray]) -> float:
    """||T||_F via a left-orthogonalising QR sweep (no squared cancellation):
    the norm is that of the last core after the sweep."""
    cur = [c.copy() for c in cores]
    for k in range(len(cur) - 1):
        c = cur[k]
        q, rr = np.linalg.qr(c.reshape(-1, c.shape[2]))
        cur[k] = q.reshape(c.shape[0], c.shape[1], q.shape[1])
        nxt = cur[k + 1]
        cur[k + 1] = (rr @ nxt.reshape(nxt.shape[0], -1)).reshape(rr.shape[0], nxt.shape[1], nxt.shape[2])
    return float(np.linalg.norm(cur[-1]))


def tt_dist(a, b) -> float:
    """||A - B||_F."""
    return tt_norm(tt_add(a, b, -1.0))


# ---------------------------------------------------------------------------
# Problem pieces (Eq. (model: Low TT), Section 3.2)
# ---------------------------------------------------------------------------
def residual(cores, idx, y) -> np.ndarray:
    """Entries of G_l = P_Omega(T_l - T*) on Omega (Algorithm 2, first line)."""
    return tt_eval(cores, idx) - np.asarray(y, dtype=np.float64)


def slice_energy(g: np.ndarray, xi: np.ndarray, d: int) -> np.ndarray:
    """diag(M_i(G) M_i(G)^T): squared norm of every mode-i slice of the sparse
    residual, i.e. sum of g^2 over the entries with x_i = x (Section 3.2)."""
    return np.bincount(np.asarray(xi, dtype=np.int64), weights=g * g, minlength=d).astype(np.float64)


def metric_diagonals(g, idx, n, eps) -> List[np.ndarray]:
    """Diagonals of G_{l,i} = eps I + diag(M_i(G_l) M_i(G_l)^T) (Section 3.2)."""
    return [eps + slice_energy(g, idx[:, i], n[i]) for i in range(len(n))]


def scale_cores(cores, G, power) -> Cores:
    """[T_1 x_2 G_1^power, ..., T_m x_2 G_m^power] (Proposition 3.1)."""
    return [c * (G[k] ** power)[None, :, None] for k, c in enumerate(cores)]


def weight_entries(idx, G, power) -> np.ndarray:
    """prod_k G_k(x_k)^power for every observed index: the entrywise action of
    W^{power*2m} on a sparse tensor (Eq. (new metric))."""
    w = np.ones(idx.shape[0])
    for k in range(idx.shape[1]):
        w = w * G[k][idx[:, k]] ** power
    return w


def left_orthogonalize(cores) -> Tuple[Cores, List[np.ndarray]]:
    """Left-orthogonal decomposition by a Householder-QR sweep over the left
    unfoldings L(T_i) (Section 2): returns U (U_1..U_{m-1} left-orthogonal,
    U_m carrying the remainder) and the factors R_i with T^{<=i} = U^{<=i} R_i."""
    cur = [c.copy() for c in cores]
    Rs = []
    for k in range(len(cur) - 1):
        c = cur[k]
        q, rr = np.linalg.qr(c.reshape(-1, c.shape[2]))
        cur[k] = q.reshape(c.shape[0], c.shape[1], q.shape[1])
        Rs.append(rr)
        nxt = cur[k + 1]
        cur[k + 1] = (rr @ nxt.reshape(nxt.shape[0], -1)).reshape(rr.shape[0], nxt.shape[1], nxt.shape[2])
    return cur, Rs


def interface_rows(cores, idx, i) -> Tuple[np.ndarray, np.ndarray]:
    """For mode i (0-based): left interfaces U^{<=i-1}(x_<i) as rows (N, r_{i-1})
    and right interfaces U^{>=i+1}(x_>i) as rows (N, r_i) (Section 2)."""
    N = idx.shape[0]
    m = len(cores)
    left = np.ones((N, 1))
    for k in range(i):
        left = np.einsum("ea,eab->eb", left, np.transpose(cores[k][:, idx[:, k], :], (1, 0, 2)))
    right = np.ones((N, 1))
    for k in range(m - 1, i, -1):
        right = np.einsum("eab,eb->ea", np.transpose(cores[k][:, idx[:, k], :], (1, 0, 2)), right)
    return left, right


def right_grams(cores) -> List[np.ndarray]:
    """Gam[k] = U^{>=k+1} (U^{>=k+1})^T for k = 0..m-1 (0-based; Gam[m-1] = [1]),
    by the recursion Gam = sum_x U_k(x) Gam_next U_k(x)^T."""
    m = len(cores)
    gam = [None] * m
    gam[m - 1] = np.ones((1, 1))
    for k in range(m - 1, 0, -1):
        gam[k - 1] = np.einsum("axb,bc,dxc->ad", cores[k], gam[k], cores[k])
    return gam


def tangent_project_hat(U, idx, vals, block: int = 1 << 15) -> Cores:
    """Euclidean tangent-space projection at U (left-orthogonal cores) of the
    sparse tensor with entries `vals` on `idx`, Lemma 3.5 Eq. (tsp in nm):
      L(A_i) = (I - L(U_i) L(U_i)^T) (U^{<=i-1} (x) I)^T A^{<i>} (U^{>=i+1})^T
               (U^{>=i+1} U^{>=i+1 T})^{-1},   i < m,
      L(A_m) = (U^{<=m-1} (x) I)^T A^{<m>}.
    The middle factor is written slice by slice: its (j, x, k) entry is the
    sum over observed entries with x_i = x of a * U^{<=i-1}(.., j) U^{>=i+1}(k, ..)."""
    m = len(U)
    gam = right_grams(U)
    comps = []
    for i in range(m):
        ra, d, rb = U[i].shape
        D = np.zeros((d, ra * rb))
        for s in range(0, idx.shape[0], block):
            e = min(idx.shape[0], s + block)
            left, right = interface_rows(U, idx[s:e], i)
            outer = (vals[s:e, None] * left)[:, :, None] * right[:, None, :]
            np.add.at(D, idx[s:e, i], outer.reshape(e - s, -1))
        D = D.reshape(d, ra, rb).transpose(1, 0, 2)                 # (ra, d, rb)
        LD = D.reshape(ra * d, rb)
        if i < m - 1:
            LU = U[i].reshape(ra * d, rb)
            LD = LD - LU @ (LU.T @ LD)
            LD = np.linalg.solve(gam[i].T, LD.T).T                  # right-multiply by Gam^{-1}
        comps.append(LD.reshape(ra, d, rb))
    return comps


def tangent_to_full(U, A) -> np.ndarray:
    """sum_i [U_1, ..., A_i, ..., U_m] as a dense tensor (tiny sizes only)."""
    total = 0.0
    for i in range(len(U)):
        cs = list(U)
        cs[i] = A[i]
        total = total + tt_full(cs)
    return total


def weighted_projection_components(cores, G, idx, vals):
    """tilde P_T of a sparse tensor under <.,.>_W (Lemma 3.5):
    tilde P_T = W^{-1/2} P_{T^} W^{1/2}, with T^ = W^{1/2} T.
    Returns (U, A, G): U the left-orthogonal cores of T^, A the components of
    P_{T^}(W^{1/2} vals); the tangent vector itself is W^{-1/2} sum_i [U..A_i..U]."""
    m = len(cores)
    That = scale_cores(cores, G, 1.0 / (4 * m))
    U, _ = left_orthogonalize(That)
    ahat = vals * weight_entries(idx, G, 1.0 / (4 * m))
    A = tangent_project_hat(U, idx, ahat)
    return U, A


def assemble_2r(U, A, alpha, G) -> Cores:
    """Rank-2r cores of W_l = W^{-1/2}(T^ - alpha P_{T^} W^{-1/2} G_l)
    (Algorithm 2, third line, with Lemma 3.5): V_i = -alpha A_i and
      C_1 = [V_1  U_1],  C_i = [[U_i, 0], [V_i, U_i]],  C_m = [[U_m], [U_m + V_m]],
    then every slice x of C_i is multiplied by G_i(x)^{-1/(4m)} (Proposition 3.1)."""
    m = len(U)
    C = []
    for i in range(m):
        Ui, Vi = U[i], -alpha * A[i]
        ra, d, rb = Ui.shape
        if m == 1:
            c = Ui + Vi
        elif i == 0:
            c = np.concatenate([Vi, Ui], axis=2)
        elif i == m - 1:
            c = np.concatenate([Ui, Ui + Vi], axis=0)
        else:
            c = np.zeros((2 * ra, d, 2 * rb))
            c[:ra, :, :rb] = Ui
            c[ra:, :, :rb] = Vi
            c[ra:, :, rb:] = Ui
        C.append(c * (G[i] ** (-1.0 / (4 * m)))[None, :, None])
    return C


def tangent_tt(U, A) -> Cores:
    """The tangent vector sum_i [U_1, ..., A_i, ..., U_m] (Section 3.3,
    tangent space parameterisation) as one TT of rank 2r: cores [A_1 U_1],
    [[U_i, 0], [A_i, U_i]] and [[U_m], [A_m]]."""
    m = len(U)
    out = []
    for i in range(m):
        Ui, Ai = U[i], A[i]
        ra, d, rb = Ui.shape
        if m == 1:
            c = Ai.copy()
        elif i == 0:
            c = np.concatenate([Ai, Ui], axis=2)
        elif i == m - 1:
            c = np.concatenate([Ui, Ai], axis=0)
        else:
            c = np.zeros((2 * ra, d, 2 * rb))
            c[:ra, :, :rb] = Ui
            c[ra:, :, :rb] = Ai
            c[ra:, :, rb:] = Ui
        out.append(c)
    return out


def adaptive_step(U, A, G, idx) -> float:
    """The steepest step along the search direction, Eq. (PRGD stepsize):
    alpha_l = ||Z||_W^2 / ||P_Omega Z||_F^2 with Z = tilde P_T W^{-1} G_l.
    By Lemma 3.5, W^{1/2} Z = P_{T^} W^{-1/2} G_l is the tangent TT of the
    components A at U, so ||Z||_W is its Frobenius norm; Z itself is that TT
    with every core slice scaled by G_i(x)^{-1/(4m)} (Proposition 3.1),
    evaluated at Omega."""
    m = len(U)
    Zhat = tangent_tt(U, A)
    num = tt_norm(Zhat) ** 2
    z = tt_eval(scale_cores(Zhat, G, -1.0 / (4 * m)), idx)
    return num / float(z @ z)


def tt_round(C, r) -> Cores:
    """SVD^tt_r of a TT given by cores (Algorithm 1 applied to a low-rank TT):
    right-to-left Householder QR of R(C_k)^T, then left-to-right truncated SVD
    of L(C_k), pushing S V^T into the next core.  Output is left-orthogonal."""
    cur = [c.copy() for c in C]
    m = len(cur)
    for k in range(m - 1, 0, -1):
        c = cur[k]
        q, rr = np.linalg.qr(c.reshape(c.shape[0], -1).T)          # R(C_k)^T = Q R
        cur[k] = q.T.reshape(q.shape[1], c.shape[1], c.shape[2])
        p = cur[k - 1]
        cur[k - 1] = (p.reshape(-1, p.shape[2]) @ rr.T).reshape(p.shape[0], p.shape[1], rr.shape[0])
    for k in range(m - 1):
        c = cur[k]
        u, s, vt = np.linalg.svd(c.reshape(-1, c.shape[2]), full_matrices=False)
        t = r[k + 1]
        cur[k] = u[:, :t].reshape(c.shape[0], c.shape[1], t)
        sv = s[:t, None] * vt[:t]
        nxt = cur[k + 1]
        cur[k + 1] = (sv @ nxt.reshape(nxt.shape[0], -1)).reshape(t, nxt.shape[1], nxt.shape[2])
    return cur


# ---------------------------------------------------------------------------
# Policies (readings; see module docstring)
# ---------------------------------------------------------------------------
def eps_from_residual(g, n, eps_rel) -> float:
    return max(eps_rel * float(g @ g) / float(min(n)), 1e-300)


def alpha_from_eps(eps, p, alpha_scale) -> float:
    """Theorem 4.1's form alpha_l = c * eps_l^{1/2} / p."""
    return alpha_scale * math.sqrt(eps) / p


# ---------------------------------------------------------------------------
# One iteration and the solver (Algorithm 2)
# ---------------------------------------------------------------------------
@dataclass
class StepInfo:
    eps: float
    alpha: float
    res_norm: float            # ||P_Omega(T_l - T*)||_F  (before the step)
    g: np.ndarray = field(repr=False, default=None)
    s: List[np.ndarray] = field(repr=False, default=None)


def prgd_step(cores, idx, y, n, r, eps_rel=1.0, alpha_scale=1.0, eps=None, alpha=None,
              keep=False, step="constant", metric="precond", retraction="plain"):
    """One PRGD iteration (Algorithm 2, Trim skipped):
    G_l = P_Omega(T_l - T*); G_{l,i}; W_l = T_l - alpha tilde P_T W^{-1} G_l
    (computed as W^{-1/2}(T^ - alpha P_{T^} W^{-1/2} G_l), Lemma 3.5);
    T_{l+1} = SVD^tt_r(W_l).
    Variants: step="adaptive" takes the steepest step of Eq. (PRGD
    stepsize) instead of Theorem 4.1's form; metric="uniform" sets every
    G_{l,i} = I, which makes the iteration RGD (Section 3.1), whose constant
    step is then alpha_scale / p (the limit of Theorem 4.1's form when
    G_{l,i} -> eps I); retraction="weighted" is Remark 3.6's
    W^{-1/2} SVD^tt_r W^{1/2}."""
    m = len(cores)
    N = idx.shape[0]
    p = N / float(np.prod(n))
    g = residual(cores, idx, y)
    if eps is None:
        eps = eps_from_residual(g, n, eps_rel)
    if metric == "uniform":
        G = [np.ones(n[k]) for k in range(m)]
    else:
        G = metric_diagonals(g, idx, n, eps)
    # W^{-1} G_l = W^{-1/2} (W^{-1/2} G_l): project W^{-1/2} G_l at T^ ...
    That = scale_cores(cores, G, 1.0 / (4 * m))
    U, _ = left_orthogonalize(That)
    ahat = g * weight_entries(idx, G, -1.0 / (4 * m))
    A = tangent_project_hat(U, idx, ahat)
    if alpha is None:
        if step == "adaptive":
            alpha = adaptive_step(U, A, G, idx)
        elif metric == "uniform":
            alpha = alpha_scale / p
        else:
            alpha = alpha_from_eps(eps, p, alpha_scale)
    C = assemble_2r(U, A, alpha, G)
    if retraction == "weighted":
        new = scale_cores(tt_round(scale_cores(C, G, 1.0 / (4 * m)), r), G, -1.0 / (4 * m))
    else:
        new = tt_round(C, r)
    info = StepInfo(eps, alpha, float(np.linalg.norm(g)))
    if keep:
        info.g = g
        info.s = [Gi - eps for Gi in G]
    return new, info


@dataclass
class SolveResult:
    cores: Cores
    iters: int
    converged: bool
    history: List[float]


def solve(cores, idx, y, n, r, truth=None, eps_rel=1.0, alpha_scale=1.0, max_iter=200,
          tol=1e-10, stop_rule="relerr", eps_mode="adaptive", **variants):
    """Iterate prgd_step.  stop_rule 'relerr': ||T-T*||/||T*|| <= tol (needs
    truth); 'step': ||T_{l+1}-T_l|| <= tol max(1, ||T_l||) (Section 5, noise
    experiment)."""
    cur = [np.array(c, dtype=np.float64) for c in cores]
    hist = []
    tnorm = tt_norm(truth) if truth is not None else None
    eps_fixed = None
    for it in range(1, max_iter + 1):
        kw = {}
        if eps_mode == "frozen":
            if eps_fixed is None:
                eps_fixed = eps_from_residual(residual(cur, idx, y), n, eps_rel)
            kw["eps"] = eps_fixed
        new, info = prgd_step(cur, idx, y, n, r, eps_rel=eps_rel, alpha_scale=alpha_scale, **kw, **variants)
        if stop_rule == "relerr":
            err = tt_dist(new, truth) / tnorm
        else:
            err = tt_dist(new, cur) / max(1.0, tt_norm(cur))
        hist.append(err)
        cur = new
        if err <= tol:
            return SolveResult(cur, it, True, hist)
    return SolveResult(cur, max_iter, False, hist)
