"""Seeded synthetic SDP instances shared by the CUDA path, the oracle and the bench.

This module only draws random data and writes down the problem data
(A, b, C) of each workload family; it contains none of the interior-point
or reformulation arithmetic.  Both the oracle and the CUDA path read the
identical arrays produced here.

Problem statement (Section 1, eq. sdp-pd): min <C,X> s.t. A(X) = b, X PSD,
with A given by one of three storage kinds:

* ``diag``   : A_i = e_i e_i^T, so A(X) = diag(X) (MaxCut, m = n).
* ``sparse`` : COO list of lower-triangle entries (con, row, col, val) with
               <A_i, X> = sum val * X[row, col] * (1 if row == col else 2).
* ``dense``  : m x n(n+1)/2 row-major matrix of svec(A_i) rows; svec is the
               column-by-column lower triangle with off-diagonal entries
               scaled by sqrt(2) (Notations, svec definition).

All matrices are float64 numpy arrays; symmetric n x n matrices are stored
full (row- and column-major agree).  Seeds follow ``1000 * family + instance``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

SQRT2 = math.sqrt(2.0)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Problem:
    """Standard-form SDP data (A, b, C) in one of the three storage kinds."""
    kind: str                      # "diag" | "sparse" | "dense"
    n: int
    m: int
    b: np.ndarray                  # (m,)
    C: np.ndarray                  # (n, n) symmetric
    a_con: Optional[np.ndarray] = None   # sparse: int32 (nnz,)
    a_row: Optional[np.ndarray] = None   # sparse: int32 (nnz,), row >= col
    a_col: Optional[np.ndarray] = None   # sparse: int32 (nnz,)
    a_val: Optional[np.ndarray] = None   # sparse: float64 (nnz,)
    a_dense: Optional[np.ndarray] = None  # dense: (m, n(n+1)/2) svec rows
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return 0 if self.a_val is None else int(self.a_val.shape[0])


def svec_len(n: int) -> int:
    return n * (n + 1) // 2


def _lower_svec_of_sym(M: np.ndarray) -> np.ndarray:
    """Pack a symmetric matrix into the svec layout (storage convention only)."""
    n = M.shape[0]
    out = np.empty(svec_len(n))
    k = 0
    for j in range(n):
        col = M[j:, j].copy()
        col[1:] *= SQRT2
        out[k:k + n - j] = col
        k += n - j
    return out


def _laplacian(n: int, edges: np.ndarray, w: np.ndarray) -> np.ndarray:
    L = np.zeros((n, n))
    for (i, j), wij in zip(edges, w):
        L[i, i] += wij
        L[j, j] += wij
        L[i, j] -= wij
        L[j, i] -= wij
    return L


def erdos_renyi_edges(n: int, p: float, g: np.random.Generator) -> np.ndarray:
    iu, ju = np.triu_indices(n, k=1)
    keep = g.random(iu.shape[0]) < p
    return np.stack([iu[keep], ju[keep]], axis=1)


def maxcut(n: int, p: float, seed: int, weights: str = "unit",
           edges: Optional[np.ndarray] = None) -> Problem:
    """MaxCut SDP: C = -(1/4) L(G), diag(X) = 1 (min form)."""
    g = rng(seed)
    if edges is None:
        edges = erdos_renyi_edges(n, p, g)
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    if weights == "unit":
        w = np.ones(edges.shape[0])
    elif weights == "gauss":
        w = g.standard_normal(edges.shape[0])
    else:
        raise ValueError(weights)
    L = _laplacian(n, edges, w)
    return Problem(kind="diag", n=n, m=n, b=np.ones(n), C=-0.25 * L,
                   meta={"family": "maxcut", "edges": edges, "weights": w})


def sensing(n: int, m: int, rank: int, seed: int) -> Problem:
    """Matrix sensing: A_i = (G_i + G_i^T)/2 with G_i iid N(0, 1/n); b = A(U U^T)."""
    g = rng(seed)
    N = svec_len(n)
    a = np.empty((m, N))
    il = np.tril_indices(n)
    # column-major lower triangle order == row-major upper triangle of the transpose
    order = np.lexsort((il[0], il[1]))
    rows, cols = il[0][order], il[1][order]
    scale = np.where(rows == cols, 1.0, SQRT2)
    for i in range(m):
        G = g.standard_normal((n, n)) / math.sqrt(n)
        A = 0.5 * (G + G.T)
        a[i] = A[rows, cols] * scale
    U = g.standard_normal((n, rank))
    Xs = U @ U.T
    b = a @ _lower_svec_of_sym(Xs)
    return Problem(kind="dense", n=n, m=m, b=b, C=np.eye(n), a_dense=a,
                   meta={"family": "sensing", "U": U})


def completion(n1: int, n2: int, rank: int, frac: float, seed: int) -> Problem:
    """Matrix completion in the symmetric embedding [[W1, X], [X^T, W2]].

    A_i = (e_a e_{n1+b}^T + e_{n1+b} e_a^T)/2 so <A_i, Z> = Z[a, n1+b] and
    b_i = M[a, b] with M = F1 F2^T; C = I (trace minimisation).
    """
    g = rng(seed)
    F1 = g.standard_normal((n1, rank))
    F2 = g.standard_normal((n2, rank))
    M = F1 @ F2.T
    m = int(round(frac * n1 * n2))
    flat = g.choice(n1 * n2, size=m, replace=False)
    flat.sort()
    a_idx, b_idx = flat // n2, flat % n2
    n = n1 + n2
    # lower-triangle storage: row = n1 + b > col = a, value 1/2 (entry counted twice)
    return Problem(kind="sparse", n=n, m=m, b=M[a_idx, b_idx].copy(), C=np.eye(n),
                   a_con=np.arange(m, dtype=np.int32),
                   a_row=(n1 + b_idx).astype(np.int32),
                   a_col=a_idx.astype(np.int32),
                   a_val=np.full(m, 0.5),
                   meta={"family": "completion", "F1": F1, "F2": F2, "n1": n1, "n2": n2})


def rmc(n: int, m: int, m_o: int, seed: int, rank: int = 2, lam: float = 1.0) -> Problem:
    """Robust matrix completion as Section 7 generates it (eq. rmc-sdp): X* = G G^T with G n x rank,
    entries N(0, 10^2); A(X) = m entries of svec(X) sampled without replacement (<A_i, X> =
    svec(X)_k: X_aa on the diagonal, sqrt2 X_ab off it); b = A(X*) + eps with m_o entries of eps
    drawn N(0, 10^4) and the rest zero; C = lam I.  The nonnegative variables x = [v; w] enter as
    A(X) + G_l x = b with G_l = [I, -I] and cost c_l = 1 (meta["G_l"], meta["c_l"])."""
    g = rng(seed)
    Gm = 10.0 * g.standard_normal((n, rank))
    Xs = Gm @ Gm.T
    N = svec_len(n)
    flat = np.sort(g.choice(N, size=m, replace=False))
    # svec position k -> (a, b), a >= b, column by column
    cols = np.repeat(np.arange(n), np.arange(n, 0, -1))
    starts = np.concatenate([[0], np.cumsum(np.arange(n, 0, -1))[:-1]])
    rows = np.arange(N) - starts[cols] + cols
    a_idx, b_idx = rows[flat], cols[flat]
    diag = a_idx == b_idx
    val = np.where(diag, 1.0, 1.0 / math.sqrt(2.0))        # <A_i, X> = sum val X_rc (1 or 2 for r != c)
    b = np.where(diag, Xs[a_idx, b_idx], math.sqrt(2.0) * Xs[a_idx, b_idx])
    eps = np.zeros(m)
    out = g.choice(m, size=min(m_o, m), replace=False)
    eps[out] = 100.0 * g.standard_normal(out.size)
    Gl = np.hstack([np.eye(m), -np.eye(m)])
    return Problem(kind="sparse", n=n, m=m, b=b + eps, C=lam * np.eye(n),
                   a_con=np.arange(m, dtype=np.int32), a_row=a_idx.astype(np.int32),
                   a_col=b_idx.astype(np.int32), a_val=val,
                   meta={"family": "rmc", "Xs": Xs, "outliers": out, "eps": eps, "G_l": Gl,
                         "c_l": np.ones(2 * m)})


def random_sparse(n: int, m: int, per_con: int, seed: int) -> Problem:
    """Generic sparse constraints (several lower-triangle entries per A_i) for tests."""
    g = rng(seed)
    con, row, col, val = [], [], [], []
    for i in range(m):
        for _ in range(per_con):
            a, bb = sorted(g.integers(0, n, size=2))[::-1]
            con.append(i); row.append(a); col.append(bb); val.append(g.standard_normal())
    X0 = np.eye(n)
    p = Problem(kind="sparse", n=n, m=m, b=np.zeros(m), C=np.eye(n),
                a_con=np.asarray(con, np.int32), a_row=np.asarray(row, np.int32),
                a_col=np.asarray(col, np.int32), a_val=np.asarray(val, np.float64),
                meta={"family": "random_sparse"})
    # b = A(I): the identity is strictly feasible
    diag_hits = p.a_row == p.a_col
    bvec = np.zeros(m)
    np.add.at(bvec, p.a_con[diag_hits], p.a_val[diag_hits] * X0[p.a_row[diag_hits], p.a_col[diag_hits]])
    p.b = bvec
    return p


@dataclass
class ScalingPoint:
    """Eigen-decomposition of a synthetic NT scaling point W = V diag(lam) V^T."""
    V: np.ndarray      # (n, n) orthonormal columns
    lam: np.ndarray    # (n,) positive, in random order unless sorted=True
    mu: float


def scaling_point(n: int, r_true: int, mu: float, seed: int, sorted_desc: bool = False,
                  V_top: Optional[np.ndarray] = None) -> ScalingPoint:
    """Scaling point with the two-cluster spectrum of assumption (A0) / Lemma eigsplit.

    The top r_true eigenvalues are U(1,3)/sqrt(mu), the other n - r_true are
    U(0.5,2)*sqrt(mu).  V is Haar-random (QR of a Gaussian, sign-fixed); if
    V_top is given its columns are orthonormalised into the leading block.
    """
    g = rng(seed)
    G = g.standard_normal((n, n))
    if V_top is not None:
        G[:, :V_top.shape[1]] = V_top
    Qm, R = np.linalg.qr(G)
    Qm = Qm * np.sign(np.diag(R))[None, :]
    top = g.uniform(1.0, 3.0, size=r_true) / math.sqrt(mu)
    bot = g.uniform(0.5, 2.0, size=n - r_true) * math.sqrt(mu)
    lam = np.concatenate([top, bot])
    if not sorted_desc:
        perm = g.permutation(n)
        lam = lam[perm]
        Qm = Qm[:, perm]
    else:
        order = np.argsort(-lam, kind="stable")
        lam, Qm = lam[order], Qm[:, order]
    return ScalingPoint(V=np.ascontiguousarray(Qm), lam=lam, mu=mu)


def newton_rhs(n: int, m: int, seed: int, scale: float = 1.0):
    """Random residuals (C~, b~) of the Newton subproblem (eq. newt)."""
    g = rng(seed)
    G = g.standard_normal((n, n)) * scale
    Ct = 0.5 * (G + G.T)
    bt = g.standard_normal(m) * scale
    return Ct, bt


# ---------------------------------------------------------------------------
# Named workloads (shapes and distributions of the five benchmark families)

def batch_specs(count: int = 256, seed: int = 5) -> list:
    """The batched workload: ``count`` independent SDPs, the first half MaxCut (n ~ U{32..512},
    G(n, 0.05), unit weights, diag constraints), the second half matrix sensing (n ~ U{32..256},
    m = 10 n dense constraints, planted rank 2, C = I).  Returns (family, n, instance seed)."""
    g = rng(1000 * seed)
    half = count // 2
    specs = [("maxcut", int(g.integers(32, 513)), 1000 * seed + 1 + i) for i in range(half)]
    specs += [("sensing", int(g.integers(32, 257)), 1000 * seed + 1 + half + i) for i in range(count - half)]
    return specs


def batch_problem(spec) -> Problem:
    """One instance of ``batch_specs`` on the host (numpy)."""
    fam, n, seed = spec
    if fam == "maxcut":
        return maxcut(n, 0.05, seed)
    return sensing(n, 10 * n, 2, seed)


def sensing_device(n: int, m: int, rank: int, seed: int, device):
    """Matrix sensing drawn on the GPU (torch generator seeded with ``seed``) for the large
    batched workload: svec(A_i) for A_i = (G_i + G_i^T)/2, G_i iid N(0, 1/n) has iid N(0, 1/n)
    coordinates (diagonal: N(0, 1/n); off-diagonal: sqrt2 N(0, 1/(2n))), so the svec rows are
    drawn directly; b = A(U U^T).  Same distribution as ``sensing``, a different stream of
    numbers.  Returns a Problem whose arrays are torch tensors on ``device``."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    N = svec_len(n)
    a = torch.randn((m, N), generator=gen, device=device, dtype=torch.float64) / math.sqrt(n)
    U = torch.randn((n, rank), generator=gen, device=device, dtype=torch.float64)
    il = np.tril_indices(n)
    order = np.lexsort((il[0], il[1]))
    rows = torch.from_numpy(il[0][order]).to(device)
    cols = torch.from_numpy(il[1][order]).to(device)
    Xs = U @ U.T
    sv = Xs[rows, cols] * torch.where(rows == cols, 1.0, SQRT2).to(torch.float64)
    b = a @ sv
    C = torch.eye(n, dtype=torch.float64, device=device)
    return Problem(kind="dense", n=n, m=m, b=b, C=C, a_dense=a, meta={"family": "sensing", "U": U})


def workload(name: str, instance: int = 0) -> Problem:
    if name == "maxcut64":
        return maxcut(64, 0.1, seed=1000 * 1 + instance)
    if name == "sensing200":
        return sensing(200, 2000, 3, seed=1000 * 2 + instance)
    if name == "maxcut5000":
        return maxcut(5000, 8.0 / 4999.0, seed=1000 * 3 + instance, weights="gauss")
    if name == "completion2000":
        return completion(1000, 1000, 5, 0.05, seed=1000 * 4 + instance)
    raise KeyError(name)
