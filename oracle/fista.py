"""FP64 restatement of the paper's model and algorithms (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
module.  It shares no code with the CUDA library.

Paper references (arXiv 2506.04045):
  * model (P): f(X) = sum_ij (s_ij - x_i^T x_j)^2 = ||S - X^T X||_F^2 over
    Omega = simplex^N (Sect. 2, Eq. "constraint" and problem (P));
  * projection onto Omega column by column, each by the Duchi algorithm
    (Sect. 2, Algorithm 1);
  * gradient, matrix form  grad f(X) = -4 X (S - X^T X)  (Eq. "gradient_matrix")
    and column form  col_i grad f = -4 (X s_i - X X^T x_i)  (Eq. "gradient_column");
  * Lipschitz constant L = 4 ||S||_2 + 12 N (Theorem 2.1 proof), with ||S||_F
    in place of ||S||_2 in the experiments (Sect. 5, "Hyperparameters");
  * loss by the trace identity
    f = ||S||_F^2 + ||X X^T||_F^2 - 2 sum_i <x_i, X s_i>  (Sect. 3, "Loss Update");
  * parallel GPA with loss update (Algorithm 3) and parallel FISTA
    (Algorithm 4), the latter with the stopping test as the prose after it
    states it (stop once f(Xbar^{n-1}) - f(Xbar^n) <= tol);
  * Hessian operator (Theorem 4.1, Eq. "hessian").

In U = X^T notation (rows on the simplex) the gradient reads
-4 (S U - U U^T U) and the GPA step is U <- P_Omega(U - tau * grad).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# ----------------------------------------------------------------------------
# basic quantities
# ----------------------------------------------------------------------------
def _as_csr(S) -> sp.csr_matrix:
    if sp.issparse(S):
        return sp.csr_matrix(S, dtype=np.float64)
    return sp.csr_matrix(np.asarray(S, dtype=np.float64))


def frob2(S) -> float:
    """||S||_F^2 = sum of squared entries."""
    if sp.issparse(S):
        d = S.data.astype(np.float64)
        return float(np.dot(d, d))
    A = np.asarray(S, dtype=np.float64)
    return float(np.sum(A * A))


def objective_dense(S, U) -> float:
    """f = sum_i sum_j (s_ij - sum_c u_ic u_jc)^2, the definition in Sect. 2
    written out with the dense N x N predicted similarity Y = U U^T."""
    Sd = S.toarray() if sp.issparse(S) else np.asarray(S, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64)
    Y = U @ U.T
    D = Sd - Y
    return float(np.sum(D * D))


def objective_trace(S, U) -> float:
    """f = ||S||_F^2 + ||U^T U||_F^2 - 2 sum_i <u_i, (S U)_i> (Sect. 3, "Loss
    Update": share = X X^T is C x C, prod_i = <x_i, X s_i>, merge = sum)."""
    S = _as_csr(S)
    U = np.asarray(U, dtype=np.float64)
    share = U.T @ U
    SU = S @ U
    merge = float(np.sum(U * SU))
    return frob2(S) + float(np.sum(share * share)) - 2.0 * merge


def loss_terms(S, U) -> dict:
    """The pieces of the loss update (Sect. 3): ||S||_F^2, ||share||_F^2 with
    share = U^T U, merge = sum_i <u_i, (S U)_i>, and f = ||S||_F^2 +
    ||share||_F^2 - 2 merge."""
    S = _as_csr(S)
    U = np.asarray(U, dtype=np.float64)
    share = U.T @ U
    merge = float(np.sum(U * (S @ U)))
    s2 = frob2(S)
    g2 = float(np.sum(share * share))
    return {"frob2": s2, "gram_fro2": g2, "trace": merge, "f": s2 + g2 - 2.0 * merge}


def gradient_matrix(S, U) -> np.ndarray:
    """grad f in U notation: -4 (S - U U^T) U, the transpose of the paper's
    -4 X (S - X^T X) (Eq. "gradient_matrix"; S symmetric).  Forms U U^T
    explicitly, so it is meant for small N."""
    Sd = S.toarray() if sp.issparse(S) else np.asarray(S, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64)
    return -4.0 * (Sd - U @ U.T) @ U


def gradient_columns(S, U) -> np.ndarray:
    """grad f column by column, Eq. "gradient_column": column i of grad f is
    -4 (X s_i - share x_i) with share = X X^T.  Row i of the result is that
    column, computed one i at a time."""
    S = _as_csr(S)
    U = np.asarray(U, dtype=np.float64)
    share = U.T @ U
    n = U.shape[0]
    out = np.empty_like(U)
    for i in range(n):
        lo, hi = S.indptr[i], S.indptr[i + 1]
        Xs_i = S.data[lo:hi] @ U[S.indices[lo:hi]]      # X s_i (S symmetric: row i = column i)
        out[i] = -4.0 * (Xs_i - share @ U[i])
    return out


def hessian_apply(S, U, V) -> np.ndarray:
    """Hessian operator of Theorem 4.1 (Eq. "hessian") in U notation.

    The paper maps V (C x N) to -4 V (S - Xb^T Xb) + 4 Xb (V^T Xb + Xb^T V).
    Transposing with U = Xb^T and W = V^T gives
    -4 (S - U U^T) W + 4 (W U^T + U W^T) U, evaluated here with dense N x N
    matrices (small N)."""
    Sd = S.toarray() if sp.issparse(S) else np.asarray(S, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64)
    W = np.asarray(V, dtype=np.float64)
    return -4.0 * (Sd - U @ U.T) @ W + 4.0 * (W @ U.T + U @ W.T) @ U


def hessian_apply_sparse(S, U, W) -> np.ndarray:
    """The same operator as hessian_apply without forming N x N matrices:
    (U U^T) W = U (U^T W), (W U^T) U = W (U^T U), (U W^T) U = U (W^T U), so
    H[W] = -4 S W + 4 U (U^T W) + 4 W (U^T U) + 4 U (W^T U); S stays sparse."""
    S = _as_csr(S)
    U = np.asarray(U, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    return -4.0 * (S @ W) + 4.0 * U @ (U.T @ W) + 4.0 * W @ (U.T @ U) + 4.0 * U @ (W.T @ U)


def curvature(S, U, W) -> float:
    """<W, H[W]> (Theorem 4.1): negative along a tangent direction at a
    stationary point means the point is not a local minimum (Sect. 4)."""
    return float(np.sum(np.asarray(W, dtype=np.float64) * hessian_apply_sparse(S, U, W)))


def slope(S, U, W) -> float:
    """Directional derivative <grad f(U), W>, gradient in the column form of
    Eq. "gradient_column" (sparse S)."""
    return float(np.sum(np.asarray(W, dtype=np.float64) * gradient_columns(S, U)))


# ----------------------------------------------------------------------------
# projection onto the simplex (Algorithm 1) and onto Omega
# ----------------------------------------------------------------------------
def duchi(x) -> np.ndarray:
    """Projection of one vector onto the unit simplex, Algorithm 1 step by step:
    sort descending, cumulative sums S_k, the largest k with
    x_(k) - (S_k - 1)/k >= 0, threshold (S_k - 1)/k, then max(x - threshold, 0)."""
    x = np.asarray(x, dtype=np.float64)
    C = x.shape[0]
    xs = np.sort(x)[::-1]
    Sk = np.cumsum(xs)
    ks = np.arange(1, C + 1, dtype=np.float64)
    ok = xs - (Sk - 1.0) / ks >= 0.0
    k = int(np.nonzero(ok)[0][-1]) + 1
    thr = (Sk[k - 1] - 1.0) / k
    return np.maximum(x - thr, 0.0)


def project_omega(V) -> np.ndarray:
    """P_Omega: the projection splits into one simplex projection per article
    (Sect. 2, "Projection onto Omega"); each row of V is projected by Algorithm 1."""
    V = np.asarray(V, dtype=np.float64)
    n, C = V.shape
    xs = -np.sort(-V, axis=1)
    Sk = np.cumsum(xs, axis=1)
    ks = np.arange(1, C + 1, dtype=np.float64)[None, :]
    ok = xs - (Sk - 1.0) / ks >= 0.0
    # largest k per row with the condition true (column 0 always qualifies)
    last = C - 1 - np.argmax(ok[:, ::-1], axis=1)
    thr = (Sk[np.arange(n), last] - 1.0) / (last + 1.0)
    return np.maximum(V - thr[:, None], 0.0)


# ----------------------------------------------------------------------------
# step size
# ----------------------------------------------------------------------------
def spectral_norm(S) -> float:
    """||S||_2, the largest singular value (dense eigensolver for small N,
    Lanczos otherwise; S symmetric)."""
    S = _as_csr(S)
    n = S.shape[0]
    if n <= 2000:
        ev = np.linalg.eigvalsh(S.toarray())
        return float(np.max(np.abs(ev)))
    vals = spla.eigsh(S, k=1, which="LM", return_eigenvectors=False, tol=1e-10)
    return float(abs(vals[0]))


def lipschitz(S, rule: str = "frobenius") -> float:
    """L = 4 ||S|| + 12 N.  Theorem 2.1 uses the spectral norm; the experiments
    replace it by the Frobenius norm (Sect. 5, "Hyperparameters")."""
    S = _as_csr(S)
    n = S.shape[0]
    if rule == "frobenius":
        nrm = math.sqrt(frob2(S))
    elif rule == "spectral":
        nrm = spectral_norm(S)
    else:
        raise ValueError(rule)
    return 4.0 * nrm + 12.0 * n


# ----------------------------------------------------------------------------
# Algorithms 3 and 4
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class OracleResult:
    U: np.ndarray                  # output membership matrix (N x C, rows on the simplex)
    iters: int                     # gradient evaluations performed
    stopped: bool                  # True if the loss test ended the run
    losses: list                   # losses evaluated in order (loss^0, loss^1, ...)
    pg_norms: list                 # ||Y^n - Xbar^n||_F / tau per iteration
    history: list = dataclasses.field(default_factory=list)   # iterates, if requested
    t_values: list = dataclasses.field(default_factory=list)  # FISTA: t_1, t_2, ... as used


def gpa(S, U0, tau: float, tol: float = 0.0, max_iter: int = 100,
        stop: str = "loss", keep_history: bool = False) -> OracleResult:
    """Parallel GPA with loss update, Algorithm 3.

    loss^{-1} = N^2.  For n = 0, 1, ...: share = X X^T, merge = sum_i <X s_i, x_i>,
    loss^n = ||S||_F^2 + ||share||_F^2 - 2 merge; if loss^{n-1} - loss^n <= tol
    the output is X^n; otherwise every column takes a gradient step followed
    by Algorithm 1.  ``max_iter`` bounds the number of gradient steps; if it is
    reached the last iterate X^{max_iter} is returned.  ``stop`` = "none"
    disables the loss test (fixed iteration count)."""
    S = _as_csr(S)
    n = S.shape[0]
    X = np.array(U0, dtype=np.float64)
    S2 = frob2(S)
    loss_prev = float(n) ** 2
    losses, pgs, hist = [], [], []
    for it in range(max_iter + 1):
        share = X.T @ X
        SX = S @ X
        merge = float(np.sum(SX * X))
        loss = S2 + float(np.sum(share * share)) - 2.0 * merge
        losses.append(loss)
        if stop == "loss" and loss_prev - loss <= tol:
            return OracleResult(X, it, True, losses, pgs, hist)
        if it == max_iter:
            break
        grad = -4.0 * (SX - X @ share)
        Xn = project_omega(X - tau * grad)
        pgs.append(float(np.linalg.norm(X - Xn)) / tau)
        X = Xn
        if keep_history:
            hist.append(X.copy())
        loss_prev = loss
    return OracleResult(X, max_iter, False, losses, pgs, hist)


def fista(S, U0, tau: float, tol: float = 0.0, max_iter: int = 100,
          stop: str = "loss", accel: bool = True, pg_tol: float = 0.0,
          keep_history: bool = False) -> OracleResult:
    """Parallel FISTA, Algorithm 4, literally: two products with S per iteration.

    Xbar^0 = U0, X^1 = Xbar^0, loss^0 = f(Xbar^0), t_1 = 1.  Iteration n:
      share^n = X^n X^n^T; grad_i = -4 (X^n s_i - share^n x_i^n);
      xbar_i^n = P_simplex(x_i^n - tau grad_i)                 (basic GPA)
      sharebar^n = Xbar^n Xbar^n^T; prodbar_i = <Xbar^n s_i, xbar_i^n>;
      lossbar^n = ||S||_F^2 + ||sharebar^n||_F^2 - 2 sum_i prodbar_i;
      stop if lossbar^{n-1} - lossbar^n <= tol  (the prose's sign; the listing
        prints the difference the other way round, which stops every
        decreasing run at n = 1) and output Xbar^n;
      t_{n+1} = (1 + sqrt(1 + 4 t_n^2)) / 2;
      X^{n+1} = Xbar^n + ((t_n - 1)/t_{n+1}) (Xbar^n - Xbar^{n-1}).
    ``accel`` = False keeps the momentum factor at zero (plain projected
    gradient).  ``stop``: "loss" (the paper's rule), "pg_rel" (stop when
    ||X^n - Xbar^n||_F / tau <= pg_tol times its first value), "pg_abs", or
    "none" (run ``max_iter`` iterations)."""
    S = _as_csr(S)
    Xbar_prev = np.array(U0, dtype=np.float64)
    S2 = frob2(S)

    def loss_of(Z):
        share = Z.T @ Z
        return S2 + float(np.sum(share * share)) - 2.0 * float(np.sum((S @ Z) * Z))

    X = Xbar_prev.copy()
    loss_prev = loss_of(Xbar_prev)
    losses, pgs, hist = [loss_prev], [], []
    t = 1.0
    ts = [t]
    pg_first = None
    for it in range(1, max_iter + 1):
        share = X.T @ X
        grad = -4.0 * (S @ X - X @ share)
        Xbar = project_omega(X - tau * grad)
        pg = float(np.linalg.norm(X - Xbar)) / tau
        pgs.append(pg)
        if pg_first is None:
            pg_first = pg
        if keep_history:
            hist.append(Xbar.copy())
        loss = loss_of(Xbar)
        losses.append(loss)
        if stop == "loss" and loss_prev - loss <= tol:
            return OracleResult(Xbar, it, True, losses, pgs, hist, ts)
        if stop == "pg_rel" and pg <= pg_tol * pg_first:
            return OracleResult(Xbar, it, True, losses, pgs, hist, ts)
        if stop == "pg_abs" and pg <= pg_tol:
            return OracleResult(Xbar, it, True, losses, pgs, hist, ts)
        t_next = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        beta = (t - 1.0) / t_next if accel else 0.0
        X = Xbar + beta * (Xbar - Xbar_prev)
        Xbar_prev = Xbar
        loss_prev = loss
        t = t_next
        ts.append(t)
    return OracleResult(Xbar_prev, max_iter, False, losses, pgs, hist, ts)


def momentum_factors(n_iter: int, accel: bool = True) -> list:
    """beta_n = (t_{n-1} - 1) / t_n for n = 1..n_iter with t_1 = 1 and
    t_{n+1} = (1 + sqrt(1 + 4 t_n^2)) / 2 (Algorithm 4); X^n = Xbar^{n-1} +
    beta_n (Xbar^{n-1} - Xbar^{n-2}), beta_1 = 0 since X^1 = Xbar^0."""
    out = [0.0]
    t = 1.0
    for _ in range(1, n_iter):
        t_next = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        out.append((t - 1.0) / t_next if accel else 0.0)
        t = t_next
    return out


def gram_blocks(blocks, beta=None) -> np.ndarray:
    """share = X^T X (Sect. 3; C x C with the paper's X) summed over row blocks
    of X in float64, for iterates too large to hold whole: ``blocks`` yields
    arrays of consecutive rows (any float dtype).  With ``beta`` each block is
    a pair (rows of Xbar^n, the same rows of Xbar^{n-1}) and the rows of the
    extrapolated point X^{n+1} = Xbar^n + beta (Xbar^n - Xbar^{n-1}) of
    Algorithm 4 are summed."""
    share = None
    for B in blocks:
        if beta is not None:
            Bc = np.asarray(B[0], dtype=np.float64)
            Bp = np.asarray(B[1], dtype=np.float64)
            B = Bc + beta * (Bc - Bp)
        B = np.asarray(B, dtype=np.float64)
        g = B.T @ B
        share = g if share is None else share + g
    return share


def fista_step_rows(S, Xbar_cur, Xbar_prev, beta: float, tau: float, rows, share=None) -> np.ndarray:
    """One iteration of Algorithm 4 evaluated only at the given articles.

    X = Xbar_cur + beta (Xbar_cur - Xbar_prev) (the extrapolated point),
    share = X^T X over all articles, then for each requested i:
    grad_i = -4 (X s_i - share x_i) and xbar_i = Algorithm 1 applied to
    x_i - tau grad_i.  Returns the rows of the next Xbar (float64).  When the
    arrays in hand hold only some articles (the requested rows and their
    neighbours in S), ``share`` must be given: X^T X over all articles of the
    extrapolated point (gram_blocks)."""
    S = _as_csr(S)
    Xc = np.asarray(Xbar_cur, dtype=np.float64)
    Xp = np.asarray(Xbar_prev, dtype=np.float64)
    X = Xc + beta * (Xc - Xp)
    if share is None:
        share = X.T @ X
    out = np.empty((len(rows), X.shape[1]))
    for r, i in enumerate(rows):
        lo, hi = S.indptr[i], S.indptr[i + 1]
        Xs_i = S.data[lo:hi] @ X[S.indices[lo:hi]]
        grad = -4.0 * (Xs_i - share @ X[i])
        out[r] = duchi(X[i] - tau * grad)
    return out


# ----------------------------------------------------------------------------
# similarity matrix from an edge list
# ----------------------------------------------------------------------------
def csr_from_edges(n: int, src, dst, w=None, add_unit_diag: bool = True):
    """Symmetric similarity matrix from an edge list, in CSR with sorted columns.

    s_ij = s_ji = w_e for each edge e = (i, j): article i cites or is cited by
    article j (Example 4.1).  Repeated pairs keep the largest weight.  With
    ``add_unit_diag`` the diagonal is 1 (Example 4.1, Sect. 5) and self-loop
    edges are ignored; without it self-loops keep their (largest) weight.
    Returns (row_ptr int64, col int32, val float32) as numpy arrays.  Raises
    ValueError on an endpoint outside [0, n)."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    if w is None:
        w = np.ones(src.shape[0], dtype=np.float32)
    w = np.asarray(w, dtype=np.float32)
    if src.size and (src.min() < 0 or dst.min() < 0 or src.max() >= n or dst.max() >= n):
        raise ValueError("edge endpoint out of range")
    if add_unit_diag:
        keep = src != dst
        src, dst, w = src[keep], dst[keep], w[keep]
    rows = np.concatenate([src, dst])
    cols = np.concatenate([dst, src])
    vals = np.concatenate([w, w])
    if add_unit_diag:
        d = np.arange(n, dtype=np.int64)
        rows = np.concatenate([rows, d])
        cols = np.concatenate([cols, d])
        vals = np.concatenate([vals, np.ones(n, dtype=np.float32)])
    keys = rows * n + cols
    order = np.argsort(keys, kind="stable")
    keys, vals = keys[order], vals[order]
    if keys.size:
        starts = np.concatenate([[0], np.nonzero(np.diff(keys))[0] + 1])
        ukeys = keys[starts]
        uvals = np.maximum.reduceat(vals, starts)
    else:
        ukeys = keys
        uvals = vals
    r = ukeys // n if n else ukeys
    c = ukeys % n if n else ukeys
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, r + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return row_ptr, c.astype(np.int32), uvals.astype(np.float32)
