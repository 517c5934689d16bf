"""Oracle for the graph operators of Sec. 3.1 and Sec. 4 (FP64, CPU).  Test infrastructure.

Definitions followed, in the paper's notation:
  L = D - W, D_ii = sum_j W_ij                                     (Sec. 3.1)
  T_i: nodes j reachable from i in two hops with (i, j) not an edge  (Sec. 4.1.1)
  Theta_i (Eq. 5) and Q = sum_i Theta_i                             (Sec. 4.1.1)
  A = L - mu Q + eps I                                              (Eq. 6)
  eps = lambda_2(Q), the Fiedler value of Q                         (Sec. 4.2)
  mu_i = eps / (Q_ii - sum_{j != i} Q_ij), mu = min_i mu_i          (Eq. 7-9)
  r_i = sum_{j != i} |A_ij|, b_i = r_i / (prod_j r_j)^(1/N)         (Sec. 4.3)

Readings of passages the paper leaves garbled or open:
  * Theta_i's (i, i) entry.  Eq. 5 prints 1/T_i.  The aggregate distance it is meant to
    express, and the statement that Q is a Laplacian with lambda_1(Q) = 0, need the
    star Laplacian scaled by 1/T_i, whose (i, i) entry is T_i * (1/T_i) = 1.  That
    "laplacian" reading is the default; the printed entry is kept as reading="literal"
    for documentation (it makes Q indefinite on the odd ring).
  * "Second smallest eigenvalue" counts multiplicity: if the two-hop graph (nodes, T)
    has more than one connected component (including nodes with T_i = 0), then
    eps = 0, and the result is flagged degenerate.
  * Rows whose mu_i denominator is not positive (T_i = 0) are left out of the minimum;
    mu = 0 if no row remains or eps = 0.
  * The regulariser "+ eps I" is the matrix eps * I inside A (Eq. 6), not a scalar.
  * The geometric mean in b_i is taken as exp(mean(log r)) (a product of N radii
    overflows); an isolated node (r_i = 0) makes B singular and is an error.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

DENSE_MAX = 3000  # above this, eps comes from the oracle's LOBPCG instead of dense eigh


@dataclass
class GraphOps:
    n: int
    T: np.ndarray            # int32[n], |T_i|
    t_ptr: np.ndarray        # int64[n+1] two-hop sets, CSR
    t_col: np.ndarray        # int32, ascending per row
    L: sp.csr_matrix
    Q: sp.csr_matrix
    eps: float
    mu: float
    A: sp.csr_matrix         # values on the canonical structure below
    a_ptr: np.ndarray        # int64[n+1]  structure of A = diag + E + T, ascending columns
    a_col: np.ndarray        # int32
    a_val: np.ndarray        # float64, aligned with a_col
    r: np.ndarray            # Gershgorin radii of A
    b: np.ndarray            # diagonal of B
    degenerate: bool         # eps forced to 0 (two-hop graph disconnected)
    info: dict = field(default_factory=dict)


def pattern(n, row_ptr, col) -> sp.csr_matrix:
    """0/1 adjacency pattern S of the input graph (no diagonal)."""
    data = np.ones(col.shape[0], dtype=np.int64)
    return sp.csr_matrix((data, col.astype(np.int64), row_ptr.astype(np.int64)), shape=(n, n))


def two_hop_sets(n, row_ptr, col):
    """T_i = {j : (S^2)_ij > 0, j != i, S_ij = 0}, i.e. reachable in two hops, not adjacent.

    Returns (t_ptr int64[n+1], t_col int32 ascending per row, T int32[n]).
    """
    S = pattern(n, row_ptr, col)
    S2 = (S @ S).tocsr()
    S2.setdiag(0)
    S2.eliminate_zeros()
    S2 = S2 - S2.multiply(S)     # remove 1-hop neighbours
    S2.eliminate_zeros()
    S2.sort_indices()
    t_ptr = S2.indptr.astype(np.int64)
    t_col = S2.indices.astype(np.int32)
    T = np.diff(t_ptr).astype(np.int32)
    return t_ptr, t_col, T


def laplacian(n, row_ptr, col, w) -> sp.csr_matrix:
    """L = D - W (Sec. 3.1)."""
    W = sp.csr_matrix((w.astype(np.float64), col.astype(np.int64), row_ptr.astype(np.int64)),
                      shape=(n, n))
    D = np.asarray(W.sum(axis=1)).ravel()
    return (sp.diags(D) - W).tocsr()


def q_matrix(n, t_ptr, t_col, reading: str = "laplacian") -> sp.csr_matrix:
    """Q = sum_i Theta_i with Theta_i from Eq. 5.

    For node i with T_i > 0 and each j in T_i, Theta_i holds 1/T_i at (j, j),
    -1/T_i at (i, j) and (j, i); its (i, i) entry is 1 under the Laplacian reading
    (T_i copies of 1/T_i) and 1/T_i under the literal reading.
    """
    if reading not in ("laplacian", "literal"):
        raise ValueError(reading)
    T = np.diff(t_ptr)
    rows, cols, vals = [], [], []
    for i in range(n):
        Ti = int(T[i])
        if Ti == 0:
            continue
        inv = 1.0 / Ti
        js = t_col[t_ptr[i]:t_ptr[i + 1]].astype(np.int64)
        if reading == "laplacian":
            rows.append(np.full(Ti, i)); cols.append(np.full(Ti, i)); vals.append(np.full(Ti, inv))
        else:
            rows.append(np.array([i])); cols.append(np.array([i])); vals.append(np.array([inv]))
        rows.append(js); cols.append(js); vals.append(np.full(Ti, inv))
        rows.append(np.full(Ti, i)); cols.append(js); vals.append(np.full(Ti, -inv))
        rows.append(js); cols.append(np.full(Ti, i)); vals.append(np.full(Ti, -inv))
    if not rows:
        return sp.csr_matrix((n, n))
    r = np.concatenate(rows); c = np.concatenate(cols); v = np.concatenate(vals)
    Q = sp.coo_matrix((v, (r, c)), shape=(n, n)).tocsr()
    Q.sum_duplicates()
    Q.sort_indices()
    return Q


def two_hop_components(n, t_ptr, t_col) -> int:
    """Connected components of the graph (V, {(i, j) : j in T_i})."""
    G = sp.csr_matrix((np.ones(t_col.shape[0]), t_col.astype(np.int64), t_ptr.astype(np.int64)),
                      shape=(n, n))
    ncomp, _ = connected_components(G, directed=False)
    return int(ncomp)


def fiedler_value(Q: sp.csr_matrix, n_components: int, tol: float = 1e-12, seed: int = 0):
    """eps = lambda_2(Q), counted with multiplicity (0 when the two-hop graph is disconnected).

    Dense symmetric eigendecomposition for small N; otherwise the oracle's LOBPCG on
    (Q, I) with the constant vector as a constraint.
    """
    n = Q.shape[0]
    if n < 2 or n_components > 1:
        return 0.0
    if n <= DENSE_MAX:
        ev = np.linalg.eigvalsh(Q.toarray())
        return float(ev[1])
    from .eigen import lobpcg
    Y = np.ones((n, 1)) / np.sqrt(n)
    res = lobpcg(Q, np.ones(n), 1, guard=3, Y=Y, tol=tol, seed=seed, maxiter=100000)
    return float(res.lam[0])


def fiedler_value_sparse(Q: sp.csr_matrix, n_components: int) -> tuple[float, float]:
    """eps = lambda_2(Q) for large N without an iteration tolerance of the oracle's own.

    The two smallest eigenvalues of the Laplacian Q by ARPACK's shift-invert Lanczos
    (scipy ``eigsh`` on Q - sigma I with sigma just below 0, a library step at machine
    precision).  Returns (eps, residual) where residual = ||Q v - eps v|| / ||Q||_G for the
    returned unit vector v, so a caller can check the value actually converged.
    """
    import scipy.sparse.linalg as spla
    n = Q.shape[0]
    if n < 2 or n_components > 1:
        return 0.0, 0.0
    Q = sp.csr_matrix(Q)
    absrow = np.asarray(abs(Q).sum(axis=1)).ravel()
    qn = float(np.max(absrow))
    lam, U = spla.eigsh(Q.tocsc(), k=2, sigma=-1e-9 * qn, which="LM", tol=0.0,
                        v0=np.linspace(1.0, 2.0, n))
    j = int(np.argsort(lam)[1])
    v = U[:, j] / np.linalg.norm(U[:, j])
    res = float(np.linalg.norm(Q @ v - lam[j] * v)) / qn
    return float(lam[j]), res


def mu_value(Q: sp.csr_matrix, eps: float) -> float:
    """Eq. 9: mu_i = eps / (Q_ii - sum_{j != i} Q_ij), mu = min over rows with a positive denominator."""
    if eps == 0.0:
        return 0.0
    Qd = Q.diagonal()
    rowsum = np.asarray(Q.sum(axis=1)).ravel()
    off = rowsum - Qd                 # sum_{j != i} Q_ij
    den = Qd - off
    pos = den > 0
    if not np.any(pos):
        return 0.0
    return float(np.min(eps / den[pos]))


def a_structure(n, row_ptr, col, t_ptr, t_col):
    """Canonical structure of A: diagonal, 1-hop and two-hop entries, ascending columns."""
    I = sp.identity(n, format="csr", dtype=np.int64)
    S = pattern(n, row_ptr, col)
    Tm = sp.csr_matrix((np.ones(t_col.shape[0], dtype=np.int64), t_col.astype(np.int64),
                        t_ptr.astype(np.int64)), shape=(n, n))
    P = (I + S + Tm).tocsr()
    P.sum_duplicates()
    P.sort_indices()
    return P.indptr.astype(np.int64), P.indices.astype(np.int32)


def gershgorin_radii(a_ptr, a_col, a_val) -> np.ndarray:
    """r_i = sum_{j != i} |A_ij| (Sec. 3.2)."""
    n = a_ptr.shape[0] - 1
    rows = np.repeat(np.arange(n), np.diff(a_ptr))
    off = rows != a_col
    return np.bincount(rows[off], weights=np.abs(a_val[off]), minlength=n)


def b_vector(r: np.ndarray) -> np.ndarray:
    """b_i = r_i / (prod_j r_j)^(1/N) (Sec. 4.3), geometric mean through logs."""
    if np.any(r <= 0):
        raise ValueError("isolated node: a Gershgorin radius is zero, B is not positive definite")
    g = np.exp(np.mean(np.log(r)))
    return r / g


def build_graph_ops(n, row_ptr, col, w, *, reading="laplacian", eps_override=None,
                    mu_override=None, eps_tol=1e-12, seed=0) -> GraphOps:
    """The whole operator build of Sec. 4 for one input graph."""
    t_ptr, t_col, T = two_hop_sets(n, row_ptr, col)
    L = laplacian(n, row_ptr, col, w)
    Q = q_matrix(n, t_ptr, t_col, reading)
    ncomp = two_hop_components(n, t_ptr, t_col)
    degenerate = False
    if eps_override is not None:
        eps = float(eps_override)
    else:
        eps = fiedler_value(Q, ncomp, tol=eps_tol, seed=seed)
        degenerate = ncomp > 1
    mu = float(mu_override) if mu_override is not None else mu_value(Q, eps)
    A = (L - mu * Q + eps * sp.identity(n, format="csr")).tocsr()
    a_ptr, a_col = a_structure(n, row_ptr, col, t_ptr, t_col)
    rows = np.repeat(np.arange(n), np.diff(a_ptr))
    a_val = np.asarray(A[rows, a_col.astype(np.int64)]).ravel()
    A_canon = sp.csr_matrix((a_val, a_col.astype(np.int64), a_ptr), shape=(n, n))
    r = gershgorin_radii(a_ptr, a_col, a_val)
    b = b_vector(r)
    return GraphOps(n=n, T=T, t_ptr=t_ptr, t_col=t_col, L=L, Q=Q, eps=eps, mu=mu, A=A_canon,
                    a_ptr=a_ptr, a_col=a_col, a_val=a_val, r=r, b=b, degenerate=degenerate,
                    info={"two_hop_components": ncomp})


def from_graph(g, **kw) -> GraphOps:
    return build_graph_ops(g.n, g.row_ptr, g.col, g.w, **kw)
