"""Oracle for the generalized eigenproblem of Sec. 4.3 (FP64, CPU).  Test infrastructure.

The embedding is the first K generalized eigenpairs of (A, B): A q = lambda B q with
q_i^T B q_j = delta_ij (Eq. 10-11; the constraint printed as "P B P^T = I" is read as
P^T B P = I, the dimensionally consistent form of the q_i^T B q_j condition).

* ``dense_geneig``: the plain definition.  With B = diag(b) positive definite, the
  pencil is congruent to the symmetric C = B^{-1/2} A B^{-1/2}; its eigenvectors u give
  q = B^{-1/2} u.  One dense symmetric eigendecomposition (LAPACK through numpy) is the
  library step.
* ``sparse_geneig``: the same definition for large N, with ARPACK's shift-invert
  Lanczos on C as the library step (used for reference results at the benchmark's size).
* ``lobpcg``: the locally optimal block preconditioned conjugate gradient method of
  Knyazev (2001), the solver the paper uses, written as the textbook iteration in FP64:
  Rayleigh-Ritz on span[X, W, P] with W = T (A X - B X Lambda) and P the previous step's
  W/P combination.  The preconditioner T is Jacobi, diag(A)^{-1} (the paper names none).
  Orthogonality constraints Y (Y^T B Y = I) are applied to X and W; the constant vector
  is the constraint when computing lambda_2 of a Laplacian.

Convergence and accuracy measures (the paper gives none; these are the readings used):
  relative residual  rho = ||A x - lambda B x||_{B^-1} / ((|lambda| + u ||A||_G) ||x||_B),
      the residual of B^{-1/2} A B^{-1/2} relative to the eigenvalue (ARPACK's rule for
      symmetric problems), u the unit roundoff: the stopping rule of the GPU solver;
  backward error  eta = ||A x - lambda B x||_2 / ((||A||_G + |lambda| max_i b_i) ||x||_2),
      a normwise measure that a rounded vector also satisfies (used to check returned
      FP32 vectors, whose rounding noise the relative residual would magnify);
  with ||A||_G = max_i (A_ii + r_i), a Gershgorin bound on ||A||_2.

Sign convention for returned vectors: the entry of largest magnitude is positive (the
lowest index wins ties).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


@dataclass
class EigResult:
    lam: np.ndarray          # [K] ascending
    V: np.ndarray            # [N, K], V^T B V = I
    iters: int = 0
    converged: bool = True
    eta: np.ndarray | None = None
    restarts: int = 0


def fix_signs(V: np.ndarray) -> np.ndarray:
    V = np.array(V, dtype=np.float64, copy=True)
    for k in range(V.shape[1]):
        i = int(np.argmax(np.abs(V[:, k])))   # argmax returns the lowest index on ties
        if V[i, k] < 0:
            V[:, k] = -V[:, k]
    return V


def dense_geneig(A, b: np.ndarray, K: int | None = None) -> EigResult:
    """All (or the first K) generalized eigenpairs of (A, diag(b)) by dense eigendecomposition."""
    Ad = A.toarray() if sp.issparse(A) else np.asarray(A, dtype=np.float64)
    s = 1.0 / np.sqrt(b)
    C = (Ad * s[:, None]) * s[None, :]
    C = 0.5 * (C + C.T)
    lam, U = np.linalg.eigh(C)
    V = U * s[:, None]
    if K is not None:
        lam, V = lam[:K], V[:, :K]
    return EigResult(lam=lam, V=fix_signs(V))


def gershgorin_norm(A) -> float:
    """||A||_G = max_i (A_ii + sum_{j != i} |A_ij|), an upper bound on ||A||_2."""
    A = sp.csr_matrix(A)
    absrow = np.asarray(abs(A).sum(axis=1)).ravel()
    d = A.diagonal()
    return float(np.max(absrow - np.abs(d) + d))


def backward_errors(A, b, lam, V, normA=None) -> np.ndarray:
    """eta_k for each column (see module docstring)."""
    if normA is None:
        normA = gershgorin_norm(A)
    R = A @ V - (b[:, None] * V) * lam[None, :]
    rn = np.linalg.norm(R, axis=0)
    xn = np.linalg.norm(V, axis=0)
    return rn / ((normA + np.abs(lam) * np.max(b)) * xn)


def relative_residuals(A, b, lam, V, normA=None, unit_roundoff: float = 2.0 ** -53) -> np.ndarray:
    """rho_k = ||A v - lambda B v||_{B^-1} / ((|lambda| + u ||A||_G) ||v||_B) for each column.

    The residual of the symmetric form C = B^{-1/2} A B^{-1/2} (with u = B^{1/2} v, C u -
    lambda u = B^{-1/2} r) relative to the eigenvalue -- the stopping rule ARPACK applies to
    symmetric problems -- with the unit roundoff u times ||A||_G as a floor for lambda = 0.
    Norms: ||r||_{B^-1}^2 = sum r_i^2 / b_i, ||v||_B^2 = sum b_i v_i^2."""
    if normA is None:
        normA = gershgorin_norm(A)
    R = A @ V - (b[:, None] * V) * lam[None, :]
    rn = np.sqrt(np.sum(R * R / b[:, None], axis=0))
    vn = np.sqrt(np.sum(b[:, None] * V * V, axis=0))
    return rn / ((np.abs(lam) + unit_roundoff * normA) * vn)


def _b_orthonormalize(V, b):
    """Cholesky QR in the B inner product; returns None when the Gram is not positive definite."""
    G = V.T @ (b[:, None] * V)
    G = 0.5 * (G + G.T)
    try:
        R = np.linalg.cholesky(G).T          # G = R^T R
    except np.linalg.LinAlgError:
        return None
    return sla.solve_triangular(R, V.T, trans="T", lower=False).T


def _apply_constraints(V, Y, b):
    if Y is None:
        return V
    return V - Y @ (Y.T @ (b[:, None] * V))


def lobpcg(A, b: np.ndarray, K: int, *, guard: int = 0, Y=None, tol: float = 1e-10,
           maxiter: int = 20000, seed: int = 0, X0=None, precond: str = "jacobi",
           normA: float | None = None, measure: str = "backward") -> EigResult:
    """Textbook FP64 LOBPCG for the K smallest eigenpairs of (A, diag(b)).

    m = K + guard columns are iterated; convergence is tested on the first K by the
    backward error eta <= tol (measure="backward") or by the relative residual
    rho <= tol (measure="relative", see ``relative_residuals``).
    """
    if measure not in ("backward", "relative"):
        raise ValueError(measure)
    A = sp.csr_matrix(A)
    n = A.shape[0]
    m = K + guard
    if normA is None:
        normA = gershgorin_norm(A)
    bmax = float(np.max(b))
    T = 1.0 / A.diagonal() if precond == "jacobi" else np.ones(n)
    if Y is not None:
        Y = _b_orthonormalize(np.asarray(Y, dtype=np.float64), b)
    if X0 is None:
        X0 = np.random.Generator(np.random.PCG64(seed)).standard_normal((n, m))
    X = _apply_constraints(np.array(X0, dtype=np.float64), Y, b)
    X = _b_orthonormalize(X, b)
    # initial Rayleigh-Ritz on span(X)
    AX = A @ X
    lam, C = sla.eigh(0.5 * (X.T @ AX + AX.T @ X))
    X, AX = X @ C, AX @ C
    P = AP = None
    restarts = 0
    eta = None
    for it in range(1, maxiter + 1):
        BX = b[:, None] * X
        R = AX - BX * lam[None, :]
        if measure == "backward":
            rn = np.linalg.norm(R, axis=0)
            eta = rn / ((normA + np.abs(lam) * bmax) * np.linalg.norm(X, axis=0))
        else:
            rn = np.sqrt(np.sum(R * R / b[:, None], axis=0))
            eta = rn / ((np.abs(lam) + 2.0 ** -53 * normA) * np.sqrt(np.sum(BX * X, axis=0)))
        if np.all(eta[:K] <= tol):
            return EigResult(lam[:K].copy(), fix_signs(X[:, :K]), it - 1, True, eta[:K], restarts)
        W = T[:, None] * R
        W = _apply_constraints(W, Y, b)
        W = W - X @ (BX.T @ W)
        Wn = _b_orthonormalize(W, b)
        if Wn is None:                      # W numerically rank deficient: orthonormalise by eigh
            G = W.T @ (b[:, None] * W)
            d, U = np.linalg.eigh(0.5 * (G + G.T))
            keep = d > d[-1] * 1e-14
            W = (W @ U[:, keep]) / np.sqrt(d[keep])[None, :]
        else:
            W = Wn
        AW = A @ W
        blocks = [X, W] + ([P] if P is not None else [])
        ablocks = [AX, AW] + ([AP] if AP is not None else [])
        while True:
            S = np.hstack(blocks)
            AS = np.hstack(ablocks)
            GA = S.T @ AS
            GB = S.T @ (b[:, None] * S)
            try:
                theta, Cf = sla.eigh(0.5 * (GA + GA.T), 0.5 * (GB + GB.T))
                break
            except (np.linalg.LinAlgError, sla.LinAlgError):
                if len(blocks) == 3:            # drop P and retry (restart)
                    blocks, ablocks = blocks[:2], ablocks[:2]
                    restarts += 1
                    continue
                raise
        C = Cf[:, :m]
        lam = theta[:m]
        X_new = S @ C
        AX_new = AS @ C
        nx = X.shape[1]
        P = S[:, nx:] @ C[nx:, :]
        AP = AS[:, nx:] @ C[nx:, :]
        X, AX = X_new, AX_new
    return EigResult(lam[:K].copy(), fix_signs(X[:, :K]), maxiter, False, eta[:K], restarts)


def sparse_geneig(A, b: np.ndarray, K: int, *, sigma: float | None = None,
                  tol: float = 0.0) -> EigResult:
    """The first K generalized eigenpairs of (A, diag(b)) for large sparse A.

    The same definition as ``dense_geneig`` (eigenpairs of C = B^{-1/2} A B^{-1/2},
    q = B^{-1/2} u), with ARPACK's shift-invert Lanczos (scipy ``eigsh``, a sparse LU of
    C - sigma I) as the library step that finds the K eigenvalues of C nearest sigma.  The
    default sigma sits just below zero: A is positive semidefinite (Sec. 4.2), so the
    eigenvalues nearest sigma are the smallest, and C - sigma I stays nonsingular when A
    itself is singular (eps = 0).  ``tol`` = 0 asks ARPACK for machine precision.
    """
    import scipy.sparse.linalg as spla
    A = sp.csr_matrix(A)
    n = A.shape[0]
    s = 1.0 / np.sqrt(np.asarray(b, dtype=np.float64))
    Cm = (sp.diags(s) @ A @ sp.diags(s)).tocsc()
    Cm = 0.5 * (Cm + Cm.T)
    if sigma is None:
        sigma = -1e-9 * gershgorin_norm(A)
    k = min(K, n - 1)
    lam, U = spla.eigsh(Cm, k=k, sigma=sigma, which="LM", tol=tol,
                        v0=np.ones(n) / np.sqrt(n))
    order = np.argsort(lam)
    lam, U = lam[order], U[:, order]
    return EigResult(lam=lam, V=fix_signs(U * s[:, None]))


def embed(ops, K: int, *, tol: float | None = None, dense_max: int = 3000, guard: int = 0,
          seed: int = 0, X0=None) -> EigResult:
    """First K generalized eigenpairs of (A, B) for an oracle GraphOps."""
    if ops.n <= dense_max:
        return dense_geneig(ops.A, ops.b, K)
    return lobpcg(ops.A, ops.b, K, guard=guard, tol=1e-11 if tol is None else tol, seed=seed, X0=X0)


def subspace_angle(U: np.ndarray, V: np.ndarray) -> float:
    """Largest principal angle (radians) between span(U) and span(V), Euclidean inner product."""
    Qu, _ = np.linalg.qr(U)
    Qv, _ = np.linalg.qr(V)
    s = np.linalg.svd(Qu.T @ Qv, compute_uv=False)
    s = np.clip(s, -1.0, 1.0)
    # sin of the largest angle from the complement, accurate for small angles
    Rm = Qv - Qu @ (Qu.T @ Qv)
    sin_max = float(np.linalg.norm(Rm, 2)) if Rm.size else 0.0
    return float(np.arcsin(min(1.0, sin_max))) if sin_max < 0.5 else float(np.arccos(np.min(s)))
