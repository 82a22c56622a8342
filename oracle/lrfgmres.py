"""Low-rank flexible GMRES preconditioned by RKSM (LR-FGMRES+RKSM): the comparison solver of
Section 5, Example 1 (Table 1).  Test infrastructure, like the rest of this package.

In Example 1 the paper compares RKSM with GMRES run on the space-time system B vec(U) = vec(F), every
Krylov vector held in low-rank form, preconditioned by a fixed number (five) of RKSM iterations; because
that preconditioner is a nonlinear map, GMRES is used in its flexible form.  The paper leaves the details
to a companion paper.  Readings taken here, in the order the method runs:

1.  A vector is an N_h x N_t matrix X = P Q^T.  The inner product is <X, Y> = trace(X^T Y) (the Euclidean
    product of vec X and vec Y), and the operator is the matrix form of B (Section 4):
    L(X) = M X D_t^T + A X C_t^T, so L(P Q^T) = [M P, A P] [D_t Q, C_t Q]^T.
2.  Every sum of low-rank matrices, and every operator product, is truncated: thin QRs of both factors,
    an SVD of the small core, singular values at or below ``trunc`` times the largest dropped
    (trunc = 1e-12 by default; 0 keeps every non-zero one).
3.  Flexible GMRES (Saad, SIAM J. Sci. Comput. 14, 1993) from X_0 = 0 without restart: V_1 = F / beta
    with beta = ||F||_F; step j preconditions Z_j = P(V_j), forms W = L(Z_j), orthogonalises W against
    V_1..V_j by classical Gram-Schmidt run twice (coefficients summed into column j of Hbar), and sets
    h_{j+1,j} = ||W||_F, V_{j+1} = W / h_{j+1,j}.  y_j minimises ||beta e_1 - Hbar_j y|| and the iterate
    is X_j = sum_i Z_i (y_j)_i (truncated).
4.  P(V) applies RKSM (oracle.rksm, Section 4) to L(Z) = V with V's factors as (F1, F2), stopped after a
    fixed number of shifted solves (five) unless its own residual reaches ``precond_tol`` first; the
    preconditioned vector is Z = V_m Y_m, truncated.  The spectral interval of the shifts is computed once.
5.  The iteration stops when the least-squares residual ||beta e_1 - Hbar_j y_j|| / beta is at most tol
    (Section 5 uses 1e-8), or at an exact breakdown h_{j+1,j} = 0.  The true relative residual of the
    returned X (oracle.residual, low-rank and exact) is reported beside it.
6.  Memory (Table 1 gives it as mu_mem (N_h + N_t) numbers): mu_mem counts the columns of every stored
    factor pair, V_1..V_{m+1} and Z_1..Z_m.  The numerical rank of U counts singular values above 1e-8
    of the largest, as for RKSM.

Scope: the heat equation (A symmetric), as in Example 1; the RKSM preconditioner takes its shifts from the
symmetric pencil (A, M).  A nonsymmetric A is refused unless ``precondition=False``.

Pins (tests/test_oracle_lrfgmres.py): the truncation against the Eckart-Young error of a matrix with known
singular values; without a preconditioner, the residual norms against brute-force least squares over the
explicit Krylov space of B; with RKSM run to convergence as the preconditioner, one step; the converged
solution against the direct Kronecker solve; planted mistakes in the operator fail the solution pin.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import rksm as _rksm
from .residual import relres_lowrank


def lr_truncate(P: np.ndarray, Q: np.ndarray, trunc: float = 1e-12):
    """(P', Q') with P' Q'^T the best approximation of P Q^T keeping the singular values above trunc * largest
    (reading 2).  P' = U_r S_r and Q' = V_r for the kept singular triplets."""
    n, m = P.shape[0], Q.shape[0]
    if P.shape[1] == 0:
        return np.zeros((n, 0)), np.zeros((m, 0))
    QP, RP = np.linalg.qr(P, mode="reduced")
    QQ, RQ = np.linalg.qr(Q, mode="reduced")
    U, s, Vt = np.linalg.svd(RP @ RQ.T, full_matrices=False)
    if s.size == 0 or s[0] == 0.0:
        return np.zeros((n, 0)), np.zeros((m, 0))
    r = int(np.sum(s > trunc * s[0]))
    return QP @ (U[:, :r] * s[:r]), QQ @ Vt[:r].T


def lr_inner(X, Y) -> float:
    """<X, Y> = trace(X^T Y) for X = Px Qx^T, Y = Py Qy^T, without forming either (reading 1)."""
    (Px, Qx), (Py, Qy) = X, Y
    return float(np.sum((Px.T @ Py) * (Qx.T @ Qy)))


def lr_operator(M, A, D, C, X):
    """Factors of L(X) = M X D^T + A X C^T for X = P Q^T (reading 1), before truncation."""
    P, Q = X
    return np.hstack([M @ P, A @ P]), np.hstack([D @ Q, C @ Q])


def lr_fgmres(M, A, D, C, F1, F2, tol: float = 1e-8, maxit: int = 50, precond_iters: int = 5,
              precond_tol: float = 0.0, trunc: float = 1e-12, precondition: bool = True, interval=None,
              operator=lr_operator):
    """Run LR-FGMRES+RKSM on M U D^T + A U C^T = F1 F2^T; returns a dict with the solution factors
    (U = P Q^T), the residual history (least-squares estimates, relative), iterations, mu_mem, rank and the
    true residual.  ``precondition=False`` runs plain low-rank GMRES (P = identity).  ``operator`` exists
    so that tests can plant mistakes in it."""
    M = sp.csr_matrix(M)
    A = sp.csr_matrix(A)
    D = np.asarray(D)
    C = np.asarray(C)
    n_h, n_t = M.shape[0], D.shape[0]
    F1c, F2c = _rksm.compress_rhs(F1, F2)
    beta = np.sqrt(max(lr_inner((F1c, F2c), (F1c, F2c)), 0.0))
    empty = dict(P=np.zeros((n_h, 0)), Q=np.zeros((n_t, 0)), history=[0.0], iterations=0, converged=True,
                 mu_mem=0, rank=0, relres=0.0)
    if beta == 0.0:
        return empty
    if precondition and abs(A - A.T).max() > 1e-12 * abs(A).max():
        raise NotImplementedError("the RKSM preconditioner of this oracle needs a symmetric A (heat)")
    if precondition and interval is None:
        interval = _rksm.pencil_interval(M, A)

    def prec(X):
        if not precondition:
            return X
        if X[0].shape[1] == 0:
            return X
        out = _rksm.rksm(M, A, D, C, X[0], X[1], tol=precond_tol, maxit=precond_iters, interval=interval)
        return lr_truncate(out["V"], out["Y"].T, trunc)

    V = [(F1c / beta, F2c)]
    Z = []
    H = np.zeros((maxit + 1, maxit))
    history = [1.0]
    last = None
    converged = False
    y = np.zeros(0)
    for j in range(maxit):
        Zj = prec(V[j])
        Z.append(Zj)
        W = lr_truncate(*operator(M, A, D, C, Zj), trunc)
        for _ in range(2):   # classical Gram-Schmidt, twice
            h = np.array([lr_inner(Vi, W) for Vi in V])
            P = np.hstack([W[0]] + [-hi * Vi[0] for hi, Vi in zip(h, V)])
            Q = np.hstack([W[1]] + [Vi[1] for Vi in V])
            W = lr_truncate(P, Q, trunc)
            H[: j + 1, j] += h
        hn = np.sqrt(max(lr_inner(W, W), 0.0))
        H[j + 1, j] = hn
        rhs = np.zeros(j + 2)
        rhs[0] = beta
        y = np.linalg.lstsq(H[: j + 2, : j + 1], rhs, rcond=None)[0]
        est = float(np.linalg.norm(rhs - H[: j + 2, : j + 1] @ y) / beta)
        history.append(est)
        last = W
        if est <= tol or hn == 0.0:
            converged = est <= tol or hn == 0.0
            break
        V.append((W[0] / hn, W[1]))
    m = len(Z)
    P = np.hstack([y[i] * Z[i][0] for i in range(m)])
    Q = np.hstack([Z[i][1] for i in range(m)])
    P, Q = lr_truncate(P, Q, trunc)
    mu_mem = sum(Vi[0].shape[1] for Vi in V[:m]) + (last[0].shape[1] if last is not None else 0) \
        + sum(Zi[0].shape[1] for Zi in Z)
    s = np.linalg.svd(np.linalg.qr(P, mode="r") @ np.linalg.qr(Q, mode="r").T, compute_uv=False) \
        if P.shape[1] else np.zeros(0)
    rank = int(np.sum(s > 1e-8 * s[0])) if s.size and s[0] > 0 else 0
    relres = relres_lowrank(M, A, D, C, P, Q.T, F1, F2)
    return dict(P=P, Q=Q, history=history, iterations=m, converged=converged, mu_mem=mu_mem, rank=rank,
                relres=relres, interval=interval)
