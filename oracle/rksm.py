"""Rational Krylov Galerkin projection (RKSM) reference (paper Section 4, heat part).

Steps, in the paper's order and notation:

1.  F = F1 F2^T with F1 of full column rank (Section 4, before the definition of
    RK_m).  The given factors are compressed: F1 = Q R (thin QR), then an SVD of
    R F2^T; singular values below 1e-14 of the largest are dropped.
2.  V_m has orthonormal columns spanning a rational Krylov space of the
    pencil (A, M) (Section 4, RK_m).  Readings: (a) the printed space
    range[F1, (A - s_2 M)^{-1} M F1, ...] is the rational Krylov space of M^{-1}A
    seeded with F1; the solution of U D_t^T + M^{-1}A U C_t^T = M^{-1}F1 F2^T lies
    in the one seeded with M^{-1} F1, i.e. range[M^{-1}F1, (A - s_2 M)^{-1} F1, ...].
    The two agree when M F1 is proportional to F1 (smooth loads such as the
    paper's Example 1, exactly so for sine modes) and differ for rough loads,
    where only the second contains the solution.  The second is used.
    (b) Each resolvent is applied to the newest orthonormal block (rational
    Arnoldi), which spans the same space for distinct shifts and also allows
    repeated shifts.  Orthogonalisation is block classical Gram-Schmidt run
    twice, then a thin QR of the new block.
3.  Galerkin condition V_m^T R_m = 0 gives the small generalised Sylvester
    equation (V^T M V) Y D_t^T + (V^T A V) Y C_t^T = (V^T F1) F2^T (Section 4;
    the printed "V^T F V" is read as V^T F).
4.  The small equation is solved by a Schur-type method.  The time pencil
    (D_t, C_t) is already lower triangular, so the Bartels-Stewart sweep is a
    recurrence over time columns with one k x k solve per column.
5.  Stop when the relative residual norm (Frobenius, FP64) is at most tol
    (Section 4 cheap residual; Section 5 tolerance 1e-8).  Here it is evaluated
    exactly from the low-rank factors by a thin QR, not by a cheap formula.
6.  Shifts: "determined adaptively" (Section 4).  Reading: the adaptive rule of
    Druskin and Simoncini (2011), which the paper cites for the residual: with
    [a, b] the eigenvalue interval of the pencil (A, M), theta_i the Ritz values
    of the projected pencil and s_j the shifts used so far, the next shift is
    s = argmax over a log-spaced grid of [a, b] of
    prod_j |s - s_j| / prod_i |s + theta_i|, applied as (A + s M)^{-1}
    (i.e. sigma = -s in the paper's notation).  Parity unpinned: the shift
    sequence and iteration counts are not fixed by the paper.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .residual import relres_lowrank


def compress_rhs(F1: np.ndarray, F2: np.ndarray, drop: float = 1e-14):
    """Return (F1c, F2c) with F1c orthonormal, full column rank and F1c F2c^T = F1 F2^T."""
    Q, R = np.linalg.qr(F1, mode="reduced")
    W, s, Zt = np.linalg.svd(R @ F2.T, full_matrices=False)
    r = int(np.sum(s > drop * s[0])) if s.size and s[0] > 0 else 0
    return Q @ W[:, :r], (Zt[:r].T * s[:r])


def pencil_interval(M, A):
    """Smallest and largest eigenvalue of A x = lambda M x (A, M symmetric, M SPD)."""
    n = M.shape[0]
    if n <= 2000:
        w = sla.eigh(A.toarray(), M.toarray(), eigvals_only=True)
        return float(w[0]), float(w[-1])
    lo = spla.eigsh(A.tocsc(), k=1, M=M.tocsc(), sigma=0.0, which="LM",
                    return_eigenvectors=False)[0]
    hi = spla.eigsh(A, k=1, M=M.tocsc(), which="LM", return_eigenvectors=False)[0]
    return float(lo), float(hi)


def next_shift(a: float, b: float, used, ritz, grid: int = 2000) -> float:
    s = np.geomspace(a, b, grid)
    logv = np.zeros_like(s)
    with np.errstate(divide="ignore"):
        for sj in used:
            logv += np.log(np.abs(s - sj))
        for th in ritz:
            logv -= np.log(np.abs(s + th))
    return float(s[int(np.argmax(logv))])


def projected_sylvester(Mm, Am, D, C, Rhs):
    """Solve Mm Y D^T + Am Y C^T = Rhs for lower-bidiagonal D, C (column sweep)."""
    k, n_t = Rhs.shape
    Y = np.zeros((k, n_t))
    cache = {}
    for l in range(n_t):
        key = (D[l, l], C[l, l])
        if key not in cache:
            cache[key] = sla.lu_factor(D[l, l] * Mm + C[l, l] * Am)
        r = Rhs[:, l].copy()
        if l > 0:
            r -= D[l, l - 1] * (Mm @ Y[:, l - 1]) + C[l, l - 1] * (Am @ Y[:, l - 1])
        Y[:, l] = sla.lu_solve(cache[key], r)
    return Y


def _orth_against(V, W):
    """Two passes of block classical Gram-Schmidt, returns (W_perp, coefficients)."""
    H = np.zeros((V.shape[1], W.shape[1]))
    for _ in range(2):
        h = V.T @ W
        W = W - V @ h
        H += h
    return W, H


def rksm(M, A, D, C, F1, F2, tol: float = 1e-8, maxit: int = 100, shifts=None,
         interval=None, breakdown: float = 1e-12, seed: str = "Minv"):
    """Run RKSM; returns dict with V, Y, history, shifts and counters.

    ``shifts`` (positive magnitudes s, sigma = -s) overrides the adaptive rule.
    ``seed`` = "Minv" (start block M^{-1} F1, the reading used) or "F1" (the
    printed space, kept to demonstrate the difference).
    """
    M = sp.csr_matrix(M)
    A = sp.csr_matrix(A)
    F1c, F2c = compress_rhs(F1, F2)
    if F1c.shape[1] == 0:
        return dict(V=np.zeros((M.shape[0], 0)), Y=np.zeros((0, D.shape[0])),
                    history=[0.0], shifts=[], iterations=0, converged=True, p=0)
    a, b = interval if interval is not None else pencil_interval(M, A)
    start = F1c if seed == "F1" else spla.splu(M.tocsc()).solve(F1c)
    V, _ = np.linalg.qr(start, mode="reduced")
    newest = V.copy()
    used = []
    history = []
    lus = {}
    Y = None
    converged = False
    it = 0
    while True:
        Mm = V.T @ (M @ V)
        Am = V.T @ (A @ V)
        Gm = V.T @ F1c
        Y = projected_sylvester(Mm, Am, D, C, Gm @ F2c.T)
        res = relres_lowrank(M, A, D, C, V, Y, F1c, F2c)
        history.append(res)
        if res <= tol:
            converged = True
            break
        if it >= maxit:
            break
        if shifts is not None:
            s = float(shifts[it])
        else:
            ritz = sla.eigh(0.5 * (Am + Am.T), 0.5 * (Mm + Mm.T), eigvals_only=True)
            s = next_shift(a, b, used, ritz)
        used.append(s)
        if s not in lus:
            lus[s] = spla.splu((A + s * M).tocsc())
        W = lus[s].solve(M @ newest)
        W, _ = _orth_against(V, W)
        Q, R = np.linalg.qr(W, mode="reduced")
        keep = np.abs(np.diag(R)) > breakdown * max(1.0, np.abs(R).max())
        it += 1
        if not np.any(keep):
            # the space is invariant: the Galerkin solution is exact in it
            Mm = V.T @ (M @ V)
            Am = V.T @ (A @ V)
            Y = projected_sylvester(Mm, Am, D, C, (V.T @ F1c) @ F2c.T)
            history.append(relres_lowrank(M, A, D, C, V, Y, F1c, F2c))
            converged = history[-1] <= tol
            break
        Q = Q[:, keep]
        Q, _ = _orth_against(V, Q)
        Q, _ = np.linalg.qr(Q, mode="reduced")
        V = np.hstack([V, Q])
        newest = Q
    return dict(V=V, Y=Y, history=history, shifts=used, iterations=it,
                converged=converged, p=F1c.shape[1], interval=(a, b))
