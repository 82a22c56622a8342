"""Relative residual norms (paper Section 4; Section 5 stopping rule).

R = F - (M U D_t^T + A U C_t^T).  The paper stops at a final relative residual
norm of 1e-8 without naming the norm; the reading used here is the Frobenius
norm (the 2-norm of vec R) relative to ||F||_F, evaluated in FP64.

For a low-rank iterate U = V Y and F = F1 F2^T the residual factors as
R = L Z^T with L = [F1, M V, A V] and Z = [F2, -D_t Y^T, -C_t Y^T], so
||R||_F = ||R_L Z^T||_F after a thin QR L = Q_L R_L.  This never forms the
Kronecker product or the dense residual.
"""

from __future__ import annotations

import numpy as np


def relres_dense(M, A, D, C, U: np.ndarray, F: np.ndarray) -> float:
    R = F - ((M @ U) @ D.T + (A @ U) @ C.T)
    return float(np.linalg.norm(R) / np.linalg.norm(F))


def lowrank_fro(L: np.ndarray, Z: np.ndarray) -> float:
    """||L Z^T||_F via a thin QR of the tall factor (Householder, numpy)."""
    _, RL = np.linalg.qr(L, mode="reduced")
    return float(np.linalg.norm(RL @ Z.T))


def relres_lowrank(M, A, D, C, V: np.ndarray, Y: np.ndarray, F1: np.ndarray,
                   F2: np.ndarray) -> float:
    L = np.hstack([F1, M @ V, A @ V])
    Z = np.hstack([F2, -(D @ Y.T), -(C @ Y.T)])
    return lowrank_fro(L, Z) / lowrank_fro(F1, F2)


def relres_lowrank_by_columns(M, A, D, C, V: np.ndarray, Y: np.ndarray, F1: np.ndarray, F2: np.ndarray,
                              chunk: int = 64) -> float:
    """The dense residual's relative Frobenius norm for U = V Y, without holding U or R whole.

    R = F1 F2^T - M V (Y D^T) - A V (Y C^T) (paper Section 4's matrix equation) is formed a block of
    ``chunk`` time columns at a time and its squared norm summed; the load's norm comes from F1, F2
    the same way.  This is relres_dense written out block by block, for solutions too large to form.
    """
    YD = Y @ D.T
    YC = Y @ C.T
    num = 0.0
    den = 0.0
    n_t = Y.shape[1]
    for c0 in range(0, n_t, chunk):
        c1 = min(n_t, c0 + chunk)
        F = F1 @ F2[c0:c1].T
        R = F - (M @ (V @ YD[:, c0:c1]) + A @ (V @ YC[:, c0:c1]))
        num += float(np.sum(R * R))
        den += float(np.sum(F * F))
    return float(np.sqrt(num / den))
