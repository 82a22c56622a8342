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
