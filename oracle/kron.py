"""Kronecker form of the space-time system and its exact solution (paper Sections 3-4).

Unknown U is N_h x N_t; column k holds the spatial coefficients of sigma^k.  The
equation for test function (l, j) is row j of column l of

    M U D_t^T + A U C_t^T = F                                   (Section 4)

which is the vectorised system B vec(U) = vec(F) with
B = D_t (x) M + C_t (x) A (Section 3, eq. par1; Section 4 eq. Kroneckersum and
the identity (D (x) A) vec(X) = vec(A X D^T)).  vec stacks columns, so the row
index of B is l * N_h + j.

Reading of the transposes: the paper writes both "B^T u = f" and "B u = f" and
the matrix equation without transposes.  Rows = test indices, columns = trial
indices is the orientation that is a causal recurrence in time and reproduces
Crank-Nicolson; it is the one used throughout.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def vec(U: np.ndarray) -> np.ndarray:
    return np.asarray(U).reshape(-1, order="F")


def unvec(u: np.ndarray, n_h: int, n_t: int) -> np.ndarray:
    return np.asarray(u).reshape((n_h, n_t), order="F")


def assemble(M, A, D, C) -> sp.csr_matrix:
    """B = D (x) M + C (x) A as a sparse matrix (never formed by the GPU path)."""
    return (sp.kron(sp.csr_matrix(D), M) + sp.kron(sp.csr_matrix(C), A)).tocsr()


def apply(M, A, D, C, U: np.ndarray) -> np.ndarray:
    """Matrix form of the operator: M U D^T + A U C^T."""
    U = np.asarray(U)
    return (M @ U) @ D.T + (A @ U) @ C.T


def solve_sparse(M, A, D, C, F: np.ndarray) -> np.ndarray:
    """Exact solution by sparse LU (SuperLU) of the assembled system."""
    n_h, n_t = F.shape
    B = assemble(M, A, D, C).tocsc()
    u = spla.splu(B).solve(vec(F))
    return unvec(u, n_h, n_t)


def solve_dense(M, A, D, C, F: np.ndarray) -> np.ndarray:
    """Brute force: dense LU of the assembled system (tiny sizes only)."""
    n_h, n_t = F.shape
    B = assemble(M, A, D, C).toarray()
    return unvec(np.linalg.solve(B, vec(F)), n_h, n_t)


def forward_substitution(M, A, D, C, F: np.ndarray) -> np.ndarray:
    """Block forward substitution of the block lower-bidiagonal system.

    D and C are lower bidiagonal, so B is block lower bidiagonal in time.  Row
    block l reads (D[l,l] M + C[l,l] A) u_l = F_l - (D[l,l-1] M + C[l,l-1] A) u_{l-1}.
    With a uniform grid every diagonal block is the same matrix, which is
    factored once.  This is direct elimination of B: exact up to rounding.
    """
    n_h, n_t = F.shape
    U = np.zeros((n_h, n_t))
    diag_blocks = {}
    for l in range(n_t):
        key = (D[l, l], C[l, l])
        if key not in diag_blocks:
            diag_blocks[key] = spla.splu((D[l, l] * M + C[l, l] * A).tocsc())
        rhs = np.array(F[:, l], dtype=np.float64)
        if l > 0:
            rhs -= D[l, l - 1] * (M @ U[:, l - 1]) + C[l, l - 1] * (A @ U[:, l - 1])
        U[:, l] = diag_blocks[key].solve(rhs)
    return U


def forward_substitution_cg(M, A, D, C, F1: np.ndarray, F2: np.ndarray, steps: int, rtol: float = 1e-14):
    """The first ``steps`` columns of the block forward substitution, each block solved by
    conjugate gradients (the diagonal blocks D[l,l] M + C[l,l] A are symmetric positive
    definite for the heat operator).  For grids whose direct factorisation does not fit:
    forward substitution fixes the first columns exactly whatever the later ones are.
    The load is given as factors, F[:, l] = F1 @ F2[l]."""
    n_h = M.shape[0]
    U = np.zeros((n_h, steps))
    prev = None
    for l in range(steps):
        Bl = (D[l, l] * M + C[l, l] * A).tocsr()
        rhs = F1 @ F2[l]
        if l > 0:
            rhs = rhs - (D[l, l - 1] * (M @ prev) + C[l, l - 1] * (A @ prev))
        x = _cg(Bl, rhs, rtol, 20 * n_h)
        U[:, l] = x
        prev = x
    return U


class _NormalOperator:
    """x -> B^T B x for the normal equations of a nonsymmetric block."""

    def __init__(self, B):
        self.B = B
        self.BT = B.T.tocsr()

    def __matmul__(self, x):
        return self.BT @ (self.B @ x)


def forward_substitution_normal_cg(M, A, D, C, F1: np.ndarray, F2: np.ndarray, steps: int, rtol: float = 1e-15):
    """forward_substitution_cg for a nonsymmetric operator (convection-diffusion): each diagonal block
    B_l = D[l,l] M + C[l,l] A is nonsingular but not symmetric, so the block equation B_l u = r is solved as
    the normal equations B_l^T B_l u = B_l^T r by the same textbook conjugate gradients (CGNR, Hestenes and
    Stiefel 1952, Section 10).  The first ``steps`` columns only, as forward_substitution_cg."""
    n_h = M.shape[0]
    U = np.zeros((n_h, steps))
    prev = None
    for l in range(steps):
        Bl = (D[l, l] * M + C[l, l] * A).tocsr()
        rhs = F1 @ F2[l]
        if l > 0:
            rhs = rhs - (D[l, l - 1] * (M @ prev) + C[l, l - 1] * (A @ prev))
        Nl = _NormalOperator(Bl)
        x = _cg(Nl, Nl.BT @ rhs, rtol, 50 * n_h)
        U[:, l] = x
        prev = x
    return U


def _cg(B, b: np.ndarray, rtol: float, maxiter: int) -> np.ndarray:
    """Textbook conjugate gradients (Hestenes-Stiefel) from x = 0, stopping at ||r|| <= rtol ||b||."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(r @ r)
    stop = (rtol * np.linalg.norm(b)) ** 2
    for _ in range(maxiter):
        if rr <= stop:
            return x
        q = B @ p
        alpha = rr / float(p @ q)
        x += alpha * p
        r -= alpha * q
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
    raise RuntimeError("CG did not reach the requested tolerance")
