"""Spatial finite-element matrices (paper Section 3, the conforming space X_h).

The paper takes any conforming X_h subset of H^1_0, e.g. piecewise linear
elements.  On a uniform grid of the unit interval with n interior nodes
(h = L/(n+1)) the P1 hat functions give

    M[i,i] = 4h/6, M[i,i+-1] = h/6          (L2 inner products of hats)
    K[i,i] = 2/h,  K[i,i+-1] = -1/h         (L2 inner products of derivatives)
    G[i,i+1] = 1/2, G[i,i-1] = -1/2         (integral of phi_j' phi_i)

On boxes, Q1 elements are tensor products of 1D hats, so the mass matrix is the
Kronecker product of 1D mass matrices and the stiffness matrix is the sum over
directions of one 1D stiffness factor times 1D mass factors in the other
directions.  Nodes are numbered lexicographically with x fastest, so the x
factor is the right-most Kronecker factor.

The heat operator (Section 2, A elliptic with coercive form a) is
a(u,v) = kappa (grad u, grad v).  The convection-diffusion operator is
a(u,v) = eps (grad u, grad v) + (beta . grad u, v).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def p1_mass_1d(n: int, length: float = 1.0) -> sp.csr_matrix:
    h = length / (n + 1)
    main = np.full(n, 4.0 * h / 6.0)
    off = np.full(n - 1, h / 6.0)
    return sp.diags([off, main, off], [-1, 0, 1], format="csr")


def p1_stiffness_1d(n: int, length: float = 1.0) -> sp.csr_matrix:
    h = length / (n + 1)
    main = np.full(n, 2.0 / h)
    off = np.full(n - 1, -1.0 / h)
    return sp.diags([off, main, off], [-1, 0, 1], format="csr")


def p1_convection_1d(n: int) -> sp.csr_matrix:
    """G[i,j] = integral of phi_j' phi_i (independent of h)."""
    up = np.full(n - 1, 0.5)
    lo = np.full(n - 1, -0.5)
    return sp.diags([lo, up], [-1, 1], format="csr")


def _kron_chain(factors):
    """Kronecker product of a list of factors given slowest direction first."""
    out = factors[0]
    for f in factors[1:]:
        out = sp.kron(out, f, format="csr")
    return out.tocsr()


def tensor_operators(dim: int, n, kappa: float = 1.0, length=1.0, op: str = "heat",
                     eps: float | None = None, beta=None):
    """Mass matrix M and operator matrix A of the P1 (dim=1) / Q1 (dim>1) space.

    ``n`` and ``length`` are scalars or per-direction sequences (x first).
    ``op`` is "heat" (A = kappa * stiffness) or "convdiff"
    (A = eps * stiffness + sum_d beta_d * convection_d).
    Returns CSR matrices ordered lexicographically with x fastest.
    """
    ns = [int(n)] * dim if np.isscalar(n) else [int(v) for v in n]
    ls = [float(length)] * dim if np.isscalar(length) else [float(v) for v in length]
    m1 = [p1_mass_1d(ns[d], ls[d]) for d in range(dim)]
    k1 = [p1_stiffness_1d(ns[d], ls[d]) for d in range(dim)]
    # slowest first: direction dim-1 ... 0
    order = list(range(dim - 1, -1, -1))
    M = _kron_chain([m1[d] for d in order])
    stiff = None
    for dd in range(dim):
        term = _kron_chain([k1[d] if d == dd else m1[d] for d in order])
        stiff = term if stiff is None else stiff + term
    if op == "heat":
        A = kappa * stiff
    elif op == "convdiff":
        if eps is None or beta is None:
            raise ValueError("convdiff needs eps and beta")
        g1 = [p1_convection_1d(ns[d]) for d in range(dim)]
        conv = None
        for dd in range(dim):
            term = beta[dd] * _kron_chain([g1[d] if d == dd else m1[d] for d in order])
            conv = term if conv is None else conv + term
        A = eps * stiff + conv
    else:
        raise ValueError(f"unknown operator {op!r}")
    return M.tocsr(), A.tocsr()


def node_coordinates_1d(n: int, length: float = 1.0) -> np.ndarray:
    h = length / (n + 1)
    return h * np.arange(1, n + 1)


def p1_simplex_operators(nodes: np.ndarray, elems: np.ndarray, interior: np.ndarray, kappa: float = 1.0,
                         full: bool = False):
    """P1 mass matrix M and heat operator A = kappa (grad u, grad v) on a simplex mesh (Section 3: X_h the
    piecewise linear functions vanishing on the boundary).

    Element T with vertices x_0..x_d, B = [x_1 - x_0, ..., x_d - x_0]: |T| = |det B| / d!, the gradients of the
    barycentric coordinates lambda_1..lambda_d are the rows of B^{-1} and grad lambda_0 = -sum of the others;
    local stiffness |T| grad lambda_i . grad lambda_j, local mass |T| (1 + delta_ij) / ((d + 1)(d + 2)) (the
    exact integral of a product of two barycentric coordinates).  Returns the matrices on the interior nodes
    (rows and columns in node order), or on all nodes with ``full``.
    """
    nodes = np.asarray(nodes, dtype=float)
    elems = np.asarray(elems)
    d = nodes.shape[1]
    X = nodes[elems]                                   # E x (d+1) x d
    B = np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))   # E x d x d, columns x_i - x_0
    det = np.linalg.det(B)
    fact = 1.0
    for q in range(2, d + 1):
        fact *= q
    vol = np.abs(det) / fact
    Binv = np.linalg.inv(B)                            # rows: grad lambda_1..d
    G = np.concatenate([-Binv.sum(axis=1, keepdims=True), Binv], axis=1)   # E x (d+1) x d
    Kloc = kappa * vol[:, None, None] * np.einsum("eik,ejk->eij", G, G)
    Mloc = vol[:, None, None] * (np.ones((d + 1, d + 1)) + np.eye(d + 1))[None] / ((d + 1) * (d + 2))
    rows = np.repeat(elems, d + 1, axis=1).reshape(-1)
    cols = np.tile(elems, (1, d + 1)).reshape(-1)
    N = nodes.shape[0]
    A = sp.csr_matrix((Kloc.reshape(-1), (rows, cols)), shape=(N, N))
    M = sp.csr_matrix((Mloc.reshape(-1), (rows, cols)), shape=(N, N))
    A.sum_duplicates()
    M.sum_duplicates()
    if full:
        return M, A
    keep = np.flatnonzero(np.asarray(interior))
    M = M[keep][:, keep].tocsr()
    A = A[keep][:, keep].tocsr()
    M.sort_indices()
    A.sort_indices()
    return M, A
