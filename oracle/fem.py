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
