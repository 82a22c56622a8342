"""Crank-Nicolson time stepping on a given load matrix (paper Sections 3 and 5).

Classical CN for M u' + A u = f with u(0) = 0 marches

    (M + dt/2 A) u_l = (M - dt/2 A) u_{l-1} + F[:, l],   l = 1..N_t,

one sparse solve per step, storing the full N_h x N_t solution (Section 5).
When F[:, l] is the interval integral of the load this is exactly the
Petrov-Galerkin system (Section 3 remark); with the trapezoidal rule for the
load it is textbook CN.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla


def crank_nicolson(M, A, dt: float, F: np.ndarray, steps: int | None = None) -> np.ndarray:
    """March ``steps`` (default all N_t) CN steps; returns the computed columns."""
    n_h, n_t = F.shape
    steps = n_t if steps is None else int(steps)
    P = (M + 0.5 * dt * A).tocsc()
    N = (M - 0.5 * dt * A).tocsr()
    lu = spla.splu(P)
    U = np.zeros((n_h, steps))
    prev = np.zeros(n_h)
    for l in range(steps):
        prev = lu.solve(F[:, l] + N @ prev)
        U[:, l] = prev
    return U
