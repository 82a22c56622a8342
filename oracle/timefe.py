"""Time matrices of the Petrov-Galerkin discretisation (paper Section 3).

Uniform grid t^k = k dt, dt = T / N_t.  Trial functions sigma^k (k = 1..N_t) are
the hat functions with nodes t^{k-1}, t^k, t^{k+1}; sigma^{N_t} is truncated to
the last interval (the reading of "truncated for k in {0, N_t}": sigma^0 is
absent because u(0) = 0).  Test functions tau^l are the indicators of
I^l = (t^{l-1}, t^l).  The system's time matrices, rows indexed by the test
function l and columns by the trial function k, are

    D_t[l,k] = (d/dt sigma^k, tau^l)_{L2(I)} ,   C_t[l,k] = (sigma^k, tau^l)_{L2(I)}

(Section 3, eq. par1).  On I^l only sigma^l (rising, slope 1/dt) and sigma^{l-1}
(falling, slope -1/dt) are non-zero, so both matrices are lower bidiagonal.
"""

from __future__ import annotations

import numpy as np


def time_matrices(n_t: int, T: float = 1.0):
    """Return dense (D_t, C_t), each N_t x N_t, from the integrals above."""
    dt = T / n_t
    D = np.zeros((n_t, n_t))
    C = np.zeros((n_t, n_t))
    for l in range(n_t):          # test function tau^{l+1} on I^{l+1}
        # sigma^{l+1} rises from 0 to 1 across I^{l+1}
        D[l, l] = (1.0 / dt) * dt          # integral of slope 1/dt over length dt
        C[l, l] = 0.5 * dt                 # area under the rising half-hat
        if l > 0:
            # sigma^{l} falls from 1 to 0 across I^{l+1}
            D[l, l - 1] = (-1.0 / dt) * dt
            C[l, l - 1] = 0.5 * dt
    return D, C
