"""Load matrices F (paper Section 3, eq. par2 and the separable form eq. EIM).

[F]_{j,l} = (f, tau^l (x) phi_j)_{L2(I x Omega)}.  For a separable forcing
f(t,x) = sum_p theta_p(t) f_p(x) this is F = sum_p g_p h_p^T with
g_p[j] = (f_p, phi_j) and h_p[l] = (theta_p, tau^l).

Manufactured problem: u(t,x) = sin(pi t) prod_d sin(pi x_d) on the unit box
solves u_t - Laplace u = f with
f = prod_d sin(pi x_d) * (pi cos(pi t) + dim pi^2 sin(pi t)),
i.e. two separable terms with the same space factor.  The integrals are exact:

    (sin(pi x), phi_i) = sin(pi x_i) * 2 (1 - cos(pi h)) / (pi^2 h)      per direction
    (pi cos(pi t), tau^l) = sin(pi t^l) - sin(pi t^{l-1})
    (dim pi^2 sin(pi t), tau^l) = dim pi (cos(pi t^{l-1}) - cos(pi t^l))
"""

from __future__ import annotations

import numpy as np


def sine_load_1d(n: int) -> np.ndarray:
    h = 1.0 / (n + 1)
    x = h * np.arange(1, n + 1)
    # 2 (1 - cos(pi h)) written as 4 sin^2(pi h / 2) to avoid cancellation
    return np.sin(np.pi * x) * 4.0 * np.sin(0.5 * np.pi * h) ** 2 / (np.pi ** 2 * h)


def space_kron(vectors_x_first):
    """Tensor-product vector with x fastest from per-direction vectors (x first)."""
    out = np.asarray(vectors_x_first[-1])
    for v in reversed(vectors_x_first[:-1]):
        out = np.kron(out, np.asarray(v))
    return out


def manufactured_loads(dim: int, n: int, n_t: int, T: float = 1.0, kappa: float = 1.0):
    """Return (F1, F2) with F = F1 @ F2.T for the manufactured sine solution.

    With a diffusion coefficient kappa the forcing's second time factor is
    kappa * dim * pi^2 sin(pi t).
    """
    g = space_kron([sine_load_1d(n)] * dim)
    t = (T / n_t) * np.arange(0, n_t + 1)
    mid = 0.5 * (t[1:] + t[:-1])
    half = 0.5 * (t[1:] - t[:-1])
    # sin a - sin b = 2 cos((a+b)/2) sin((a-b)/2);  cos b - cos a = 2 sin((a+b)/2) sin((a-b)/2)
    h_a = 2.0 * np.cos(np.pi * mid) * np.sin(np.pi * half)
    h_b = kappa * dim * np.pi * 2.0 * np.sin(np.pi * mid) * np.sin(np.pi * half)
    F1 = np.stack([g, g], axis=1)
    F2 = np.stack([h_a, h_b], axis=1)
    return F1, F2


def manufactured_solution(dim: int, n: int, n_t: int, T: float = 1.0) -> np.ndarray:
    """Nodal values u(t^l, x_j) of the manufactured solution, N_h x N_t."""
    h = 1.0 / (n + 1)
    x = h * np.arange(1, n + 1)
    s = space_kron([np.sin(np.pi * x)] * dim)
    t = (T / n_t) * np.arange(1, n_t + 1)
    return np.outer(s, np.sin(np.pi * t))


def trapezoidal_loads(space_loads: np.ndarray, time_fn, n_t: int, T: float = 1.0):
    """Load matrix with the time integral replaced by the trapezoidal rule.

    For f(t,x) = sum_p theta_p(t) f_p(x) with space loads g_p (columns of
    ``space_loads``) and ``time_fn(t)`` returning the row (theta_1(t), ...),
    F[:, l] = (dt/2) sum_p g_p (theta_p(t^{l-1}) + theta_p(t^l)).
    This is the quadrature under which the scheme equals Crank-Nicolson
    (Section 3).
    """
    dt = T / n_t
    t = dt * np.arange(0, n_t + 1)
    th = np.array([np.atleast_1d(time_fn(tt)) for tt in t])       # (n_t+1, P)
    H = 0.5 * dt * (th[:-1] + th[1:])                               # (n_t, P)
    return np.asarray(space_loads) @ H.T
