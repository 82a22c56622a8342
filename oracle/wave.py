"""The wave equation in space-time Petrov-Galerkin form (paper Section 3 "The Wave Equation", Section 4
"Discretized Wave problem", Section 5 Example 2).  Test infrastructure only: plain SciPy, FP64.

u_tt + A u = f on I x Omega, A = -d^2/dx^2 on Omega = (0, 1) with homogeneous Dirichlet conditions,
u(0) = u_t(0) = 0 (natural in this formulation).  Test space V = R (x) Z with
  Z = span{psi_i} in H^2 cap H^1_0: the cubic B-splines of an open uniform knot vector on n_x intervals of
      (0, 1) without the first and the last (the two that do not vanish at an end point): N_h = n_x + 1;
  R = span{rho^k} in H^2_T = {rho(T) = rho'(T) = 0}: the cubic B-splines on n_t intervals of (0, T) without
      the last two (the two whose value or slope is nonzero at T): N_t = n_t + 1.
Trial space: v_{k,i} = (rho^k)'' psi_i + rho^k A psi_i.  The bilinear form b(v_{k,i}, rho^l psi_j) is the L2(I;H)
inner product of trial functions, so
  B = Q_t (x) M_h + (D_t + D_t^T) (x) A_h + M_t (x) Q_h   (symmetric positive definite),
  M_h = (psi_i, psi_j), A_h = (psi_i', psi_j') = (psi_i, A psi_j), Q_h = (psi_i'', psi_j'') = (A psi_i, A psi_j),
  M_t = (rho^k, rho^l), D_t[k, l] = ((rho^k)'', rho^l), Q_t = ((rho^k)'', (rho^l)''),
and with U (N_h x N_t, U[i, k] the coefficient of v_{k,i}) the matrix equation (eq. 3terms)
  M_h U Q_t^T + A_h U (D_t + D_t^T) + Q_h U M_t = F.
Integrals: Gauss-Legendre with 4 points a knot interval (exact for the products of cubic pieces).
Solver (Section 4): GMRES on the vectorised system, right-preconditioned by P(W) = M_h W Q_t^T + Q_h W M_t, which
is solved by diagonalising the pencils (Q_h, M_h) and (Q_t, M_t).
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.interpolate import BSpline

DEGREE = 3


def knots(n_int: int, length: float) -> np.ndarray:
    """Open uniform knot vector of cubic B-splines on n_int intervals of (0, length)."""
    inner = np.linspace(0.0, length, n_int + 1)
    return np.concatenate([np.zeros(DEGREE), inner, np.full(DEGREE, length)])


def kept_space(n_int: int) -> np.ndarray:
    """Indices of the spatial B-splines kept: all n_int + 3 but the first and the last."""
    return np.arange(1, n_int + 2)


def kept_time(n_int: int) -> np.ndarray:
    """Indices of the temporal B-splines kept: all n_int + 3 but the last two."""
    return np.arange(0, n_int + 1)


def _gauss(n_int: int, length: float, npts: int = 4):
    g, w = np.polynomial.legendre.leggauss(npts)
    edges = np.linspace(0.0, length, n_int + 1)
    a, b = edges[:-1], edges[1:]
    x = (0.5 * (b - a)[:, None] * g[None, :] + 0.5 * (a + b)[:, None]).reshape(-1)
    wx = (0.5 * (b - a)[:, None] * w[None, :]).reshape(-1)
    return x, wx


def basis_values(n_int: int, length: float, x: np.ndarray, deriv: int, kept: np.ndarray) -> np.ndarray:
    """len(x) x len(kept) values of the kept B-splines' derivative of order `deriv` at x."""
    t = knots(n_int, length)
    nb = n_int + DEGREE
    out = np.zeros((len(x), nb))
    for b in range(nb):
        c = np.zeros(nb)
        c[b] = 1.0
        s = BSpline(t, c, DEGREE, extrapolate=False)
        v = s(x, nu=deriv) if deriv else s(x)
        out[:, b] = np.nan_to_num(v)
    return out[:, kept]


def gram(n_int: int, length: float, da: int, db: int, kept: np.ndarray) -> np.ndarray:
    """(d^da phi_a, d^db phi_b) over (0, length) for the kept cubic B-splines."""
    x, w = _gauss(n_int, length)
    Pa = basis_values(n_int, length, x, da, kept)
    Pb = basis_values(n_int, length, x, db, kept)
    return Pa.T @ (w[:, None] * Pb)


def wave_matrices(n_x: int, n_t: int, T: float = 1.0):
    """(M_h, A_h, Q_h, M_t, D_t, Q_t) as dense arrays (banded: bandwidth 3)."""
    ks, kt = kept_space(n_x), kept_time(n_t)
    Mh = gram(n_x, 1.0, 0, 0, ks)
    Ah = gram(n_x, 1.0, 1, 1, ks)
    Qh = gram(n_x, 1.0, 2, 2, ks)
    Mt = gram(n_t, T, 0, 0, kt)
    Dt = gram(n_t, T, 2, 0, kt)   # D_t[k, l] = ((rho^k)'', rho^l)
    Qt = gram(n_t, T, 2, 2, kt)
    return Mh, Ah, Qh, Mt, Dt, Qt


def load_factors(n_x: int, n_t: int, T, space_funcs, time_funcs):
    """F = F1 F2^T with F1[:, p] = (f_p, psi_j) and F2[:, p] = (theta_p, rho^l), by the same quadrature (the
    load of Section 3, [f]_(l,j) = sum_p (theta_p, rho^l)(f_p, psi_j))."""
    xs, ws = _gauss(n_x, 1.0)
    xt, wt = _gauss(n_t, T)
    Ps = basis_values(n_x, 1.0, xs, 0, kept_space(n_x))
    Pt = basis_values(n_t, T, xt, 0, kept_time(n_t))
    F1 = np.stack([Ps.T @ (ws * f(xs)) for f in space_funcs], axis=1)
    F2 = np.stack([Pt.T @ (wt * g(xt)) for g in time_funcs], axis=1)
    return F1, F2


def apply(Mh, Ah, Qh, Mt, Dt, Qt, U):
    """The matrix form of B: M_h U Q_t^T + A_h U (D_t + D_t^T) + Q_h U M_t."""
    return Mh @ U @ Qt.T + Ah @ U @ (Dt + Dt.T) + Qh @ U @ Mt


def assemble(Mh, Ah, Qh, Mt, Dt, Qt) -> sp.csr_matrix:
    """B = Q_t (x) M_h + (D_t + D_t^T) (x) A_h + M_t (x) Q_h (vec stacks columns)."""
    S = lambda X: sp.csr_matrix(X)
    return (sp.kron(S(Qt), S(Mh)) + sp.kron(S(Dt + Dt.T), S(Ah)) + sp.kron(S(Mt), S(Qh))).tocsr()


def solve_direct(Mh, Ah, Qh, Mt, Dt, Qt, F):
    """The exact solution of the assembled system by sparse LU."""
    nh, nt = F.shape
    B = assemble(Mh, Ah, Qh, Mt, Dt, Qt)
    u = spla.splu(B.tocsc()).solve(F.reshape(-1, order="F"))
    return u.reshape((nh, nt), order="F")


class Lyap:
    """P(W) = M_h W Q_t^T + Q_h W M_t and its inverse by the generalised eigenvectors of (Q_h, M_h) and
    (Q_t, M_t): S^T M S = I, S^T Q S = diag(lam), so P^{-1}(V) = S_h [(S_h^T V S_t) / (lam_h_i + lam_t_j)] S_t^T."""

    def __init__(self, Mh, Qh, Mt, Qt):
        self.lh, self.Sh = sla.eigh(Qh, Mh)
        self.lt, self.St = sla.eigh(Qt, Mt)
        self.Mh, self.Qh, self.Mt, self.Qt = Mh, Qh, Mt, Qt

    def apply(self, W):
        return self.Mh @ W @ self.Qt.T + self.Qh @ W @ self.Mt

    def solve(self, V):
        Vh = self.Sh.T @ V @ self.St
        return self.Sh @ (Vh / (self.lh[:, None] + self.lt[None, :])) @ self.St.T


def gmres_lyap(Mh, Ah, Qh, Mt, Dt, Qt, F, tol: float = 1e-8, maxit: int = 200):
    """GMRES on vec(U), X_0 = 0, right-preconditioned by P^{-1} (Lyap.solve), classical Gram-Schmidt twice, Givens
    rotations, no restart; stops when the residual estimate |g_{j+1}| / ||F|| <= tol.  Returns dict(U, iterations,
    history)."""
    P = Lyap(Mh, Qh, Mt, Qt)
    nh, nt = F.shape
    beta = np.linalg.norm(F)
    V = [F / beta]
    Z = []
    H = np.zeros((maxit + 1, maxit))
    cs, sn = np.zeros(maxit), np.zeros(maxit)
    g = np.zeros(maxit + 1)
    g[0] = beta
    hist = []
    j = 0
    for j in range(maxit):
        z = P.solve(V[j])
        Z.append(z)
        w = apply(Mh, Ah, Qh, Mt, Dt, Qt, z)
        for _ in range(2):
            h = np.array([np.sum(v * w) for v in V])
            w = w - sum(hh * v for hh, v in zip(h, V))
            H[: j + 1, j] += h
        hn = np.linalg.norm(w)
        H[j + 1, j] = hn
        for i in range(j):
            a, b = H[i, j], H[i + 1, j]
            H[i, j], H[i + 1, j] = cs[i] * a + sn[i] * b, -sn[i] * a + cs[i] * b
        r = np.hypot(H[j, j], H[j + 1, j])
        cs[j], sn[j] = H[j, j] / r, H[j + 1, j] / r
        H[j, j], H[j + 1, j] = r, 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        hist.append(abs(g[j + 1]) / beta)
        if hist[-1] <= tol or hn == 0.0:
            break
        V.append(w / hn)
    m = j + 1
    y = sla.solve_triangular(H[:m, :m], g[:m])
    U = sum(yy * z for yy, z in zip(y, Z))
    return dict(U=U, iterations=m, history=hist)


def evaluate(U, n_x: int, n_t: int, T: float, x: np.ndarray, t: np.ndarray) -> np.ndarray:
    """u(t, x) = sum_{k,i} U[i, k] ((rho^k)''(t) psi_i(x) - rho^k(t) psi_i''(x)) on the grid t x x."""
    Ps0 = basis_values(n_x, 1.0, x, 0, kept_space(n_x))
    Ps2 = basis_values(n_x, 1.0, x, 2, kept_space(n_x))
    Pt0 = basis_values(n_t, T, t, 0, kept_time(n_t))
    Pt2 = basis_values(n_t, T, t, 2, kept_time(n_t))
    return Pt2 @ U.T @ Ps0.T - Pt0 @ U.T @ Ps2.T
