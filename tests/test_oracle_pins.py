"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test pins a part of ``oracle/`` to something other than the oracle itself:
Gauss quadrature of the basis functions, closed-form eigenpairs, an exact
rational solve, the Crank-Nicolson equivalence, a manufactured solution and its
convergence order, and the Galerkin invariants of the RKSM reference.  The last
tests plant mistakes in the oracle (on the CPU) and check that a pin catches them.
"""

from fractions import Fraction
from pathlib import Path

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import cn, fem, kron, residual, rhs, rksm, timefe
import workloads

GOLDEN = Path(__file__).resolve().parent / "golden"

# ---------------------------------------------------------------- helpers


def hat(x, xc, h):
    return np.maximum(0.0, 1.0 - np.abs(x - xc) / h)


def dhat(x, xc, h):
    # derivative of the hat function inside its support (piecewise constant)
    return np.where((x > xc - h) & (x < xc), 1.0 / h, np.where((x > xc) & (x < xc + h), -1.0 / h, 0.0))


def quad_1d(n, length, kind):
    """1D P1 matrix by 3-point Gauss-Legendre quadrature on every element."""
    h = length / (n + 1)
    nodes = h * np.arange(1, n + 1)
    g, w = np.polynomial.legendre.leggauss(3)
    out = np.zeros((n, n))
    for e in range(n + 1):
        a, b = e * h, (e + 1) * h
        xq = 0.5 * (b - a) * g + 0.5 * (a + b)
        wq = 0.5 * (b - a) * w
        for i in range(n):
            for j in range(n):
                if kind == "M":
                    f = hat(xq, nodes[i], h) * hat(xq, nodes[j], h)
                elif kind == "K":
                    f = dhat(xq, nodes[i], h) * dhat(xq, nodes[j], h)
                else:  # G[i, j] = int phi_j' phi_i
                    f = dhat(xq, nodes[j], h) * hat(xq, nodes[i], h)
                out[i, j] += np.sum(wq * f)
    return out


def quad_q1_2d(nx, ny, lx, ly):
    """2D Q1 mass and stiffness by tensor Gauss quadrature over every rectangle."""
    hx, hy = lx / (nx + 1), ly / (ny + 1)
    g, w = np.polynomial.legendre.leggauss(3)
    N = nx * ny
    Mq = np.zeros((N, N))
    Kq = np.zeros((N, N))
    xs = hx * np.arange(1, nx + 1)
    ys = hy * np.arange(1, ny + 1)
    for ex in range(nx + 1):
        for ey in range(ny + 1):
            ax, bx = ex * hx, (ex + 1) * hx
            ay, by = ey * hy, (ey + 1) * hy
            xq = 0.5 * (bx - ax) * g + 0.5 * (ax + bx)
            yq = 0.5 * (by - ay) * g + 0.5 * (ay + by)
            X, Yg = np.meshgrid(xq, yq, indexing="ij")
            W = np.outer(0.5 * (bx - ax) * w, 0.5 * (by - ay) * w)
            vals, gx, gy = [], [], []
            for j in range(ny):
                for i in range(nx):     # x fastest
                    vals.append(hat(X, xs[i], hx) * hat(Yg, ys[j], hy))
                    gx.append(dhat(X, xs[i], hx) * hat(Yg, ys[j], hy))
                    gy.append(hat(X, xs[i], hx) * dhat(Yg, ys[j], hy))
            for a in range(N):
                if not vals[a].any() and not gx[a].any():
                    continue
                for b in range(N):
                    Mq[a, b] += np.sum(W * vals[a] * vals[b])
                    Kq[a, b] += np.sum(W * (gx[a] * gx[b] + gy[a] * gy[b]))
    return Mq, Kq


def textbook_cn(M, A, dt, loads_at_nodes):
    """(M + dt/2 A) u^l = (M - dt/2 A) u^{l-1} + dt/2 (f^{l-1} + f^l), dense."""
    Md, Ad = M.toarray(), A.toarray()
    n, nt1 = loads_at_nodes.shape
    u = np.zeros(n)
    out = []
    for l in range(1, nt1):
        rhs_ = (Md - 0.5 * dt * Ad) @ u + 0.5 * dt * (loads_at_nodes[:, l - 1] + loads_at_nodes[:, l])
        u = np.linalg.solve(Md + 0.5 * dt * Ad, rhs_)
        out.append(u)
    return np.array(out).T


# ---------------------------------------------------------------- space


@pytest.mark.parametrize("n,length", [(7, 1.0), (20, 1.0), (9, 2.5)])
def test_p1_matrices_match_quadrature(n, length):
    assert np.allclose(fem.p1_mass_1d(n, length).toarray(), quad_1d(n, length, "M"), rtol=0, atol=1e-15)
    assert np.allclose(fem.p1_stiffness_1d(n, length).toarray(), quad_1d(n, length, "K"), rtol=0, atol=1e-13)
    assert np.allclose(fem.p1_convection_1d(n).toarray(), quad_1d(n, length, "G"), rtol=0, atol=1e-14)


@pytest.mark.parametrize("n,length", [(7, 1.0), (31, 1.0), (12, 3.0)])
def test_p1_generalised_eigenpairs_closed_form(n, length):
    """K s_j = lam_j M s_j with s_j = sin(j pi x_i / L), lam_j = (6/h^2)(1-cos)/(2+cos)."""
    M = fem.p1_mass_1d(n, length).toarray()
    K = fem.p1_stiffness_1d(n, length).toarray()
    h = length / (n + 1)
    j = np.arange(1, n + 1)
    th = j * np.pi / (n + 1)
    lam = (6.0 / h ** 2) * (1 - np.cos(th)) / (2 + np.cos(th))
    S = np.sin(np.outer(np.arange(1, n + 1), j) * np.pi / (n + 1))
    assert np.allclose(K @ S, (M @ S) * lam[None, :], rtol=1e-12, atol=1e-10 * lam.max())
    w = sla.eigh(K, M, eigvals_only=True)
    assert np.allclose(np.sort(w), np.sort(lam), rtol=1e-12)


def test_q1_2d_matches_quadrature_anisotropic():
    M, A = fem.tensor_operators(2, (3, 4), kappa=1.0, length=(1.0, 2.0))
    Mq, Kq = quad_q1_2d(3, 4, 1.0, 2.0)
    assert np.allclose(M.toarray(), Mq, atol=1e-15)
    assert np.allclose(A.toarray(), Kq, atol=1e-13)


@pytest.mark.parametrize("dim,n", [(1, 9), (2, 6), (3, 4)])
def test_q1_eigenvalues_are_sums(dim, n):
    M, A = fem.tensor_operators(dim, n, kappa=1.7)
    h = 1.0 / (n + 1)
    th = np.arange(1, n + 1) * np.pi / (n + 1)
    lam1 = (6.0 / h ** 2) * (1 - np.cos(th)) / (2 + np.cos(th))
    grids = np.meshgrid(*([lam1] * dim), indexing="ij")
    expect = np.sort(1.7 * sum(grids).ravel())
    w = sla.eigh(A.toarray(), M.toarray(), eigvals_only=True)
    assert np.allclose(np.sort(w), expect, rtol=1e-11)


@pytest.mark.parametrize("dim,n", [(1, 11), (2, 7), (3, 4)])
def test_mass_and_operator_symmetric_positive_definite(dim, n):
    M, A = fem.tensor_operators(dim, n)
    for X in (M.toarray(), A.toarray()):
        assert np.array_equal(X, X.T)
        np.linalg.cholesky(X)
        assert np.linalg.eigvalsh(X).min() > 0


def test_convdiff_operator_parts():
    eps, beta = 0.3, (1.0, 0.5)
    M, A = fem.tensor_operators(2, 5, op="convdiff", eps=eps, beta=beta)
    _, K = fem.tensor_operators(2, 5, kappa=1.0)
    C = A - eps * K
    assert abs(C + C.T).max() < 1e-15            # convection is skew
    x = np.linspace(0.1, 0.9, 25)
    assert np.all(np.linalg.eigvals(A.toarray()).real > 0)


# ---------------------------------------------------------------- time


@pytest.mark.parametrize("n_t,T", [(1, 1.0), (5, 1.0), (12, 3.0)])
def test_time_matrices_match_quadrature(n_t, T):
    """D[l,k] = int_{I^l} d/dt sigma^k, C[l,k] = int_{I^l} sigma^k from pointwise hats."""
    D, C = timefe.time_matrices(n_t, T)
    dt = T / n_t
    g, w = np.polynomial.legendre.leggauss(4)
    Dq = np.zeros((n_t, n_t))
    Cq = np.zeros((n_t, n_t))
    tk = dt * np.arange(0, n_t + 1)
    for l in range(1, n_t + 1):
        a, b = tk[l - 1], tk[l]
        tq = 0.5 * (b - a) * g + 0.5 * (a + b)
        wq = 0.5 * (b - a) * w
        for k in range(1, n_t + 1):
            sig = hat(tq, tk[k], dt)
            if k == n_t:   # truncated at T
                sig = np.where(tq <= tk[k], sig, 0.0)
            dsig = dhat(tq, tk[k], dt)
            Dq[l - 1, k - 1] = np.sum(wq * dsig)
            Cq[l - 1, k - 1] = np.sum(wq * sig)
    assert np.allclose(D, Dq, atol=1e-14)
    assert np.allclose(C, Cq, atol=1e-15)


# ---------------------------------------------------------------- Kronecker system


def test_kronecker_entries_from_definition_and_vec_identity():
    M, A = fem.tensor_operators(1, 4)
    D, C = timefe.time_matrices(3, 1.0)
    Md, Ad = M.toarray(), A.toarray()
    n, nt = 4, 3
    B = np.zeros((n * nt, n * nt))
    for l in range(nt):
        for j in range(n):
            for k in range(nt):
                for i in range(n):
                    B[l * n + j, k * n + i] = D[l, k] * Md[j, i] + C[l, k] * Ad[j, i]
    assert np.array_equal(kron.assemble(M, A, D, C).toarray(), B)
    U = np.random.default_rng(0).standard_normal((n, nt))
    assert np.allclose(kron.vec(kron.apply(M, A, D, C, U)), B @ kron.vec(U), atol=1e-13)


def _frac_solve(Bf, bf):
    n = len(bf)
    A = [row[:] + [bf[i]] for i, row in enumerate(Bf)]
    for c in range(n):
        piv = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        for r in range(n):
            if r != c and A[r][c] != 0:
                f = A[r][c] / A[c][c]
                A[r] = [x - f * y for x, y in zip(A[r], A[c])]
    return [A[i][n] / A[i][i] for i in range(n)]


def test_exact_rational_solution_of_tiny_system():
    """n = 3 interior nodes (h = 1/4), N_t = 3 (dt = 1/3): exact solve in rationals."""
    n, nt = 3, 3
    h, dt = Fraction(1, 4), Fraction(1, 3)
    Mf = [[h * 4 / 6 if i == j else (h / 6 if abs(i - j) == 1 else Fraction(0)) for j in range(n)] for i in range(n)]
    Kf = [[2 / h if i == j else (-1 / h if abs(i - j) == 1 else Fraction(0)) for j in range(n)] for i in range(n)]
    Df = [[Fraction(1) if l == k else (Fraction(-1) if l == k + 1 else Fraction(0)) for k in range(nt)] for l in range(nt)]
    Cf = [[dt / 2 if (l == k or l == k + 1) else Fraction(0) for k in range(nt)] for l in range(nt)]
    Bf = [[Df[l][k] * Mf[j][i] + Cf[l][k] * Kf[j][i] for k in range(nt) for i in range(n)]
          for l in range(nt) for j in range(n)]
    F = np.array([[1, -2, 3], [0, 5, -1], [2, 2, 4]], dtype=float)
    bf = [Fraction(int(F[j, l])) for l in range(nt) for j in range(n)]
    exact = np.array([float(v) for v in _frac_solve(Bf, bf)]).reshape((n, nt), order="F")
    M, A = fem.tensor_operators(1, n)
    D, C = timefe.time_matrices(nt, 1.0)
    for U in (kron.solve_sparse(M, A, D, C, F), kron.solve_dense(M, A, D, C, F),
              kron.forward_substitution(M, A, D, C, F), cn.crank_nicolson(M, A, 1.0 / nt, F)):
        assert np.allclose(U, exact, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("dim,n,nt", [(1, 9, 7), (2, 4, 6)])
def test_sparse_lu_equals_dense_bruteforce(dim, n, nt):
    M, A = fem.tensor_operators(dim, n, kappa=0.7)
    D, C = timefe.time_matrices(nt, 2.0)
    F = np.random.default_rng(3).standard_normal((M.shape[0], nt))
    Us = kron.solve_sparse(M, A, D, C, F)
    Ud = kron.solve_dense(M, A, D, C, F)
    assert np.allclose(Us, Ud, rtol=1e-12, atol=1e-14)
    assert np.allclose(kron.forward_substitution(M, A, D, C, F), Ud, rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------- Crank-Nicolson (Section 3 remark)


@pytest.mark.parametrize("dim,n,nt", [(1, 15, 16), (2, 7, 9)])
def test_pg_with_trapezoidal_load_equals_textbook_cn(dim, n, nt):
    """The PG scheme with trapezoidal load integration is the CN scheme (Section 3)."""
    M, A = fem.tensor_operators(dim, n)
    D, C = timefe.time_matrices(nt, 1.0)
    dt = 1.0 / nt
    g = rhs.space_kron([rhs.sine_load_1d(n)] * dim)
    time_fn = lambda t: np.array([np.exp(-t) * (1 + 3 * t), np.cos(5 * t)])
    space = np.stack([g, g[::-1] * 0.5], axis=1)
    Ftrap = rhs.trapezoidal_loads(space, time_fn, nt, 1.0)
    U_pg = kron.solve_sparse(M, A, D, C, Ftrap)
    nodes = np.array([space @ time_fn(l * dt) for l in range(nt + 1)]).T
    U_cn = textbook_cn(M, A, dt, nodes)
    assert np.linalg.norm(U_pg - U_cn) <= 1e-13 * np.linalg.norm(U_cn)


# ---------------------------------------------------------------- manufactured solution


@pytest.mark.parametrize("dim,n,nt", [(1, 15, 20), (2, 7, 12), (3, 3, 5)])
def test_manufactured_closed_form_recurrence(dim, n, nt):
    """U = s (x) y: M s = mu s, K s = lam mu s per direction gives a scalar recurrence."""
    M, A = fem.tensor_operators(dim, n)
    D, C = timefe.time_matrices(nt, 1.0)
    F1, F2 = rhs.manufactured_loads(dim, n, nt)
    U = kron.solve_sparse(M, A, D, C, F1 @ F2.T)
    h = 1.0 / (n + 1)
    x = h * np.arange(1, n + 1)
    s = rhs.space_kron([np.sin(np.pi * x)] * dim)
    mu1 = h * (4 + 2 * np.cos(np.pi * h)) / 6
    lam1 = (6 / h ** 2) * (1 - np.cos(np.pi * h)) / (2 + np.cos(np.pi * h))
    mu, lam = mu1 ** dim, dim * lam1
    c = 4 * np.sin(0.5 * np.pi * h) ** 2 / (np.pi ** 2 * h)      # load of sin on one hat
    hl = (F2 @ np.ones(2))
    dt = 1.0 / nt
    y = np.zeros(nt)
    prev = 0.0
    for l in range(nt):
        # mu (y_l - y_{l-1}) + dt/2 lam mu (y_l + y_{l-1}) = c^dim h_l
        prev = (c ** dim * hl[l] / mu + (1 - 0.5 * dt * lam) * prev) / (1 + 0.5 * dt * lam)
        y[l] = prev
    assert np.allclose(U, np.outer(s, y), rtol=1e-11, atol=1e-13)


def test_manufactured_second_order_convergence():
    errs = []
    for n in (15, 31, 63):
        nt = n + 1
        M, A = fem.tensor_operators(1, n)
        D, C = timefe.time_matrices(nt, 1.0)
        F1, F2 = rhs.manufactured_loads(1, n, nt)
        U = kron.forward_substitution(M, A, D, C, F1 @ F2.T)
        errs.append(np.abs(U - rhs.manufactured_solution(1, n, nt)).max())
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(3.8 < r < 4.2 for r in ratios), ratios


# ---------------------------------------------------------------- residuals


def test_lowrank_residual_equals_dense_residual():
    M, A = fem.tensor_operators(2, 6)
    D, C = timefe.time_matrices(9, 1.0)
    rng = np.random.default_rng(5)
    V = rng.standard_normal((36, 4))
    Y = rng.standard_normal((4, 9))
    F1, F2 = rng.standard_normal((36, 2)), rng.standard_normal((9, 2))
    a = residual.relres_lowrank(M, A, D, C, V, Y, F1, F2)
    b = residual.relres_dense(M, A, D, C, V @ Y, F1 @ F2.T)
    assert abs(a - b) <= 1e-13 * b


@pytest.mark.parametrize("chunk", [1, 4, 9, 64])
def test_blockwise_residual_equals_dense_residual(chunk):
    """The block-by-block residual (for solutions too large to form) is the dense residual, for any block
    size; near the exact solution it resolves a relative residual at rounding level."""
    M, A = fem.tensor_operators(2, 6, kappa=0.8)
    D, C = timefe.time_matrices(9, 1.0)
    rng = np.random.default_rng(6)
    V = rng.standard_normal((36, 4))
    Y = rng.standard_normal((4, 9))
    F1, F2 = rng.standard_normal((36, 2)), rng.standard_normal((9, 2))
    a = residual.relres_lowrank_by_columns(M, A, D, C, V, Y, F1, F2, chunk=chunk)
    b = residual.relres_dense(M, A, D, C, V @ Y, F1 @ F2.T)
    assert abs(a - b) <= 1e-13 * b
    U = kron.solve_sparse(M, A, D, C, F1 @ F2.T)
    Uv, s_, Ut = np.linalg.svd(U, full_matrices=False)
    Vx, Yx = Uv * s_, Ut
    exact = residual.relres_lowrank_by_columns(M, A, D, C, Vx, Yx, F1, F2, chunk=chunk)
    assert exact <= 1e-13
    Yp = Yx + 1e-9 * rng.standard_normal(Yx.shape)
    pert = residual.relres_lowrank_by_columns(M, A, D, C, Vx, Yp, F1, F2, chunk=chunk)
    assert abs(pert - residual.relres_dense(M, A, D, C, Vx @ Yp, F1 @ F2.T)) <= 1e-6 * pert


# ---------------------------------------------------------------- RKSM reference


def test_rank_compression_of_manufactured_load_is_rank_one():
    F1, F2 = rhs.manufactured_loads(2, 9, 10)
    F1c, F2c = rksm.compress_rhs(F1, F2)
    assert F1c.shape[1] == 1
    assert np.allclose(F1c.T @ F1c, np.eye(1), atol=1e-14)
    assert np.allclose(F1c @ F2c.T, F1 @ F2.T, atol=1e-15 * np.abs(F1 @ F2.T).max() * 10)


@pytest.mark.parametrize("dim,n,nt,p", [(1, 31, 40, 2), (2, 11, 24, 2), (3, 5, 16, 3)])
def test_rksm_converges_to_exact_solution_with_galerkin_invariants(dim, n, nt, p):
    M, A = fem.tensor_operators(dim, n)
    D, C = timefe.time_matrices(nt, 1.0)
    F1, F2 = workloads.gaussian_factors(M.shape[0], nt, p, seed=7)
    out = rksm.rksm(M, A, D, C, F1, F2, tol=1e-12, maxit=200)
    V, Y = out["V"], out["Y"]
    U = kron.solve_sparse(M, A, D, C, F1 @ F2.T)
    assert out["converged"]
    assert np.linalg.norm(V.T @ V - np.eye(V.shape[1])) < 1e-12
    R = F1 @ F2.T - kron.apply(M, A, D, C, V @ Y)
    assert np.linalg.norm(V.T @ R) <= 1e-11 * np.linalg.norm(F1 @ F2.T)        # Galerkin condition
    assert np.linalg.norm(V @ Y - U) <= 1e-10 * np.linalg.norm(U)
    assert abs(out["history"][-1] - residual.relres_dense(M, A, D, C, V @ Y, F1 @ F2.T)) < 1e-13


def test_rksm_manufactured_load_converges_immediately():
    M, A = fem.tensor_operators(2, 15)
    D, C = timefe.time_matrices(16, 1.0)
    F1, F2 = rhs.manufactured_loads(2, 15, 16)
    out = rksm.rksm(M, A, D, C, F1, F2, tol=1e-12)
    assert out["V"].shape[1] == 1 and out["iterations"] == 0


def test_rational_arnoldi_spans_the_resolvent_space():
    """Reading (b): the newest-block recursion spans range[M^-1 F1, (A + s_j M)^-1 F1, ...]."""
    M, A = fem.tensor_operators(2, 8)
    D, C = timefe.time_matrices(10, 1.0)
    F1, F2 = workloads.gaussian_factors(64, 10, 1, seed=2)
    shifts = [30.0, 300.0, 90.0, 1500.0]
    out = rksm.rksm(M, A, D, C, F1, F2, tol=0.0, maxit=4, shifts=shifts)
    F1c, _ = rksm.compress_rhs(F1, F2)
    Md, Ad = M.toarray(), A.toarray()
    cols = [np.linalg.solve(Md, F1c)] + [np.linalg.solve(Ad + s * Md, F1c) for s in shifts]
    Q, _ = np.linalg.qr(np.hstack(cols))
    V = out["V"]
    ang = sla.subspace_angles(V, Q)
    assert V.shape[1] == 5 and ang.max() < 1e-8


def test_printed_space_misses_rough_load_solution():
    """Reading (a): seeded with F1 the space stalls for a Gaussian load; seeded with M^-1 F1 it converges."""
    M, A = fem.tensor_operators(2, 11)
    D, C = timefe.time_matrices(24, 1.0)
    F1, F2 = workloads.gaussian_factors(121, 24, 2, seed=2)
    lit = rksm.rksm(M, A, D, C, F1, F2, tol=1e-10, maxit=30, seed="F1")
    good = rksm.rksm(M, A, D, C, F1, F2, tol=1e-10, maxit=30, seed="Minv")
    assert lit["history"][-1] > 1e-4
    assert good["history"][-1] <= 1e-10


def test_table1_memory_accounting_matches_paper():
    """Table 1: mu_mem = Its + 1 for RKSM with a rank-1 load; the oracle counts the same way."""
    rows = [list(map(float, l.split())) for l in (GOLDEN / "table1.txt").read_text().splitlines()
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 6
    for r in rows:
        assert r[3] == r[2] + 1
    M, A = fem.tensor_operators(2, 9)
    D, C = timefe.time_matrices(12, 1.0)
    F1, F2 = workloads.gaussian_factors(81, 12, 1, seed=4)
    out = rksm.rksm(M, A, D, C, F1, F2, tol=1e-8)
    assert out["V"].shape[1] == out["iterations"] + 1


# ---------------------------------------------------------------- planted mistakes


def _cn_pin_error(time_matrices):
    n, nt = 7, 8
    M, A = fem.tensor_operators(1, n)
    D, C = time_matrices(nt, 1.0)
    g = rhs.sine_load_1d(n)[:, None]
    time_fn = lambda t: np.array([1 + t * t])
    Ft = rhs.trapezoidal_loads(g, time_fn, nt, 1.0)
    U_pg = kron.solve_sparse(M, A, D, C, Ft)
    nodes = np.array([g[:, 0] * time_fn(l / nt)[0] for l in range(nt + 1)]).T
    U_cn = textbook_cn(M, A, 1.0 / nt, nodes)
    return np.linalg.norm(U_pg - U_cn) / np.linalg.norm(U_cn)


def test_planted_time_matrix_mistakes_are_caught():
    assert _cn_pin_error(timefe.time_matrices) < 1e-13
    transposed = lambda nt, T: tuple(X.T.copy() for X in timefe.time_matrices(nt, T))
    assert _cn_pin_error(transposed) > 1e-3

    def wrong_sign(nt, T):
        D, C = timefe.time_matrices(nt, T)
        return D, np.diag(np.diag(C)) - (C - np.diag(np.diag(C)))
    assert _cn_pin_error(wrong_sign) > 1e-3


def test_planted_mass_mistake_is_caught(monkeypatch):
    good = fem.p1_mass_1d(7).toarray()
    monkeypatch.setattr(fem, "p1_mass_1d", lambda n, length=1.0: sp.csr_matrix(
        np.diag(np.full(n, 4.0 / 6.0 / (n + 1)))))     # dropped off-diagonal terms
    bad = fem.p1_mass_1d(7).toarray()
    assert not np.allclose(bad, quad_1d(7, 1.0, "M"), atol=1e-15)
    assert np.allclose(good, quad_1d(7, 1.0, "M"), atol=1e-15)


def test_cg_forward_substitution_equals_direct_elimination():
    """The CG variant of block forward substitution (used where a factorisation does not fit)
    reproduces the direct one on the first columns."""
    M, A = fem.tensor_operators(3, 9)
    D, C = timefe.time_matrices(7, 1.0)
    F1, F2 = workloads.gaussian_factors(M.shape[0], 7, 3, seed=1)
    U = kron.forward_substitution(M, A, D, C, F1 @ F2.T)
    Uc = kron.forward_substitution_cg(M, A, D, C, F1, F2, 3, rtol=1e-14)
    assert np.linalg.norm(Uc - U[:, :3]) <= 1e-12 * np.linalg.norm(U[:, :3])


def test_normal_equations_forward_substitution_matches_direct_elimination():
    """CG on the normal equations of each nonsymmetric block gives the direct elimination's first columns."""
    M, A = fem.tensor_operators(2, (9, 7), op="convdiff", eps=0.05, beta=(1.0, 0.5))
    D, C = timefe.time_matrices(6, 1.0)
    F1, F2 = workloads.gaussian_factors(M.shape[0], 6, 2, seed=4)
    assert abs(A - A.T).max() > 1e-3                      # the operator really is nonsymmetric
    U = kron.forward_substitution(M, A, D, C, F1 @ F2.T)
    Un = kron.forward_substitution_normal_cg(M, A, D, C, F1, F2, 3)
    assert np.linalg.norm(Un - U[:, :3]) <= 1e-11 * np.linalg.norm(U[:, :3])


# ---------------------------------------------------------------- P1 simplex meshes (general meshes)

@pytest.mark.parametrize("dim,n", [(2, 6), (3, 3)])
@pytest.mark.parametrize("jitter,flip", [(0.0, False), (0.25, True)])
def test_p1_simplex_operators_pins(dim, n, jitter, flip):
    """P1 assembly on a jittered simplex mesh: the full mass matrix integrates 1 to the domain's measure, the
    full stiffness matrix annihilates constants, and linear functions are harmonic at interior nodes (no
    interior load for a linear solution); M and A share one sparsity pattern."""
    import workloads
    msh = workloads.simplex_mesh(dim, n, seed=1, jitter=jitter, flip=flip)
    Mf, Af = fem.p1_simplex_operators(msh["nodes"], msh["elems"], msh["interior"], full=True)
    one = np.ones(Mf.shape[0])
    assert abs(one @ Mf @ one - 1.0) <= 1e-13
    assert np.abs(Af @ one).max() <= 1e-13
    lin = msh["nodes"] @ np.arange(1.0, dim + 1.0) + 0.3
    assert np.abs((Af @ lin)[msh["interior"]]).max() <= 1e-12
    M, A = fem.p1_simplex_operators(msh["nodes"], msh["elems"], msh["interior"], kappa=0.7)
    assert M.shape == (n ** dim, n ** dim)
    assert np.array_equal(M.indptr, A.indptr) and np.array_equal(M.indices, A.indices)
    assert abs((A - A.T)).max() <= 1e-15 and np.linalg.eigvalsh(A.toarray()).min() > 0
    assert np.linalg.eigvalsh(M.toarray()).min() > 0


@pytest.mark.parametrize("dim,n", [(2, 7), (3, 4)])
def test_p1_on_the_regular_simplex_mesh_is_the_finite_difference_stencil(dim, n):
    """Textbook closed form: on the right-triangle (Kuhn-tetrahedron) mesh of a uniform grid, the P1 stiffness
    matrix is h^(d-2) times the (2d+1)-point difference Laplacian (2d on the diagonal, -1 to the axis
    neighbours, 0 across the cell diagonals), and the mass matrix's diagonal is h^d/2 (2D) or 2h^3/5 (3D)."""
    import workloads
    msh = workloads.simplex_mesh(dim, n, seed=1, jitter=0.0, flip=False)
    M, A = fem.p1_simplex_operators(msh["nodes"], msh["elems"], msh["interior"])
    h = 1.0 / (n + 1)
    K1 = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1])
    I = sp.identity(n)
    lap = sp.kron(I, K1) + sp.kron(K1, I) if dim == 2 else \
        sp.kron(sp.kron(I, I), K1) + sp.kron(sp.kron(I, K1), I) + sp.kron(sp.kron(K1, I), I)
    assert abs(A - h ** (dim - 2) * lap).max() <= 1e-13
    assert np.allclose(M.diagonal(), (0.5 if dim == 2 else 0.4) * h ** dim, rtol=1e-13, atol=0)
