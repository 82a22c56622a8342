"""Pins of the wave-equation oracle (oracle/wave.py; paper Section 3 "The Wave Equation", Section 4 eq. 3terms,
Section 5 Example 2) against what the mathematics fixes: the textbook Gram matrices of uniform cubic B-splines,
the symmetry and positivity of B, the Kronecker form against the matrix form, the preconditioner's inverse, and
second-order convergence to Example 2's solution u = t^2 sin(2 pi x)."""

import numpy as np
import pytest

from oracle import wave


def interior_row(Mat, n):
    i = n // 2
    return Mat[i, i - 3:i + 4]


def test_cubic_bspline_gram_matrices_are_the_textbook_ones():
    """Interior rows on a uniform grid of spacing h: (B_i, B_j) = h (1, 120, 1191, 2416, ...)/5040,
    (B_i', B_j') = (-1/120, -1/5, -1/8, 2/3, ...)/h, (B_i'', B_j'') = (1/6, 0, -3/2, 8/3, ...)/h^3 (the
    symmetric seven-term stencils of the degree-6 B-spline and its derivatives at the integers)."""
    n = 14
    h = 1.0 / n
    Mh, Ah, Qh, Mt, Dt, Qt = wave.wave_matrices(n, n, 1.0)
    m = np.array([1, 120, 1191, 2416, 1191, 120, 1]) / 5040.0
    k = np.array([-1 / 120, -1 / 5, -1 / 8, 2 / 3, -1 / 8, -1 / 5, -1 / 120])
    q = np.array([1 / 6, 0.0, -1.5, 8 / 3, -1.5, 0.0, 1 / 6])
    assert np.allclose(interior_row(Mh, n), h * m, rtol=1e-12, atol=1e-15)
    assert np.allclose(interior_row(Ah, n), k / h, rtol=1e-12, atol=1e-12)
    assert np.allclose(interior_row(Qh, n), q / h ** 3, rtol=1e-12, atol=1e-9)
    # the same stencils in time on (0, T) with T = 2: spacing 2/n
    Mh2, _, _, Mt2, Dt2, Qt2 = wave.wave_matrices(n, n, 2.0)
    assert np.allclose(interior_row(Mt2, n), (2.0 / n) * m, rtol=1e-12, atol=1e-15)
    assert np.allclose(interior_row(Qt2, n), q / (2.0 / n) ** 3, rtol=1e-12, atol=1e-9)
    # ((rho^k)'', rho^l) = -((rho^k)', (rho^l)') in the interior (integration by parts, rows away from T)
    assert np.allclose(interior_row(Dt2, n), -k / (2.0 / n), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("nx,nt", [(5, 7), (9, 4)])
def test_the_space_time_matrix_is_symmetric_positive_definite_and_matches_the_matrix_form(nx, nt):
    mats = wave.wave_matrices(nx, nt, 1.0)
    B = wave.assemble(*mats).toarray()
    assert B.shape == ((nx + 1) * (nt + 1),) * 2
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    assert np.linalg.eigvalsh(B).min() > 0
    U = np.random.default_rng(1).standard_normal((nx + 1, nt + 1))
    via_kron = (B @ U.reshape(-1, order="F")).reshape(U.shape, order="F")
    assert np.allclose(wave.apply(*mats, U), via_kron, rtol=1e-12, atol=1e-10 * np.abs(via_kron).max())


def test_the_preconditioner_inverse_by_diagonalisation():
    Mh, Ah, Qh, Mt, Dt, Qt = wave.wave_matrices(11, 9, 1.0)
    P = wave.Lyap(Mh, Qh, Mt, Qt)
    V = np.random.default_rng(2).standard_normal(Mh.shape[:1] + Mt.shape[:1])
    W = P.solve(V)
    assert np.linalg.norm(P.apply(W) - V) <= 1e-11 * np.linalg.norm(V)


def example2(n):
    mats = wave.wave_matrices(n, n, 1.0)
    # f = (2 + 4 pi^2 t^2) sin(2 pi x) makes u = t^2 sin(2 pi x) exact (u_tt - u_xx)
    F1, F2 = wave.load_factors(n, n, 1.0, [lambda x: np.sin(2 * np.pi * x)] * 2,
                               [lambda t: 2.0 + 0.0 * t, lambda t: 4.0 * np.pi ** 2 * t ** 2])
    return mats, F1 @ F2.T


def test_example2_converges_at_second_order():
    x = np.linspace(0.01, 0.99, 57)
    t = np.linspace(0.01, 0.99, 53)
    exact = t[:, None] ** 2 * np.sin(2 * np.pi * x)[None, :]
    errs = []
    for n in (8, 16, 32):
        mats, F = example2(n)
        U = wave.solve_direct(*mats, F)
        errs.append(np.abs(wave.evaluate(U, n, n, 1.0, x, t) - exact).max())
    assert errs[2] <= 5e-3
    assert errs[0] / errs[1] >= 3.5 and errs[1] / errs[2] >= 3.5, errs


def test_gmres_lyap_reaches_the_direct_solution():
    mats, F = example2(16)
    U = wave.solve_direct(*mats, F)
    r = wave.gmres_lyap(*mats, F, tol=1e-11, maxit=300)
    assert np.linalg.norm(r["U"] - U) <= 1e-9 * np.linalg.norm(U)
    assert r["history"][-1] <= 1e-11 and 10 <= r["iterations"] <= 150
    # the estimate is the true preconditioned-system residual
    res = np.linalg.norm(wave.apply(*mats, r["U"]) - F) / np.linalg.norm(F)
    assert res <= 1e-10
