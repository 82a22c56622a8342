"""LR-FGMRES+RKSM on the GPU (st_solve_lrfgmres; Section 5, Example 1, Table 1's comparison solver) against the
CPU oracle: the converged solution against the direct Kronecker solve and the oracle's own LR-FGMRES+RKSM
solution, the exact residual of the returned factors, and Table 1's pattern (a few outer steps, several times
RKSM's stored columns)."""

import numpy as np
import pytest
import torch

import paper_1912_10082_gb300 as st
from oracle import fem, kron, lrfgmres, residual, rksm, timefe
import workloads

pytestmark = pytest.mark.gpu


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dim,n,nt,p,seed", [(2, 15, 24, 2, 41), (2, (21, 13), 16, 1, 42), (3, 7, 12, 2, 43)])
def test_lrfgmres_matches_direct_solution_and_oracle(dim, n, nt, p, seed):
    M, A = fem.tensor_operators(dim, n, kappa=0.7)
    D, C = timefe.time_matrices(nt, 1.0)
    F1, F2 = workloads.gaussian_factors(M.shape[0], nt, p, seed=seed)
    U_ref = kron.solve_sparse(M, A, D, C, F1 @ F2.T)
    tol = 1e-10
    with st.Problem(dim, n, nt, 1.0, kappa=0.7, tol=tol) as prob:
        V, Y, stats, status = prob.solve_lrfgmres(np.asfortranarray(F1), np.asfortranarray(F2), maxit=40,
                                                  precond_iters=5, trunc=1e-12)
        Vh, Yh = V.cpu().numpy(), Y.cpu().numpy()
    assert status == st.ST_OK and stats["converged"] == 1
    U = Vh @ Yh
    assert relerr(U, U_ref) <= 1e-8
    # the exact residual of the returned factors, formed by the oracle
    true_res = residual.relres_lowrank(M, A, D, C, Vh, Yh, F1, F2)
    assert true_res <= 20 * tol, (true_res, stats["relres"])
    # the oracle's LR-FGMRES+RKSM on the same problem converges to the same solution in a comparable count
    ref = lrfgmres.lr_fgmres(M, A, D, C, F1, F2, tol=tol, maxit=40, precond_iters=5, trunc=1e-12)
    assert relerr(U, ref["P"] @ ref["Q"].T) <= 1e-8
    assert abs(stats["iterations"] - ref["iterations"]) <= 2, (stats["iterations"], ref["iterations"])
    assert stats["inner_iterations"] >= stats["iterations"]


def test_lrfgmres_table1_pattern_on_a_non_modal_load():
    """Example 1's time profile with a Gaussian-bump space factor on a uniform grid of (-1,1)^3 (the oracle
    tests' stand-in for the unstructured meshes): LR-FGMRES+RKSM takes a few outer steps and stores several
    times the columns RKSM does, as in Table 1."""
    n, nt = 7, 40
    L = 2.0
    M, A = fem.tensor_operators(3, n, length=L)
    D, C = timefe.time_matrices(nt, 10.0)
    x = -1.0 + L * np.arange(1, n + 1) / (n + 1)
    g = np.exp(-((x[:, None, None] - 0.2) / 0.35) ** 2 - ((x[None, :, None] + 0.1) / 0.35) ** 2
               - ((x[None, None, :] - 0.3) / 0.35) ** 2)
    F1 = (M @ g.transpose(2, 1, 0).reshape(-1))[:, None]
    t = np.linspace(0.0, 10.0, nt + 1)
    F2 = np.array([10.0 * (np.sin(b) - b * np.cos(b) - np.sin(a) + a * np.cos(a)) for a, b in zip(t[:-1], t[1:])])[:, None]
    U_ref = kron.solve_sparse(M, A, D, C, F1 @ F2.T)
    with st.Problem(3, n, nt, 10.0, length=(L, L, L), tol=1e-8) as prob:
        V, Y, s_lr, status = prob.solve_lrfgmres(np.asfortranarray(F1), np.asfortranarray(F2), maxit=30)
        U = (V @ Y).cpu().numpy()
        _, _, s_rk, st_rk = prob.solve(np.asfortranarray(F1), np.asfortranarray(F2))
    assert status == st.ST_OK and st_rk == st.ST_OK
    assert relerr(U, U_ref) <= 1e-6
    assert s_lr["iterations"] <= 6
    assert s_lr["mu_mem"] >= 2 * s_rk["mu_mem"], (s_lr["mu_mem"], s_rk["mu_mem"])


def test_lrfgmres_zero_load_and_bad_arguments():
    with st.Problem(2, 9, 8, 1.0) as prob:
        F1 = np.zeros((81, 1), order="F")
        F2 = np.ones((8, 1), order="F")
        V, Y, stats, status = prob.solve_lrfgmres(F1, F2)
        assert status == st.ST_OK and V.shape[1] == 0 and stats["converged"] == 1
        L = st.lib()
        assert L.st_solve_lrfgmres(prob.h, F1.ctypes.data, 81, F2.ctypes.data, 8, 1, 0, 5, 1e-12, None, None) == st.ST_EINVAL
        assert L.st_solve_lrfgmres(prob.h, F1.ctypes.data, 80, F2.ctypes.data, 8, 1, 5, 5, 1e-12, None, None) == st.ST_EINVAL
