"""General meshes: problems given as CSR matrices (P1 on seeded jittered simplex meshes of the unit square and cube,
assembled by the oracle) through the algebraic inner solver (Jacobi-preconditioned block CG) — the shifted solves
against sparse LU, and whole RKSM solves (paper Section 4) against the oracle's direct solve of the space-time
system and its exact residual of the returned factors."""

import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

import paper_1912_10082_gb300 as st
from oracle import fem, kron, residual, timefe
import workloads

pytestmark = pytest.mark.gpu


def mesh_ops(dim, n, seed=6, kappa=1.0):
    msh = workloads.simplex_mesh(dim, n, seed=seed)
    M, A = fem.p1_simplex_operators(msh["nodes"], msh["elems"], msh["interior"], kappa=kappa)
    assert np.array_equal(M.indptr, A.indptr) and np.array_equal(M.indices, A.indices)
    return M, A


def csr_problem(M, A, nt, **kw):
    return st.Problem(0, 1, nt, 1.0, csr=(M.indptr, M.indices, M.data, A.data), **kw)


def dev(a):
    t = torch.empty((a.shape[1], a.shape[0]), dtype=torch.float64, device="cuda").t()
    t.copy_(torch.from_numpy(np.ascontiguousarray(a)))
    return t


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dim,n", [(2, 20), (3, 6)])
def test_csr_shift_solve_matches_sparse_lu(dim, n):
    M, A = mesh_ops(dim, n, kappa=0.8)
    X = np.random.default_rng(4).standard_normal((M.shape[0], 5))
    with csr_problem(M, A, 4) as prob:
        for s in (1.0, 300.0):
            ref = spla.splu((A + s * M).tocsc()).solve(M @ X)
            out = prob.shift_solve(s, dev(X)).cpu().numpy()
            assert relerr(out, ref) <= 1e-10, (s, relerr(out, ref))


@pytest.mark.parametrize("dim,n,nt,p", [(2, 24, 16, 2), (3, 7, 12, 2), (2, 17, 9, 3)])
def test_csr_solve_matches_direct_solution(dim, n, nt, p):
    M, A = mesh_ops(dim, n, seed=7 + n, kappa=0.6)
    D, C = timefe.time_matrices(nt, 1.0)
    F1, F2 = workloads.gaussian_factors(M.shape[0], nt, p, seed=30 + n)
    F1, F2 = np.asfortranarray(F1), np.asfortranarray(F2)
    ref = kron.solve_sparse(M, A, D, C, F1 @ F2.T)
    with csr_problem(M, A, nt, tol=1e-10, maxit=300) as prob:
        V, Y, stats, status = prob.solve(dev(F1), dev(F2))
        Vh, Yh = V.cpu().numpy(), Y.cpu().numpy()
    assert status == st.ST_OK and stats["relres"] <= 1e-10, stats
    U = Vh @ Yh
    assert relerr(U, ref) <= 1e-8
    colerr = np.linalg.norm(U - ref, axis=0) / np.maximum(np.linalg.norm(ref, axis=0), 1e-300)
    assert colerr.max() <= 1e-7
    # the exact residual of the returned factors, formed by the oracle, against the solver's own estimate
    true_res = residual.relres_lowrank(M, A, D, C, Vh, Yh, F1, F2)
    assert true_res <= 1.01e-10 and abs(true_res - stats["relres"]) <= 1e-3 * true_res + 1e-13, \
        (true_res, stats["relres"])


def test_csr_problem_requested_in_mixed_precision_runs_in_fp64_and_in_a_batch_as_alone():
    M, A = mesh_ops(2, 15, seed=3)
    nt = 10
    F1, F2 = workloads.gaussian_factors(M.shape[0], nt, 2, seed=8)
    F1, F2 = np.asfortranarray(F1), np.asfortranarray(F2)
    with csr_problem(M, A, nt, tol=1e-11, precision=st.ST_FP64) as p64, \
            csr_problem(M, A, nt, tol=1e-11, precision=st.ST_MIXED) as pmx, \
            st.Problem(2, 9, 8, 1.0, tol=1e-11) as box:
        V, Y, s64, _ = p64.solve(dev(F1), dev(F2))
        V, Y = V.clone(), Y.clone()
        Vm, Ym, smx, _ = pmx.solve(dev(F1), dev(F2))
        assert torch.equal(V, Vm) and torch.equal(Y, Ym) and s64["iterations"] == smx["iterations"]
        G1, G2 = workloads.gaussian_factors(81, 8, 2, seed=9)
        res, bs = st.solve_batch([p64, box], [F1, np.asfortranarray(G1)], [F2, np.asfortranarray(G2)])
        assert bs["grouped"] == 1 and res[0][3] == st.ST_OK and res[1][3] == st.ST_OK
        assert torch.equal(res[0][0], V) and torch.equal(res[0][1], Y)


def test_csr_lrfgmres_matches_direct_solution_and_oracle():
    """LR-FGMRES+RKSM (Table 1's comparison solver) on a general mesh: the direct solve, the oracle's
    LR-FGMRES+RKSM solution, and the exact residual of the returned factors."""
    from oracle import lrfgmres
    M, A = mesh_ops(3, 6, seed=12, kappa=0.7)
    nt = 12
    D, C = timefe.time_matrices(nt, 1.0)
    F1, F2 = workloads.gaussian_factors(M.shape[0], nt, 2, seed=44)
    ref = kron.solve_sparse(M, A, D, C, F1 @ F2.T)
    tol = 1e-10
    with csr_problem(M, A, nt, tol=tol) as prob:
        V, Y, stats, status = prob.solve_lrfgmres(np.asfortranarray(F1), np.asfortranarray(F2), maxit=40,
                                                  precond_iters=5, trunc=1e-12)
        Vh, Yh = V.cpu().numpy(), Y.cpu().numpy()
    assert status == st.ST_OK and stats["converged"] == 1
    assert relerr(Vh @ Yh, ref) <= 1e-8
    assert residual.relres_lowrank(M, A, D, C, Vh, Yh, F1, F2) <= 20 * tol
    orc = lrfgmres.lr_fgmres(M, A, D, C, F1, F2, tol=tol, maxit=40, precond_iters=5, trunc=1e-12)
    assert relerr(Vh @ Yh, orc["P"] @ orc["Q"].T) <= 1e-8
