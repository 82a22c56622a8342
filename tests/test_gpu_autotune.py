"""st_autotune: launch variants picked by timing on the GPU change how the shifted solves run, never what they
compute.

Each case solves with the built-in launch choices, tunes the problem's shapes (fast-diagonalisation mode products,
x-line solves), and solves again through the tuned choices; both results are held to the oracle's bar: the sparse
direct solve on small grids, the residual of the resolvent equation (A + sM) W = M X on grids too large for a
direct solve, and the exact low-rank residual for full RKSM solves.  Every test leaves the process-wide table empty.
"""

import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

import paper_1912_10082_gb300 as st
from oracle import cn, fem, kron, residual, timefe
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def empty_table():
    st.autotune_reset()
    yield
    st.autotune_reset()


def dev(a):
    a = np.asarray(a)
    t = torch.empty((a.shape[1], a.shape[0]), dtype=torch.float64, device="cuda").t()
    t.copy_(torch.from_numpy(np.ascontiguousarray(a)))
    return t


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def col_residuals(M, A, s, X, W):
    B = M @ X
    R = B - (A @ W + s * (M @ W))
    return np.linalg.norm(R, axis=0) / np.linalg.norm(B, axis=0)


@pytest.mark.parametrize("dim,n", [(2, (40, 37)), (3, (35, 18, 5))])
@pytest.mark.parametrize("prec,tol", [(st.ST_FP64, 1e-12), (st.ST_MIXED, 1e-10)])
def test_tuned_heat_shift_solve_matches_sparse_lu(dim, n, prec, tol):
    M, A = fem.tensor_operators(dim, n, kappa=0.8)
    X = np.random.default_rng(21).standard_normal((M.shape[0], 3))
    s = 250.0
    ref = np.linalg.solve((A + s * M).toarray(), M @ X)
    with st.Problem(dim, n, 4, 1.0, kappa=0.8) as prob:
        before = host(prob.shift_solve(s, dev(X), precision=prec))
        added = prob.autotune(3.0, 3, precision=prec)
        assert added > 0 and st.autotune_count() == added
        assert prob.autotune(3.0, 3, precision=prec) == 0   # every shape is in the table now
        after = host(prob.shift_solve(s, dev(X), precision=prec))
    assert relerr(before, ref) <= tol
    assert relerr(after, ref) <= tol
    assert relerr(after, before) <= tol


@pytest.mark.parametrize("dim,n,eps", [(1, 31, 0.05), (2, (40, 21), 0.01), (3, (33, 9, 5), 0.05)])
@pytest.mark.parametrize("prec", [st.ST_FP64, st.ST_MIXED])
def test_tuned_convdiff_shift_solve_matches_sparse_lu(dim, n, eps, prec):
    """x-line preconditioned FGMRES: the line solve runs in place in 2D and 3D, out of place in 1D."""
    beta = (1.0, 0.5, 0.25)[:dim]
    M, A = fem.tensor_operators(dim, n, op="convdiff", eps=eps, beta=beta)
    X = np.random.default_rng(22).standard_normal((M.shape[0], 4))
    s = 40.0
    ref = np.linalg.solve((A + s * M).toarray(), M @ X)
    with st.Problem(dim, n, 4, 1.0, op=st.ST_CONVDIFF, eps=eps, beta=beta) as prob:
        added = prob.autotune(s, 4, precision=prec)
        assert added > 0
        out = host(prob.shift_solve(s, dev(X), precision=prec))
    assert np.all(col_residuals(M, A, s, X, out) <= 5e-12)
    assert relerr(out, ref) <= 1e-8


@pytest.mark.parametrize("dim,n,op", [(2, (255, 255), "heat"), (3, (63, 63, 63), "heat"),
                                      (2, (255, 200), "convdiff"), (3, (63, 40, 30), "convdiff")])
@pytest.mark.parametrize("prec", [st.ST_FP64, st.ST_MIXED])
def test_tuned_shift_solve_at_benchmark_sizes(dim, n, op, prec):
    """Grid sides of the benchmark workloads: the tuned solve against the built-in launch choices.

    The mode-product variants sum in the same order, so heat results agree to rounding; the line-solve variants
    round differently, so the convection-diffusion solves (FGMRES to 1e-12 per column) agree to about cond(A + sM)
    times that.  Neither residual may grow.  On the 2D heat grid both are also checked against the oracle's sparse
    LU solve (whose own forward error is up to cond(A + sM) u, about 1e-12 here).
    """
    if op == "convdiff":
        beta = (1.0, 0.5, 0.25)[:dim]
        M, A = fem.tensor_operators(dim, n, op="convdiff", eps=0.02, beta=beta)
        kw = dict(op=st.ST_CONVDIFF, eps=0.02, beta=beta)
    else:
        M, A = fem.tensor_operators(dim, n)
        kw = {}
    X = np.random.default_rng(23).standard_normal((M.shape[0], 2))
    s = 30.0
    with st.Problem(dim, n, 4, 1.0, **kw) as prob:
        before = host(prob.shift_solve(s, dev(X), precision=prec))
        assert prob.autotune(s, 2, precision=prec) > 0
        after = host(prob.shift_solve(s, dev(X), precision=prec))
    r0, r1 = col_residuals(M, A, s, X, before), col_residuals(M, A, s, X, after)
    if op == "heat":
        assert relerr(after, before) <= (1e-12 if prec == st.ST_FP64 else 1e-9)
        assert np.all(r1 <= 2 * r0 + 1e-15), (r0, r1)
    else:
        assert relerr(after, before) <= 1e-6
        assert np.all(r1 <= np.maximum(4 * r0, 5e-12)), (r0, r1)
    if op == "heat" and dim == 2:
        ref = spla.splu((A + s * M).tocsc()).solve(M @ X)
        assert relerr(before, ref) <= 1e-10 and relerr(after, ref) <= 1e-10


@pytest.mark.parametrize("dim,n,nt,p,op", [(2, 15, 32, 2, "heat"), (3, 7, 16, 3, "heat"),
                                           (2, (40, 21), 12, 2, "convdiff")])
@pytest.mark.parametrize("prec", [st.ST_FP64, st.ST_MIXED])
def test_tuned_rksm_solve_matches_direct_solution(dim, n, nt, p, op, prec):
    beta = (1.0, 0.5, 0.25)[:dim]
    if op == "convdiff":
        M, A = fem.tensor_operators(dim, n, op="convdiff", eps=0.05, beta=beta)
        kw = dict(op=st.ST_CONVDIFF, eps=0.05, beta=beta)
    else:
        M, A = fem.tensor_operators(dim, n)
        kw = {}
    D, C = timefe.time_matrices(nt, 1.0)
    F1, F2 = workloads.gaussian_factors(M.shape[0], nt, p, seed=24)
    ref = kron.solve_sparse(M, A, D, C, F1 @ F2.T)
    tol = 1e-11 if prec == st.ST_FP64 else 1e-10
    with st.Problem(dim, n, nt, 1.0, precision=prec, tol=tol, maxit=300, **kw) as prob:
        assert prob.autotune(10.0, p, precision=prec) > 0
        Ud = st.empty_colmajor(prob.n_h, prob.n_t)
        V, Y, stats, status = prob.solve(dev(F1), dev(F2), U_dense=Ud)
        U, Vh, Yh = host(Ud), host(V), host(Y)
    assert status == st.ST_OK and stats["converged"] == 1
    assert relerr(U, ref) <= (1e-8 if prec == st.ST_FP64 else 1e-6)
    true_res = residual.relres_lowrank(M, A, D, C, Vh, Yh, F1, F2)
    assert true_res <= 10 * tol
    assert abs(stats["relres"] - true_res) <= 0.5 * true_res + 1e-11


def test_tuned_choices_inside_a_captured_cn_graph():
    """Crank-Nicolson records its steps in a CUDA graph: tuned shapes are looked up, never timed, in capture."""
    dim, n, nt = 2, 31, 24
    M, A = fem.tensor_operators(dim, n)
    F1, F2 = workloads.gaussian_factors(M.shape[0], nt, 2, seed=25)
    ref = cn.crank_nicolson(M, A, 1.0 / nt, F1 @ F2.T)
    with st.Problem(dim, n, nt, 1.0) as prob:
        assert prob.autotune(2.0 / prob.dt, 1) > 0
        out = host(prob.timestep_cn(dev(F1), dev(F2)))
    assert relerr(out, ref) <= 1e-12


def test_tuning_cache_round_trip(tmp_path):
    """Choices tuned on this GPU, saved, forgotten and loaded again drive the same (bitwise equal) heat solve."""
    dim, n, s = 2, (45, 38), 40.0
    M, A = fem.tensor_operators(dim, n)
    X = np.random.default_rng(26).standard_normal((M.shape[0], 2))
    ref = np.linalg.solve((A + s * M).toarray(), M @ X)
    path = tmp_path / "tune.txt"
    with st.Problem(dim, n, 4, 1.0) as prob:
        added = prob.autotune(s, 2)
        tuned = host(prob.shift_solve(s, dev(X)))
        st.autotune_save(path)
        st.autotune_reset()
        assert st.autotune_load(path, "another device") == 0 and st.autotune_count() == 0
        assert st.autotune_load(path) == added and st.autotune_count() == added
        loaded = host(prob.shift_solve(s, dev(X)))
    assert relerr(tuned, ref) <= 1e-12
    assert np.array_equal(tuned, loaded)


def test_autotune_rejects_bad_arguments():
    L = st.lib()
    with st.Problem(2, 9, 4, 1.0) as prob:
        assert L.st_autotune(prob.h, 1.0, 0, st.ST_FP64, None) == st.ST_EINVAL
        assert L.st_autotune(prob.h, 1.0, 17, st.ST_FP64, None) == st.ST_EINVAL
        assert L.st_autotune(prob.h, 1.0, 2, 7, None) == st.ST_EINVAL
        assert L.st_autotune(prob.h, -1e9, 2, st.ST_FP64, None) == st.ST_EINVAL
        assert L.st_autotune(None, 1.0, 2, st.ST_FP64, None) == st.ST_EINVAL
    assert st.autotune_count() == 0
