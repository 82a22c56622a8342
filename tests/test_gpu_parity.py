"""GPU path against the CPU oracle, through the C ABI (paper Sections 3-5).

Tolerances: index work bit-exact; assembled FP64 values exact (same operation
order, no fused multiply-add); FP64 kernels within a small multiple of the
rounding of the longest dot product; FP64 solves to 1e-8 relative error and
mixed solves to 1e-6 (the stated targets), run at tighter residual tolerances.
"""

import numpy as np
import scipy.sparse.linalg as spla
import pytest
import torch

import paper_1912_10082_gb300 as st
from oracle import cn, fem, kron, residual, rhs, rksm, timefe
import workloads

pytestmark = pytest.mark.gpu


def dev(a, dtype=torch.float64):
    a = np.asarray(a)
    if a.ndim == 1:
        a = a[:, None]
    t = torch.empty((a.shape[1], a.shape[0]), dtype=dtype, device="cuda").t()
    t.copy_(torch.from_numpy(np.ascontiguousarray(a)).to(dtype))
    return t


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def colerr(a, b):
    """Largest relative error of a time column (columns whose reference is below 1e-12 of the largest column
    norm are measured against that floor), so an early, small column cannot hide under the late ones."""
    num = np.linalg.norm(a - b, axis=0)
    den = np.linalg.norm(b, axis=0)
    return float(np.max(num / np.maximum(den, 1e-12 * den.max() + 1e-300)))


def ops(dim, n, kappa=1.0, length=None, **kw):
    return fem.tensor_operators(dim, n, kappa=kappa, length=length if length is not None else 1.0, **kw)


# ---------------------------------------------------------------- A0 set-up

@pytest.mark.parametrize("dim,n,kw", [
    (1, 7, {}), (1, 1, {}), (2, (5, 3), {"length": (1.0, 2.0)}), (3, (4, 3, 2), {}), (3, 9, {"kappa": 0.37}),
    (2, 6, {"op": "convdiff", "eps": 0.05, "beta": (1.0, 0.5)}),
    (3, 4, {"op": "convdiff", "eps": 0.2, "beta": (1.0, 0.5, 0.25)}),
])
def test_setup_csr_matches_oracle(dim, n, kw):
    kw = dict(kw)
    op = kw.pop("op", "heat")
    length = kw.pop("length", None)
    if op == "convdiff":
        M, A = fem.tensor_operators(dim, n, op="convdiff", eps=kw["eps"], beta=kw["beta"])
        prob = st.Problem(dim, n, 5, 1.0, op=st.ST_CONVDIFF, eps=kw["eps"], beta=kw["beta"])
    else:
        M, A = fem.tensor_operators(dim, n, kappa=kw.get("kappa", 1.0), length=length or 1.0)
        prob = st.Problem(dim, n, 5, 1.0, kappa=kw.get("kappa", 1.0), length=length)
    with prob:
        rp, col, mv, av = prob.get_csr()
    Ms = M.tocsr()
    Ms.sort_indices()
    assert np.array_equal(rp, Ms.indptr) and np.array_equal(col, Ms.indices)
    assert np.array_equal(mv, Ms.data)
    # A on the pattern of M: the 3D Q1 stiffness has exact zeros (face neighbours)
    # that scipy drops from its own pattern
    rows = np.repeat(np.arange(Ms.shape[0]), np.diff(Ms.indptr))
    a_on_m = np.asarray(A.tocsr()[rows, Ms.indices]).ravel()
    assert np.max(np.abs(av - a_on_m)) <= 1e-15 * np.max(np.abs(a_on_m))


# ---------------------------------------------------------------- A2 fused apply (K1)

@pytest.mark.parametrize("dim,n,nt,pad", [(1, 13, 5, 0), (2, 7, 33, 3), (2, 33, 100, 0), (3, 6, 17, 1), (1, 1, 1, 0),
                                         # several CTA tiles a direction, ragged edges, n_t not a multiple of 8
                                         (3, (65, 37, 19), 45, 5), (2, (300, 70), 77, 0), (3, (97, 9, 8), 9, 0),
                                         # 2D FP32 time pairs: interior CTAs in y and time (unchecked loads),
                                         # full and ragged 15-column chunks, a single column
                                         (2, (200, 130), 46, 2), (2, 64, 15, 0), (2, (61, 97), 31, 1),
                                         (2, 40, 1, 0)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_apply_matches_kronecker_form(dim, n, nt, pad, dtype):
    M, A = ops(dim, n, kappa=1.3)
    D, C = timefe.time_matrices(nt, 0.7)
    U = np.random.default_rng(1).standard_normal((M.shape[0], nt))
    ref = kron.apply(M, A, D, C, U)
    with st.Problem(dim, n, nt, 0.7, kappa=1.3) as prob:
        Ud = torch.zeros((nt, M.shape[0] + pad), dtype=dtype, device="cuda").t()[: M.shape[0]]
        Ud.copy_(torch.from_numpy(U).to(dtype))
        Yd = prob.apply(Ud)
        out = host(Yd)
    tol = 1e-14 if dtype == torch.float64 else 2e-6
    assert relerr(out, ref) <= tol


@pytest.mark.parametrize("dim,n,nt,kw", [
    (2, (70, 45), 33, {"op": "convdiff", "eps": 0.05, "beta": (1.0, 0.5)}),
    (3, (40, 21, 13), 20, {"op": "convdiff", "eps": 0.2, "beta": (1.0, 0.5, 0.25)}),
    (2, (66, 80), 17, {"length": (1.0, 2.5)}),
    (3, (35, 12, 9), 16, {"length": (1.0, 0.5, 2.0)}),
])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_apply_convdiff_and_box_lengths_match_kronecker_form(dim, n, nt, kw, dtype):
    """The box kernels on non-symmetric (convection) and anisotropic (unequal box sides) 1D factors: the 2D
    stencil from the assembled rows, the 3D FP32 sum factorisation from the 1D factors."""
    if kw.get("op") == "convdiff":
        M, A = fem.tensor_operators(dim, n, op="convdiff", eps=kw["eps"], beta=kw["beta"])
        prob = st.Problem(dim, n, nt, 0.9, op=st.ST_CONVDIFF, eps=kw["eps"], beta=kw["beta"])
    else:
        M, A = fem.tensor_operators(dim, n, kappa=0.8, length=kw["length"])
        prob = st.Problem(dim, n, nt, 0.9, kappa=0.8, length=kw["length"])
    D, C = timefe.time_matrices(nt, 0.9)
    U = np.random.default_rng(3).standard_normal((M.shape[0], nt))
    ref = kron.apply(M, A, D, C, U)
    with prob:
        Ud = torch.from_numpy(U).to(dtype).cuda().t().contiguous().t()
        out = host(prob.apply(Ud))
    tol = 1e-14 if dtype == torch.float64 else 2e-6
    assert relerr(out, ref) <= tol


def test_apply_user_csr_generic_rows():
    """User CSR with rows longer than 27 goes through the generic kernel."""
    rng = np.random.default_rng(2)
    n, nt = 40, 9
    Md = np.eye(n) * 2 + (rng.random((n, n)) < 0.8) * rng.random((n, n)) * 0.01
    Md = 0.5 * (Md + Md.T)
    Ad = Md * 3 + np.eye(n)
    import scipy.sparse as sp
    M = sp.csr_matrix(Md)
    A = sp.csr_matrix(Ad)
    A = (A + 0 * M).tocsr()
    M = (M + 0 * A).tocsr()
    M.sort_indices(); A.sort_indices()
    assert np.array_equal(M.indices, A.indices)
    D, C = timefe.time_matrices(nt, 1.0)
    U = rng.standard_normal((n, nt))
    with st.Problem(0, 1, nt, 1.0, csr=(M.indptr, M.indices, M.data, A.data)) as prob:
        out = host(prob.apply(dev(U)))
    assert relerr(out, kron.apply(M, A, D, C, U)) <= 1e-14


# ---------------------------------------------------------------- A0 manufactured loads

@pytest.mark.parametrize("dim,n,nt", [(1, 63, 64), (2, 31, 20), (3, 7, 9)])
def test_manufactured_loads_match_oracle(dim, n, nt):
    F1, F2 = rhs.manufactured_loads(dim, n, nt)
    with st.Problem(dim, n, nt, 1.0) as prob:
        f1, f2 = prob.rhs_manufactured()
        f1, f2 = host(f1), host(f2)
    assert relerr(f1, F1) <= 1e-14 and relerr(f2, F2) <= 1e-14


# ---------------------------------------------------------------- A3 shifted solve (K2)

@pytest.mark.parametrize("dim,n", [(1, 15), (2, (9, 6)), (3, 5), (3, (4, 6, 3)), (2, (40, 37)), (3, (35, 18, 5))])
@pytest.mark.parametrize("prec,tol", [(st.ST_FP64, 1e-12), (st.ST_MIXED, 1e-10)])
def test_shift_solve_matches_sparse_lu(dim, n, prec, tol):
    M, A = ops(dim, n, kappa=0.8)
    X = np.random.default_rng(4).standard_normal((M.shape[0], 3))
    for s in (3.0, 250.0, 1e5):
        ref = np.linalg.solve((A + s * M).toarray(), M @ X)
        with st.Problem(dim, n, 4, 1.0, kappa=0.8) as prob:
            out = host(prob.shift_solve(s, dev(X), precision=prec))
        assert relerr(out, ref) <= tol, (s, relerr(out, ref))


@pytest.mark.parametrize("dim,n", [(2, (255, 255)), (2, (257, 131)), (3, (255, 7, 6))])
def test_shift_solve_many_columns_tensor_core_tiles(dim, n):
    """64 columns: the FP32 mode products along the 255+ point directions take the tensor-core (3xTF32) tiles,
    the others the SIMT tiles; mixed precision (FP32 transform, FP64 refinement) against a sparse LU solve."""
    M, A = ops(dim, n, kappa=0.8)
    X = np.random.default_rng(5).standard_normal((M.shape[0], 64))
    for s in (3.0, 1e4):
        ref = spla.splu((A + s * M).tocsc()).solve(M @ X)
        with st.Problem(dim, n, 4, 1.0, kappa=0.8) as prob:
            out = host(prob.shift_solve(s, dev(X), precision=st.ST_MIXED))
        assert relerr(out, ref) <= 1e-10, (s, relerr(out, ref))


@pytest.mark.parametrize("dim,n,eps", [(1, 31, 0.05), (2, (40, 21), 0.01), (2, 15, 0.5), (3, (33, 9, 5), 0.05)])
@pytest.mark.parametrize("prec", [st.ST_FP64, st.ST_MIXED])
def test_shift_solve_convdiff_matches_sparse_lu(dim, n, eps, prec):
    """Convection-diffusion resolvent: batched flexible GMRES (five columns advanced together)."""
    beta = (1.0, 0.5, 0.25)[:dim]
    M, A = fem.tensor_operators(dim, n, op="convdiff", eps=eps, beta=beta)
    X = np.random.default_rng(6).standard_normal((M.shape[0], 5))
    X[:, 3] = 0.0   # a zero column converges at once
    for s in (0.3, 40.0, 1e4):
        ref = np.linalg.solve((A + s * M).toarray(), M @ X)
        with st.Problem(dim, n, 4, 1.0, op=st.ST_CONVDIFF, eps=eps, beta=beta) as prob:
            out = host(prob.shift_solve(s, dev(X), precision=prec))
        assert np.all(out[:, 3] == 0.0)
        # each column stops at a relative residual of 1e-12; the error is at most cond(A + sM) times that
        K, B = (A + s * M).toarray(), M @ X
        for j in (0, 1, 2, 4):
            res = np.linalg.norm(B[:, j] - K @ out[:, j]) / np.linalg.norm(B[:, j])
            assert res <= 5e-12, (s, j, res)
        assert relerr(out, ref) <= 1e-8, (s, relerr(out, ref))


@pytest.mark.parametrize("dim,n", [(2, (384, 345)), (3, (60, 50, 45))])
def test_shift_solve_convdiff_iterative_refinement(dim, n):
    """Mixed precision on a grid of at least 2^17 points: FP32 inner FGMRES cycles refined on the FP64 residual."""
    beta = (1.0, 0.5, 0.25)[:dim]
    eps = 0.02
    M, A = fem.tensor_operators(dim, n, op="convdiff", eps=eps, beta=beta)
    assert M.shape[0] >= 1 << 17
    X = np.random.default_rng(8).standard_normal((M.shape[0], 3))
    for s in (0.5, 200.0):
        with st.Problem(dim, n, 4, 1.0, op=st.ST_CONVDIFF, eps=eps, beta=beta) as prob:
            out = host(prob.shift_solve(s, dev(X), precision=st.ST_MIXED))
        B = M @ X
        R = B - (A @ out + s * (M @ out))
        for j in range(3):
            res = np.linalg.norm(R[:, j]) / np.linalg.norm(B[:, j])
            assert res <= 5e-12, (s, j, res)


def test_solve_convdiff_large_grid_mixed_residual():
    """RKSM with FP32-refined FGMRES resolvents: the oracle's exact residual of the returned (V, Y)."""
    dim, n, nt, eps = 2, (384, 345), 16, 0.05
    beta = (1.0, 0.5)
    M, A = fem.tensor_operators(dim, n, op="convdiff", eps=eps, beta=beta)
    D, C = timefe.time_matrices(nt, 1.0)
    F1, F2 = workloads.gaussian_factors(M.shape[0], nt, 2, seed=19)
    tol = 1e-9
    with st.Problem(dim, n, nt, 1.0, op=st.ST_CONVDIFF, eps=eps, beta=beta, precision=st.ST_MIXED, tol=tol,
                    maxit=300) as prob:
        V, Y, stats, status = prob.solve(dev(F1), dev(F2))
        Vh, Yh = host(V), host(Y)
    assert status == st.ST_OK and stats["converged"] == 1
    true_res = residual.relres_lowrank(M, A, D, C, Vh, Yh, F1, F2)
    assert true_res <= 10 * tol
    assert abs(stats["relres"] - true_res) <= 0.5 * true_res + 1e-11


# ---------------------------------------------------------------- A10 Crank-Nicolson (K10)

@pytest.mark.parametrize("dim,n,nt,p", [(1, 63, 64, 2), (2, 15, 40, 3), (3, 7, 12, 1)])
def test_cn_matches_oracle_forward_substitution(dim, n, nt, p):
    M, A = ops(dim, n)
    D, C = timefe.time_matrices(nt, 1.0)
    F1, F2 = workloads.gaussian_factors(M.shape[0], nt, p, seed=5)
    ref = cn.crank_nicolson(M, A, 1.0 / nt, F1 @ F2.T)
    with st.Problem(dim, n, nt, 1.0) as prob:
        U = prob.timestep_cn(dev(F1), dev(F2))
        U2 = prob.timestep_cn(F1.copy(order="F"), F2.copy(order="F"))   # host inputs, cached graph
        out, out2 = host(U), host(U2)
    assert relerr(out, ref) <= 1e-12
    assert np.array_equal(out, out2)


# ---------------------------------------------------------------- st_solve (A1-A9)

@pytest.mark.parametrize("dim,n,nt,p,seed", [(1, 63, 64, 2, 1), (2, 15, 32, 2, 2), (2, (12, 9), 20, 3, 3),
                                             (3, 7, 16, 4, 4)])
@pytest.mark.parametrize("prec", [st.ST_FP64, st.ST_MIXED])
def test_solve_matches_direct_solution(dim, n, nt, p, seed, prec):
    M, A = ops(dim, n)
    D, C = timefe.time_matrices(nt, 1.0)
    F1, F2 = workloads.gaussian_factors(M.shape[0], nt, p, seed=seed)
    ref = kron.solve_sparse(M, A, D, C, F1 @ F2.T)
    tol = 1e-12 if prec == st.ST_FP64 else 1e-10
    with st.Problem(dim, n, nt, 1.0, precision=prec, tol=tol, maxit=300) as prob:
        Ud = st.empty_colmajor(prob.n_h, prob.n_t)
        V, Y, stats, status = prob.solve(dev(F1), dev(F2), U_dense=Ud)
        U, Vh, Yh = host(Ud), host(V), host(Y)
    assert status == st.ST_OK and stats["converged"] == 1
    err_tol = 1e-8 if prec == st.ST_FP64 else 1e-6
    assert relerr(U, ref) <= err_tol
    assert colerr(U, ref) <= 10 * err_tol
    assert np.allclose(U, Vh @ Yh, rtol=1e-12, atol=1e-14 * np.abs(U).max())
    # the residual the solver reports agrees with the oracle's exact residual of (V, Y)
    true_res = residual.relres_lowrank(M, A, D, C, Vh, Yh, F1, F2)
    assert true_res <= 10 * tol
    # the reported residual is exact up to the rounding of the rational Arnoldi relation: FP64 basis
    # products in FP64 mode; in mixed mode they carry about 48 bits (double-float), a floor near 1e-11
    floor = 1e-14 if prec == st.ST_FP64 else 1e-11
    assert abs(stats["relres"] - true_res) <= 0.5 * true_res + floor
    assert np.linalg.norm(Vh.T @ Vh - np.eye(Vh.shape[1])) < 1e-10


@pytest.mark.parametrize("dim,n,nt,eps", [(1, 31, 24, 0.05), (2, 15, 16, 0.05), (2, (12, 9), 20, 0.5),
                                           (3, 7, 10, 0.2), (2, (40, 21), 12, 0.05), (3, (33, 9, 5), 8, 0.2)])
@pytest.mark.parametrize("prec", [st.ST_FP64, st.ST_MIXED])
def test_solve_convdiff_matches_direct_solution(dim, n, nt, eps, prec):
    """Convection-diffusion (nonsymmetric A): FGMRES shifted solves, unsymmetrised projections."""
    beta = (1.0, 0.5, 0.25)[:dim]
    M, A = fem.tensor_operators(dim, n, op="convdiff", eps=eps, beta=beta)
    D, C = timefe.time_matrices(nt, 1.0)
    F1, F2 = workloads.gaussian_factors(M.shape[0], nt, 2, seed=17)
    ref = kron.solve_sparse(M, A, D, C, F1 @ F2.T)
    tol = 1e-11 if prec == st.ST_FP64 else 1e-10
    with st.Problem(dim, n, nt, 1.0, op=st.ST_CONVDIFF, eps=eps, beta=beta, precision=prec, tol=tol,
                    maxit=300) as prob:
        Ud = st.empty_colmajor(prob.n_h, prob.n_t)
        V, Y, stats, status = prob.solve(dev(F1), dev(F2), U_dense=Ud)
        U, Vh, Yh = host(Ud), host(V), host(Y)
    assert status == st.ST_OK and stats["converged"] == 1 and stats["inner_iterations"] > 0
    if dim == 1 and prec == st.ST_FP64:
        # in 1D the x-line preconditioner is the shifted operator itself: about one FGMRES step a column
        assert stats["inner_iterations"] <= 2 * 2 * stats["iterations"] + 4, stats
    assert relerr(U, ref) <= (1e-8 if prec == st.ST_FP64 else 1e-6)
    assert colerr(U, ref) <= 10 * (1e-8 if prec == st.ST_FP64 else 1e-6)
    true_res = residual.relres_lowrank(M, A, D, C, Vh, Yh, F1, F2)
    assert true_res <= 10 * tol
    assert abs(stats["relres"] - true_res) <= 0.5 * true_res + 1e-11


@pytest.mark.parametrize("dim,n,nt", [(1, 63, 64), (2, 31, 40), (3, 9, 12)])
def test_solve_manufactured_is_exact_in_one_block(dim, n, nt):
    M, A = ops(dim, n)
    D, C = timefe.time_matrices(nt, 1.0)
    F1, F2 = rhs.manufactured_loads(dim, n, nt)
    ref = kron.solve_sparse(M, A, D, C, F1 @ F2.T)
    with st.Problem(dim, n, nt, 1.0, tol=1e-12) as prob:
        f1, f2 = prob.rhs_manufactured()
        Ud = st.empty_colmajor(prob.n_h, prob.n_t)
        V, Y, stats, status = prob.solve(f1, f2, U_dense=Ud)
        U = host(Ud)
    assert status == st.ST_OK and stats["p"] == 1 and stats["basis_cols"] == 1
    assert relerr(U, ref) <= 1e-12


def test_solve_rank1_memory_accounting():
    """mu_mem = iterations + 1 for a rank-1 load, as in the paper's Table 1."""
    M, A = ops(2, 15)
    F1, F2 = workloads.gaussian_factors(M.shape[0], 24, 1, seed=9)
    with st.Problem(2, 15, 24, 1.0, tol=1e-8) as prob:
        _, _, stats, status = prob.solve(dev(F1), dev(F2))
    assert status == st.ST_OK
    assert stats["mu_mem"] == stats["iterations"] + 1
    assert stats["basis_cols"] == stats["iterations"]


@pytest.mark.parametrize("prec,tol,err_tol", [(st.ST_FP64, 1e-12, 1e-8), (st.ST_MIXED, 1e-10, 1e-6)])
def test_solve_load_with_more_columns_than_time_steps(prec, tol, err_tol):
    """F1 F2^T with 12 columns on a 4-step time grid (rank at most 4): the rank compression keeps the time
    factor's 4 directions; single and batched solves against the oracle's direct solve."""
    for dim, n in ((2, (15, 11)), (3, (6, 5, 4))):
        M, A = ops(dim, n, kappa=0.9)
        D, C = timefe.time_matrices(4, 1.0)
        F1, F2 = workloads.gaussian_factors(M.shape[0], 4, 12, seed=6)
        F1, F2 = np.asfortranarray(F1), np.asfortranarray(F2)
        ref = kron.solve_sparse(M, A, D, C, F1 @ F2.T)
        with st.Problem(dim, n, 4, 1.0, kappa=0.9, precision=prec, tol=tol) as prob:
            V, Y, stats, status = prob.solve(dev(F1), dev(F2))
            assert status == st.ST_OK and stats["p"] <= 4, stats
            assert relerr(host(V @ Y), ref) <= err_tol
            res, _ = st.solve_batch([prob], [F1], [F2])
            assert res[0][3] == st.ST_OK
            assert relerr(host(res[0][0] @ res[0][1]), ref) <= err_tol


def test_solve_zero_load_and_bad_arguments():
    with st.Problem(2, 7, 6, 1.0) as prob:
        V, Y, stats, status = prob.solve(dev(np.zeros((49, 2))), dev(np.ones((6, 2))))
        assert status == st.ST_OK and stats["basis_cols"] == 0
        with pytest.raises(st.StError):
            prob.solve(dev(np.ones((48, 2))), dev(np.ones((6, 2))))   # ld < n_h
    with pytest.raises(st.StError):
        st.Problem(2, 7, 0, 1.0)


def test_solve_not_converged_returns_best_iterate():
    M, A = ops(2, 15)
    F1, F2 = workloads.gaussian_factors(M.shape[0], 32, 2, seed=3)
    with st.Problem(2, 15, 32, 1.0, tol=1e-14, maxit=2) as prob:
        V, Y, stats, status = prob.solve(dev(F1), dev(F2), ok=(st.ST_OK, st.ST_ENOTCONV))
    assert status == st.ST_ENOTCONV and stats["converged"] == 0 and stats["iterations"] == 2


def test_solve_refuses_non_finite_loads():
    """A NaN in F1 (device) or an Inf in F2 (host) is refused with ST_EINVAL and a message, never solved as F = 0;
    the handle then solves a finite load."""
    F1, F2 = workloads.gaussian_factors(15 * 15, 16, 2, seed=30)
    F1n = F1.copy()
    F1n[7, 1] = np.nan
    F2i = np.asfortranarray(F2.copy())
    F2i[3, 0] = np.inf
    with st.Problem(2, 15, 16, 1.0) as prob:
        for a, b in ((dev(F1n), dev(F2)), (dev(F1), F2i)):
            with pytest.raises(st.StError) as e:
                prob.solve(a, b)
            assert e.value.status == st.ST_EINVAL and "NaN or Inf" in str(e.value)
        V, Y, stats, status = prob.solve(dev(F1), dev(F2))
    assert status == st.ST_OK and stats["converged"] == 1 and stats["basis_cols"] > 0


# ---------------------------------------------------------------- residual entry points

def test_residual_entry_points_match_oracle():
    M, A = ops(2, 9)
    D, C = timefe.time_matrices(11, 1.0)
    rng = np.random.default_rng(8)
    V, Y = rng.standard_normal((81, 5)), rng.standard_normal((5, 11))
    F1, F2 = rng.standard_normal((81, 2)), rng.standard_normal((11, 2))
    want = residual.relres_lowrank(M, A, D, C, V, Y, F1, F2)
    with st.Problem(2, 9, 11, 1.0) as prob:
        r_lr = prob.residual_lowrank(dev(V), dev(Y), dev(F1), dev(F2))
        r_dense = prob.residual(dev(V @ Y), dev(F1), dev(F2))
    assert abs(r_lr - want) <= 1e-12 * want
    assert abs(r_dense - want) <= 1e-12 * want


def test_residual_lowrank_rank_deficient_factors():
    """Repeated load columns and a one-mode basis (the manufactured case) still give the exact residual."""
    dim, n, nt = 2, 15, 12
    M, A = ops(dim, n)
    D, C = timefe.time_matrices(nt, 1.0)
    F1, F2 = rhs.manufactured_loads(dim, n, nt)
    Uex = kron.solve_sparse(M, A, D, C, F1 @ F2.T)
    V = Uex[:, :1] / np.linalg.norm(Uex[:, :1])
    Y = V.T @ Uex + 1e-3 * np.random.default_rng(0).standard_normal((1, nt))
    want = residual.relres_lowrank(M, A, D, C, V, Y, F1, F2)
    with st.Problem(dim, n, nt, 1.0) as prob:
        got = prob.residual_lowrank(dev(V), dev(Y), dev(F1), dev(F2))
        got0 = prob.residual_lowrank(dev(V), dev(V.T @ Uex), dev(F1), dev(F2))
    assert abs(got - want) <= 1e-10 * want
    assert got0 <= 1e-12


def test_residual_lowrank_large_rank_deficient_factor():
    """[F1, M V, A V] with F1 in range(M V) and more than 256 columns: the certification stays exact."""
    dim, n, nt, k = 2, 63, 40, 140
    M, A = ops(dim, n)
    D, C = timefe.time_matrices(nt, 1.0)
    rng = np.random.default_rng(12)
    V = np.linalg.qr(rng.standard_normal((n * n, k)))[0]
    Y = rng.standard_normal((k, nt)) * 0.1
    F1 = (M @ V[:, :2]) @ rng.standard_normal((2, 2))
    F2 = rng.standard_normal((nt, 2))
    want = residual.relres_lowrank(M, A, D, C, V, Y, F1, F2)
    with st.Problem(dim, n, nt, 1.0) as prob:
        got = prob.residual_lowrank(dev(V), dev(Y), dev(F1), dev(F2))
    assert abs(got - want) <= 1e-9 * want


# ---------------------------------------------------------------- full-size workload, sampled

@pytest.mark.slow
def test_heat2d_full_size_fp64_solve_and_cn():
    """2D Q1 255^2 x 256, manufactured load: RKSM and CN against the oracle's exact solution."""
    cfg = workloads.WORKLOADS["heat2d"]
    dim, n, nt = cfg["dim"], cfg["n"], cfg["n_t"]
    M, A = ops(dim, n)
    D, C = timefe.time_matrices(nt, 1.0)
    F1, F2 = rhs.manufactured_loads(dim, n, nt)
    ref = kron.forward_substitution(M, A, D, C, F1 @ F2.T)
    with st.Problem(dim, n, nt, 1.0, tol=1e-8) as prob:
        f1, f2 = prob.rhs_manufactured()
        Ud = st.empty_colmajor(prob.n_h, prob.n_t)
        V, Y, stats, status = prob.solve(f1, f2, U_dense=Ud)
        Ucn = prob.timestep_cn(f1, f2)
        U, Uc = host(Ud), host(Ucn)
    assert status == st.ST_OK
    assert relerr(U, ref) <= 1e-8
    assert relerr(Uc, ref) <= 1e-10
