"""Lock-step batched RKSM (st_solve_batch) against st_solve and the CPU oracle.

Every problem of a mixed batch (2D and 3D grids, ragged sizes, several kappa,
time-grid lengths and load ranks, FP64 and mixed precision, plus problems the
grouped path leaves to the one-by-one driver) must give what st_solve gives on
the same problem -- the same iterations, basis and numbers -- and match the
oracle's direct solve of the assembled space-time system (paper Section 3,
eqs. par1/par2) to 1e-8 (FP64) or 1e-6 (mixed), in total and per time column.
A problem solved alone in a batch of one gives the numbers it gives in the mix.
"""

import numpy as np
import pytest
import torch

import paper_1912_10082_gb300 as st
from oracle import fem, kron, residual, timefe
import workloads

pytestmark = pytest.mark.gpu


def make_cases(seed=31):
    rng = np.random.default_rng(seed)
    shapes = [(2, 7), (2, 15), (2, 23), (2, 31), (3, 5), (3, 9), (2, (13, 6)), (3, (7, 5, 4))]
    cases = []
    for i, (dim, n) in enumerate(shapes * 2):
        nt = int(rng.choice([6, 13, 24, 40]))
        p = int(rng.choice([1, 2, 3]))
        kappa = float(10.0 ** rng.uniform(-1, 1))
        ns = [n] * dim if np.isscalar(n) else list(n)
        nh = int(np.prod(ns))
        F1, F2 = workloads.gaussian_factors(nh, nt, p, seed=500 + i)
        cases.append(dict(dim=dim, n=ns, n_t=nt, kappa=kappa, F1=np.asfortranarray(F1), F2=np.asfortranarray(F2)))
    return cases


def oracle_solution(c, op="heat", eps=1.0, beta=(0.0, 0.0, 0.0)):
    if op == "heat":
        M, A = fem.tensor_operators(c["dim"], c["n"], kappa=c["kappa"])
    else:
        M, A = fem.tensor_operators(c["dim"], c["n"], op="convdiff", eps=eps, beta=beta)
    D, C = timefe.time_matrices(c["n_t"], 1.0)
    return kron.solve_sparse(M, A, D, C, c["F1"] @ c["F2"].T)


def dev(a):
    t = torch.empty((a.shape[1], a.shape[0]), dtype=torch.float64, device="cuda").t()
    t.copy_(torch.from_numpy(np.ascontiguousarray(a)))
    return t


def dense(V, Y):
    return (V @ Y).cpu().numpy() if V.shape[1] else np.zeros((V.shape[0], Y.shape[1]))


def column_errors(U, ref):
    num = np.linalg.norm(U - ref, axis=0)
    den = np.linalg.norm(ref, axis=0)
    return num / np.maximum(den, 1e-300 + np.max(den) * 1e-12)


@pytest.mark.parametrize("prec,tol,err_tol", [(st.ST_FP64, 1e-12, 1e-8), (st.ST_MIXED, 1e-10, 1e-6)])
def test_batch_matches_single_solves_and_oracle(prec, tol, err_tol):
    cases = make_cases()
    probs = [st.Problem(c["dim"], c["n"], c["n_t"], 1.0, c["kappa"], precision=prec, tol=tol, maxit=300)
             for c in cases]
    # host loads for half the problems, device loads for the rest
    F1s = [c["F1"] if i % 2 else dev(c["F1"]) for i, c in enumerate(cases)]
    F2s = [c["F2"] if i % 2 else dev(c["F2"]) for i, c in enumerate(cases)]
    try:
        res, bs = st.solve_batch(probs, F1s, F2s)
        torch.cuda.synchronize()
        assert bs["grouped"] == len(cases) and bs["rounds"] >= 1 and bs["grouped_launches"] > 0
        Ub = []
        for i, (V, Y, stats, status) in enumerate(res):
            assert status == st.ST_OK, (i, status, stats)
            Ub.append(dense(V, Y))
            assert stats["relres"] <= tol
        # the same problems one by one through st_solve on twin handles
        for i, c in enumerate(cases):
            with st.Problem(c["dim"], c["n"], c["n_t"], 1.0, c["kappa"], precision=prec, tol=tol,
                            maxit=300) as twin:
                V, Y, stats, status = twin.solve(c["F1"], c["F2"])
                torch.cuda.synchronize()
                assert status == st.ST_OK
                assert stats["iterations"] == res[i][2]["iterations"], i
                assert stats["basis_cols"] == res[i][2]["basis_cols"], i
                # the same basis and coefficients, bit for bit
                assert torch.equal(V, res[i][0]) and torch.equal(Y, res[i][1]), i
                # the reported residual is rounding-level at the last check (about 1e-13 and below); its host
                # evaluation may round differently in its last digits
                assert abs(stats["relres"] - res[i][2]["relres"]) <= 1e-6 * stats["relres"] + 1e-20, i
        for i, c in enumerate(cases):
            ref = oracle_solution(c)
            err = np.linalg.norm(Ub[i] - ref) / np.linalg.norm(ref)
            assert err <= err_tol, (i, err)
            # per time column: an early column must not hide under the large late ones
            assert np.max(column_errors(Ub[i], ref)) <= 10 * err_tol, (i, np.max(column_errors(Ub[i], ref)))
    finally:
        for p in probs:
            p.close()


def test_problem_alone_and_in_the_mix_agree():
    cases = make_cases(seed=32)[:9]
    probs = [st.Problem(c["dim"], c["n"], c["n_t"], 1.0, c["kappa"], precision=st.ST_MIXED, tol=1e-10, maxit=300)
             for c in cases]
    try:
        res, _ = st.solve_batch(probs, [c["F1"] for c in cases], [c["F2"] for c in cases])
        mix = [dense(V, Y) for V, Y, _, _ in res]
        for i in (0, 4, 8):
            alone, _ = st.solve_batch([probs[i]], [cases[i]["F1"]], [cases[i]["F2"]])
            assert np.array_equal(dense(alone[0][0], alone[0][1]), mix[i]), i
    finally:
        for p in probs:
            p.close()


def test_batch_sends_other_problems_to_the_one_by_one_driver():
    """1D, convection-diffusion and a zero load sit beside grouped problems; all are solved as st_solve would."""
    rng = np.random.default_rng(7)
    c1 = dict(dim=1, n=[63], n_t=20, kappa=0.7)
    c1["F1"], c1["F2"] = (np.asfortranarray(x) for x in workloads.gaussian_factors(63, 20, 2, seed=1))
    c2 = dict(dim=2, n=[15, 15], n_t=12, kappa=1.0)
    c2["F1"], c2["F2"] = (np.asfortranarray(x) for x in workloads.gaussian_factors(225, 12, 2, seed=2))
    c3 = dict(dim=2, n=[11, 11], n_t=10, kappa=2.0)
    c3["F1"] = np.zeros((121, 1), order="F")
    c3["F2"] = np.asfortranarray(rng.standard_normal((10, 1)))
    c4 = dict(dim=2, n=[9, 9], n_t=8, kappa=1.5)
    c4["F1"], c4["F2"] = (np.asfortranarray(x) for x in workloads.gaussian_factors(81, 8, 2, seed=4))
    probs = [st.Problem(1, 63, 20, 1.0, 0.7, tol=1e-12),
             st.Problem(2, 15, 12, 1.0, op=st.ST_CONVDIFF, eps=0.1, beta=(1.0, 0.5), tol=1e-12),
             st.Problem(2, 11, 10, 1.0, 2.0, tol=1e-12),
             st.Problem(2, 9, 8, 1.0, 1.5, tol=1e-12)]
    try:
        res, bs = st.solve_batch(probs, [c["F1"] for c in (c1, c2, c3, c4)], [c["F2"] for c in (c1, c2, c3, c4)])
        assert bs["grouped"] == 2
        assert all(r[3] == st.ST_OK for r in res), [r[3] for r in res]
        refs = [oracle_solution(c1), oracle_solution(c2, op="convdiff", eps=0.1, beta=(1.0, 0.5)), None,
                oracle_solution(c4)]
        for i in (0, 1, 3):
            U = dense(res[i][0], res[i][1])
            assert np.linalg.norm(U - refs[i]) <= 1e-8 * np.linalg.norm(refs[i]), i
        assert res[2][0].shape[1] == 0 and res[2][2]["converged"] == 1   # F = 0: U = 0
    finally:
        for p in probs:
            p.close()


def test_batch_rejects_a_handle_given_twice():
    with st.Problem(2, 9, 8, 1.0) as p:
        F1, F2 = workloads.gaussian_factors(81, 8, 1, seed=5)
        F1, F2 = np.asfortranarray(F1), np.asfortranarray(F2)
        with pytest.raises(st.StError) as e:
            st.solve_batch([p, p], [F1, F1], [F2, F2])
        assert e.value.status == st.ST_EINVAL


def test_batch_fills_dense_outputs():
    cases = make_cases(seed=33)[:4]
    probs = [st.Problem(c["dim"], c["n"], c["n_t"], 1.0, c["kappa"], tol=1e-12, maxit=300) for c in cases]
    try:
        Us = [st.empty_colmajor(p.n_h, p.n_t) for p in probs]
        res, _ = st.solve_batch(probs, [c["F1"] for c in cases], [c["F2"] for c in cases], U_dense=Us)
        torch.cuda.synchronize()
        for i, (V, Y, _, status) in enumerate(res):
            assert status == st.ST_OK
            assert np.allclose(Us[i].cpu().numpy(), dense(V, Y), rtol=0, atol=1e-14 * float(Us[i].abs().max()))
    finally:
        for p in probs:
            p.close()



def test_batch_tensor_core_mode_products_match_oracle():
    """Mixed precision batch of 16-column problems whose long directions (folded length 128 and more, 64+ tiles
    a launch) take the tensor-core (3xTF32) tiles for the mode products, beside a problem that stays on the SIMT
    tiles; the same numbers as st_solve on each problem, and the oracle's direct solve."""
    rng = np.random.default_rng(41)
    shapes = [(2, [255, 255]), (2, [257, 131]), (3, [255, 20, 8]), (2, [63, 63])]
    cases = []
    for i, (dim, ns) in enumerate(shapes):
        nt = 16   # rank 16 loads keep 16-column blocks
        nh = int(np.prod(ns))
        F1, F2 = workloads.gaussian_factors(nh, nt, 16, seed=700 + i)
        cases.append(dict(dim=dim, n=ns, n_t=nt, kappa=float(10.0 ** rng.uniform(-1, 1)),
                          F1=np.asfortranarray(F1), F2=np.asfortranarray(F2)))
    probs = [st.Problem(c["dim"], c["n"], c["n_t"], 1.0, c["kappa"], precision=st.ST_MIXED, tol=1e-10, maxit=300)
             for c in cases]
    try:
        res, bs = st.solve_batch(probs, [c["F1"] for c in cases], [c["F2"] for c in cases])
        torch.cuda.synchronize()
        assert bs["grouped"] == len(cases)
        for i, c in enumerate(cases):
            V, Y, stats, status = res[i]
            assert status == st.ST_OK and stats["relres"] <= 1e-10, (i, status, stats)
            with st.Problem(c["dim"], c["n"], c["n_t"], 1.0, c["kappa"], precision=st.ST_MIXED, tol=1e-10,
                            maxit=300) as twin:
                V1, Y1, s1, _ = twin.solve(c["F1"], c["F2"])
                torch.cuda.synchronize()
                assert s1["iterations"] == stats["iterations"] and torch.equal(V1, V) and torch.equal(Y1, Y), i
            U = dense(V, Y)
            M, A = fem.tensor_operators(c["dim"], c["n"], kappa=c["kappa"])
            D, C = timefe.time_matrices(c["n_t"], 1.0)
            ref = kron.forward_substitution(M, A, D, C, c["F1"] @ c["F2"].T)
            err = np.linalg.norm(U - ref) / np.linalg.norm(ref)
            assert err <= 1e-6, (i, err)
            assert np.max(column_errors(U, ref)) <= 1e-5, i
    finally:
        for p in probs:
            p.close()


@pytest.mark.parametrize("prec,tol", [(st.ST_MIXED, 1e-9), (st.ST_FP64, 1e-10)])
def test_batch_larger_grids_match_single_solves(prec, tol):
    """Grids whose mode products fill the 64 x 64 vector-read FP32 tiles of the grouped launches (the single
    solve picks its own tile shapes): the same basis and coefficients bit for bit, and the oracle's FP64 residual
    of the batched solution within the tolerance."""
    shapes = [(2, [127, 127]), (2, [200, 70]), (3, [70, 66, 9]), (2, [255, 64])]
    cases = []
    for i, (dim, ns) in enumerate(shapes):
        nt = [24, 13, 6, 9][i]
        F1, F2 = workloads.gaussian_factors(int(np.prod(ns)), nt, 2, seed=800 + i)
        cases.append(dict(dim=dim, n=ns, n_t=nt, kappa=[0.3, 1.0, 3.0, 0.7][i],
                          F1=np.asfortranarray(F1), F2=np.asfortranarray(F2)))
    probs = [st.Problem(c["dim"], c["n"], c["n_t"], 1.0, c["kappa"], precision=prec, tol=tol, maxit=300)
             for c in cases]
    try:
        res, bs = st.solve_batch(probs, [c["F1"] for c in cases], [c["F2"] for c in cases])
        torch.cuda.synchronize()
        assert bs["grouped"] == len(cases)
        for i, c in enumerate(cases):
            V, Y, stats, status = res[i]
            assert status == st.ST_OK, (i, status)
            with st.Problem(c["dim"], c["n"], c["n_t"], 1.0, c["kappa"], precision=prec, tol=tol,
                            maxit=300) as twin:
                V1, Y1, s1, _ = twin.solve(c["F1"], c["F2"])
                torch.cuda.synchronize()
                assert s1["iterations"] == stats["iterations"], i
                assert torch.equal(V1, V) and torch.equal(Y1, Y), i
            M, A = fem.tensor_operators(c["dim"], c["n"], kappa=c["kappa"])
            D, C = timefe.time_matrices(c["n_t"], 1.0)
            true_res = residual.relres_lowrank(M, A, D, C, V.cpu().numpy(), Y.cpu().numpy(), c["F1"], c["F2"])
            assert true_res <= 1.01 * tol, (i, true_res)
    finally:
        for p in probs:
            p.close()


def test_batch_mixes_precisions_and_stops_at_maxit_like_st_solve():
    """One batch holding FP64 and mixed-precision problems, some stopped by a small iteration limit: every problem
    gets st_solve's status, iterations and numbers (the not-converged best iterate included)."""
    cases = make_cases(seed=34)[:8]
    specs = [(st.ST_FP64 if i % 2 else st.ST_MIXED, 3 if i % 3 == 0 else 300) for i in range(len(cases))]
    probs = [st.Problem(c["dim"], c["n"], c["n_t"], 1.0, c["kappa"], precision=prec, tol=1e-11, maxit=mx)
             for c, (prec, mx) in zip(cases, specs)]
    try:
        res, bs = st.solve_batch(probs, [c["F1"] for c in cases], [c["F2"] for c in cases])
        torch.cuda.synchronize()
        assert bs["grouped"] == len(cases)
        for i, (c, (prec, mx)) in enumerate(zip(cases, specs)):
            V, Y, stats, status = res[i]
            with st.Problem(c["dim"], c["n"], c["n_t"], 1.0, c["kappa"], precision=prec, tol=1e-11, maxit=mx) as twin:
                V1, Y1, s1, st1 = twin.solve(c["F1"], c["F2"], ok=(st.ST_OK, st.ST_ENOTCONV))
                torch.cuda.synchronize()
                assert st1 == status, (i, st1, status)
                assert s1["iterations"] == stats["iterations"] and s1["converged"] == stats["converged"], i
                assert torch.equal(V1, V) and torch.equal(Y1, Y), i
            if mx == 3:
                assert status == st.ST_ENOTCONV and stats["iterations"] == 3, (i, status, stats["iterations"])
            else:
                assert status == st.ST_OK
                ref = oracle_solution(c)
                assert np.linalg.norm(dense(V, Y) - ref) <= (1e-8 if prec == st.ST_FP64 else 1e-6) * np.linalg.norm(ref)
    finally:
        for p in probs:
            p.close()


def test_batch_of_one_and_empty_batch():
    c = make_cases(seed=35)[1]
    with st.Problem(c["dim"], c["n"], c["n_t"], 1.0, c["kappa"], tol=1e-12) as p:
        res, bs = st.solve_batch([p], [c["F1"]], [c["F2"]])
        assert bs["grouped"] == 1 and res[0][3] == st.ST_OK
        assert np.linalg.norm(dense(res[0][0], res[0][1]) - oracle_solution(c)) <= 1e-8 * np.linalg.norm(oracle_solution(c))
    res, bs = st.solve_batch([], [], [])
    assert res == [] and bs["instances"] == 0
