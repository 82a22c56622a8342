"""Many independent solves on one GPU (st_executor_*), against the CPU oracle.

Every result of a mixed batch is compared with the oracle's direct solve of the
assembled space-time system (paper Section 3, eqs. par1/par2); the same
requests solved alone give the same numbers as in the mix; and the HBM
admission rule keeps requests whose footprints do not fit together from
running at the same time.
"""

import time

import numpy as np
import pytest
import torch

import paper_1912_10082_gb300 as st
from oracle import fem, kron, timefe
import workloads

pytestmark = pytest.mark.gpu


def small_batch(count=12, seed=21):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice([7, 15, 23]))
        nt = int(rng.choice([8, 16, 24]))
        kappa = float(10.0 ** rng.uniform(-1, 1))
        F1, F2 = workloads.gaussian_factors(n * n, nt, 2, seed=100 + i)
        out.append(dict(n=n, n_t=nt, kappa=kappa, F1=np.asfortranarray(F1), F2=np.asfortranarray(F2)))
    return out


def oracle_solution(r):
    M, A = fem.tensor_operators(2, r["n"], kappa=r["kappa"])
    D, C = timefe.time_matrices(r["n_t"], 1.0)
    return kron.solve_sparse(M, A, D, C, r["F1"] @ r["F2"].T)


@pytest.mark.parametrize("prec,err_tol", [(st.ST_FP64, 1e-8), (st.ST_MIXED, 1e-6)])
def test_batch_results_match_oracle_and_solo_runs(prec, err_tol):
    reqs = small_batch()
    tol = 1e-12 if prec == st.ST_FP64 else 1e-10
    outs = [np.zeros((r["n"] ** 2, r["n_t"]), order="F") for r in reqs]
    with st.Executor(slots=6) as ex:
        for i, r in enumerate(reqs):
            d = st.make_desc(2, r["n"], r["n_t"], 1.0, r["kappa"], precision=prec, tol=tol, maxit=300)
            ex.submit(d, r["F1"], r["F2"], tag=i, U_out=outs[i])
        got = {}
        while len(got) < len(reqs):
            for res in ex.wait(64, timeout=1.0):
                got[res["tag"]] = res
    for i, r in enumerate(reqs):
        assert got[i]["status"] == st.ST_OK, got[i]
        ref = oracle_solution(r)
        err = np.linalg.norm(outs[i] - ref) / np.linalg.norm(ref)
        assert err <= err_tol, (i, err)
    # the same requests alone, one handle each: identical results
    for i in (0, 5, 11):
        r = reqs[i]
        with st.Problem(2, r["n"], r["n_t"], 1.0, r["kappa"], precision=prec, tol=tol, maxit=300) as prob:
            U = st.empty_colmajor(prob.n_h, prob.n_t)
            prob.solve(r["F1"], r["F2"], U_dense=U)
            solo = U.cpu().numpy()
        assert np.max(np.abs(solo - outs[i])) <= 1e-13 * np.max(np.abs(solo)), i


def test_batch_cn_requests_match_oracle():
    reqs = small_batch(count=6, seed=3)
    outs = [np.zeros((r["n"] ** 2, r["n_t"]), order="F") for r in reqs]
    with st.Executor(slots=3) as ex:
        for i, r in enumerate(reqs):
            d = st.make_desc(2, r["n"], r["n_t"], 1.0, r["kappa"])
            ex.submit(d, r["F1"], r["F2"], tag=i, U_out=outs[i], method=st.ST_METHOD_CN)
        got = []
        while len(got) < len(reqs):
            got += ex.wait(64, timeout=1.0)
    assert all(g["status"] == st.ST_OK for g in got)
    for i, r in enumerate(reqs):
        ref = oracle_solution(r)
        assert np.linalg.norm(outs[i] - ref) / np.linalg.norm(ref) <= 1e-10


def test_admission_keeps_oversubscribed_requests_apart():
    """A budget that holds one request at a time serialises the requests."""
    reqs = small_batch(count=5, seed=4)
    d0 = st.make_desc(2, 23, 24, 1.0)
    one = st.request_bytes(d0, 2)
    with st.Executor(slots=4, hbm_budget_bytes=1.5 * one) as ex:
        for i, r in enumerate(reqs):
            d = st.make_desc(2, 23, 24, 1.0, r["kappa"])
            F1, F2 = workloads.gaussian_factors(23 * 23, 24, 2, seed=i)
            ex.submit(d, np.asfortranarray(F1), np.asfortranarray(F2), tag=i)
        got = []
        while len(got) < len(reqs):
            got += ex.wait(64, timeout=1.0)
    assert all(g["status"] == st.ST_OK for g in got)
    spans = sorted((g["t_start"], g["t_end"]) for g in got)
    for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
        assert b0 >= a1 - 1e-6


def test_request_larger_than_budget_runs_alone():
    d = st.make_desc(2, 15, 16, 1.0)
    F1, F2 = workloads.gaussian_factors(225, 16, 2, seed=7)
    with st.Executor(slots=2, hbm_budget_bytes=1024.0) as ex:
        ex.submit(d, np.asfortranarray(F1), np.asfortranarray(F2), tag=1)
        got = []
        while not got:
            got = ex.wait(4, timeout=1.0)
    assert got[0]["status"] == st.ST_OK and got[0]["stats"]["converged"] == 1


def test_set_coefficients_matches_fresh_setup():
    F1, F2 = workloads.gaussian_factors(15 * 15, 12, 2, seed=8)
    F1, F2 = np.asfortranarray(F1), np.asfortranarray(F2)
    with st.Problem(2, 15, 12, 1.0, kappa=0.3, tol=1e-12) as a, st.Problem(2, 15, 12, 1.0, kappa=4.0,
                                                                                 tol=1e-12) as b:
        a.set_coefficients(st.ST_HEAT, kappa=4.0)
        ra, rb = a.get_csr(), b.get_csr()
        for x, y in zip(ra, rb):
            assert np.array_equal(x, y)
        Ua, Ub = st.empty_colmajor(225, 12), st.empty_colmajor(225, 12)
        a.solve(F1, F2, U_dense=Ua)
        b.solve(F1, F2, U_dense=Ub)
        assert torch.equal(Ua, Ub)
        # Crank-Nicolson: the graph captured before the change is updated in place
        a2 = st.Problem(2, 15, 12, 1.0, kappa=0.3)
        with a2:
            U0 = a2.timestep_cn(F1, F2)
            a2.set_coefficients(st.ST_HEAT, kappa=4.0)
            Ua2 = a2.timestep_cn(F1, F2, U0)
            Ub2 = b.timestep_cn(F1, F2)
            torch.cuda.synchronize()
            assert torch.equal(Ua2, Ub2)


@pytest.mark.parametrize("policy", [st.ST_SCHED_FIFO, st.ST_SCHED_HRRN])
def test_admission_policy_orders_waiting_requests(policy):
    """One slot, busy with a long solve while a large request and three small ones queue up behind it:
    FIFO admits them in arrival order, HRRN admits the small ones (higher response ratio) first."""
    def req(n, nt, seed):
        F1, F2 = workloads.gaussian_factors(n * n, nt, 2, seed=seed)
        return st.make_desc(2, n, nt, 1.0, 1.0), np.asfortranarray(F1), np.asfortranarray(F2)

    blocker = req(127, 256, 1)
    big = req(63, 256, 2)
    small = [req(7, 8, 3 + i) for i in range(3)]
    with st.Executor(slots=1, policy=policy) as ex:
        ex.submit(*blocker, tag=0)
        t_end = time.monotonic() + 60.0
        while ex.pending()[0] > 0:   # the blocker is admitted before the others arrive
            assert time.monotonic() < t_end, "the first request was not admitted within 60 s"
            time.sleep(0.001)
        ex.submit(*big, tag=1)
        for i, s in enumerate(small):
            ex.submit(*s, tag=2 + i)
        got = {}
        while len(got) < 5:
            for res in ex.wait(8, timeout=1.0):
                got[res["tag"]] = res
    assert all(g["status"] == st.ST_OK for g in got.values())
    starts = {t: g["t_start"] for t, g in got.items()}
    assert all(starts[0] < starts[t] for t in range(1, 5))
    if policy == st.ST_SCHED_FIFO:
        assert all(starts[1] < starts[t] for t in range(2, 5))
    else:
        assert all(starts[t] < starts[1] for t in range(2, 5))


def test_set_policy_rejects_unknown_policy():
    with st.Executor(slots=1) as ex:
        with pytest.raises(st.StError):
            ex.set_policy(7)
