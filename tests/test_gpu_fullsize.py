"""The benchmark configurations at full size, checked on samples the oracle can compute.

* 3D heat, Q1 127^3 (N_h = 2,048,383), n_t = 512, rank-4 Gaussian load, mixed precision, tol 1e-8:
  the first two time columns of U = V Y against the oracle's block forward substitution with
  conjugate gradients (forward substitution fixes the first columns exactly whatever the later
  ones are), and the FP64 residual of the whole solution formed by the oracle from (V, Y).
* The batched workload (256 2D instances of mixed sizes, mixed precision) in the bench's launch
  configuration (one st_solve_batch call) and through the executor: every instance on the 63^2
  grid against the oracle's direct solve; a sample of the larger ones by the oracle's residual.
* 3D served requests (31^3 and 63^3, heat and convection-diffusion) on their first time columns.
* The served stream (heat and convection-diffusion): the requests of its opening stretch small
  enough for a direct oracle solve, replayed at their arrival times among the others.
Tolerance: 1e-6 relative error for mixed precision (the stated target).
"""

import numpy as np
import pytest
import torch

import paper_1912_10082_gb300 as st
from paper_1912_10082_gb300 import serve
from oracle import fem, kron, residual, timefe
import workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_heat3d_full_size_mixed_first_columns():
    cfg = workloads.WORKLOADS["heat3d"]
    dim, n, nt, p = cfg["dim"], cfg["n"], cfg["n_t"], cfg["p"]
    n_h = n ** dim
    F1, F2 = workloads.gaussian_factors(n_h, nt, p, cfg["seed"])
    with st.Problem(dim, n, nt, cfg["T"], precision=st.ST_MIXED, tol=1e-8, maxit=400) as prob:
        f1 = st.empty_colmajor(n_h, p)
        f1.copy_(torch.from_numpy(F1))
        f2 = st.empty_colmajor(nt, p)
        f2.copy_(torch.from_numpy(F2))
        V, Y, stats, status = prob.solve(f1, f2)
        U2 = (V @ Y[:, :2]).cpu().numpy()
        Vh, Yh = V.cpu().numpy(), Y.cpu().numpy()
    assert status == st.ST_OK and stats["relres"] <= 1e-8
    M, A = fem.tensor_operators(dim, n)
    D, C = timefe.time_matrices(nt, cfg["T"])
    ref = kron.forward_substitution_cg(M, A, D, C, F1, F2, 2, rtol=1e-13)
    err = np.linalg.norm(U2 - ref) / np.linalg.norm(ref)
    assert err <= 1e-6, err
    # the FP64 residual of the whole solution, formed from (V, Y) by the oracle (not the solver's estimate)
    true_res = residual.relres_lowrank_by_columns(M, A, D, C, Vh, Yh, F1, F2, chunk=32)
    assert true_res <= 1e-8 + 1e-10, true_res
    assert abs(true_res - stats["relres"]) <= 0.01 * true_res, (true_res, stats["relres"])


def test_batched_workload_sample_matches_oracle():
    cfg = workloads.WORKLOADS["batched"]
    insts = workloads.batched_instances(count=cfg["count"], seed=cfg["seed"], p=cfg["p"])
    for r in insts:
        r["F1"], r["F2"] = np.asfortranarray(r["F1"]), np.asfortranarray(r["F2"])
    sample = [i for i, r in enumerate(insts) if r["n"] == 63]
    outs = [np.zeros((r["n"] ** 2, r["n_t"]), order="F") if i in sample else None for i, r in enumerate(insts)]
    res = serve.run_batch(insts, precision=st.ST_MIXED, slots=16, outputs=outs)
    assert all(r["status"] == st.ST_OK for r in res["results"])
    assert len(sample) >= 40
    for i in sample:
        r = insts[i]
        M, A = fem.tensor_operators(2, r["n"], kappa=r["kappa"])
        D, C = timefe.time_matrices(r["n_t"], 1.0)
        ref = kron.forward_substitution(M, A, D, C, r["F1"] @ r["F2"].T)
        err = np.linalg.norm(outs[i] - ref) / np.linalg.norm(ref)
        assert err <= 1e-6, (i, err)


def test_batched_workload_through_the_grouped_solver():
    """The bench's launch configuration: all 256 instances in one st_solve_batch call, mixed precision.  Every
    63^2 instance against the oracle's direct solve (whole and per time column); a sample of the 127^2 and
    255^2 instances through the oracle's FP64 residual of their (V, Y)."""
    cfg = workloads.WORKLOADS["batched"]
    insts = workloads.batched_instances(count=cfg["count"], seed=cfg["seed"], p=cfg["p"])
    probs = [st.Problem(2, r["n"], r["n_t"], 1.0, r["kappa"], precision=st.ST_MIXED, tol=1e-8, maxit=400)
             for r in insts]
    try:
        F1s = [st.colmajor(torch.from_numpy(r["F1"]).cuda()) for r in insts]
        F2s = [st.colmajor(torch.from_numpy(r["F2"]).cuda()) for r in insts]
        res, bs = st.solve_batch(probs, F1s, F2s)
        torch.cuda.synchronize()
        assert bs["grouped"] == len(insts)
        assert all(r[3] == st.ST_OK for r in res)
        small = [i for i, r in enumerate(insts) if r["n"] == 63]
        big = [i for i, r in enumerate(insts) if r["n"] != 63][::12]
        assert len(small) >= 40 and len(big) >= 10
        for i in small:
            r = insts[i]
            M, A = fem.tensor_operators(2, r["n"], kappa=r["kappa"])
            D, C = timefe.time_matrices(r["n_t"], 1.0)
            ref = kron.forward_substitution(M, A, D, C, r["F1"] @ r["F2"].T)
            U = (res[i][0] @ res[i][1]).cpu().numpy()
            err = np.linalg.norm(U - ref) / np.linalg.norm(ref)
            assert err <= 1e-6, (i, err)
            colerr = np.linalg.norm(U - ref, axis=0) / np.maximum(np.linalg.norm(ref, axis=0), 1e-12)
            assert np.max(colerr) <= 1e-5, (i, float(np.max(colerr)))
        for i in big:
            r = insts[i]
            M, A = fem.tensor_operators(2, r["n"], kappa=r["kappa"])
            D, C = timefe.time_matrices(r["n_t"], 1.0)
            V, Y = res[i][0].cpu().numpy(), res[i][1].cpu().numpy()
            true_res = residual.relres_lowrank(M, A, D, C, V, Y, r["F1"], r["F2"])
            assert true_res <= 1e-8 + 1e-10, (i, true_res)
    finally:
        for p in probs:
            p.close()


def three_d_requests():
    """3D heat and convection-diffusion requests of the served stream's kinds at 31^3 and 63^3, 64 time steps,
    rank-2 Gaussian loads (child generators of the stream's seed)."""
    reqs = []
    for j, (n, op) in enumerate([(31, "heat"), (31, "convdiff"), (63, "heat"), (63, "convdiff")]):
        reqs.append(dict(index=j, arrival_s=0.002 * j, op=op, dim=3, n=n, n_t=64, T=1.0, eps=0.3 if op == "heat" else 0.05,
                         beta=(1.0, 0.5, 0.25), p=2, seed=(5, 9000 + j)))
    return reqs


def test_served_three_d_requests_match_oracle_first_columns():
    """3D requests through the executor (replayed as a stream): the first two time columns of each solution
    against the oracle's forward substitution (conjugate gradients for heat, CG on the normal equations for
    convection-diffusion: direct factorisations of 63^3 blocks do not fit the test's time)."""
    reqs = three_d_requests()
    facs = [tuple(np.asfortranarray(x) for x in workloads.request_factors(r)) for r in reqs]
    outs = {i: np.zeros((r["n"] ** 3, r["n_t"]), order="F") for i, r in enumerate(reqs)}
    out = serve.run_stream(reqs, facs, precision=st.ST_MIXED, slots=4, outputs=outs)
    assert out["ok"] == len(reqs)
    for i, r in enumerate(reqs):
        if r["op"] == "heat":
            M, A = fem.tensor_operators(3, r["n"], kappa=r["eps"])
            D, C = timefe.time_matrices(r["n_t"], 1.0)
            ref = kron.forward_substitution_cg(M, A, D, C, facs[i][0], facs[i][1], 2, rtol=1e-13)
        else:
            M, A = fem.tensor_operators(3, r["n"], op="convdiff", eps=r["eps"], beta=r["beta"])
            D, C = timefe.time_matrices(r["n_t"], 1.0)
            ref = kron.forward_substitution_normal_cg(M, A, D, C, facs[i][0], facs[i][1], 2, rtol=1e-12)
        err = np.linalg.norm(outs[i][:, :2] - ref) / np.linalg.norm(ref)
        assert err <= 1e-6, (i, r["op"], r["n"], err)


def test_served_stream_sample_matches_oracle():
    cfg = workloads.WORKLOADS["served"]
    reqs = workloads.served_requests(count=60, seed=cfg["seed"], mean_gap_s=cfg["mean_gap_s"], p=cfg["p"])
    # the opening stretch without the largest 3D grids (their direct oracle does not fit)
    reqs = [r for r in reqs if r["n"] ** r["dim"] <= 127 ** 2]
    facs = [tuple(np.asfortranarray(x) for x in workloads.request_factors(r)) for r in reqs]
    outs = {i: np.zeros((r["n"] ** r["dim"], r["n_t"]), order="F") for i, r in enumerate(reqs)}
    out = serve.run_stream(reqs, facs, precision=st.ST_MIXED, slots=8, outputs=outs)
    assert out["ok"] == len(reqs)
    kinds = set()
    for i, r in enumerate(reqs):
        if r["op"] == "heat":
            M, A = fem.tensor_operators(r["dim"], r["n"], kappa=r["eps"])
        else:
            M, A = fem.tensor_operators(r["dim"], r["n"], op="convdiff", eps=r["eps"], beta=r["beta"])
        D, C = timefe.time_matrices(r["n_t"], 1.0)
        F1, F2 = facs[i]
        ref = kron.forward_substitution(M, A, D, C, F1 @ F2.T)
        err = np.linalg.norm(outs[i] - ref) / np.linalg.norm(ref)
        assert err <= 1e-6, (i, r["op"], r["dim"], r["n"], err)
        kinds.add(r["op"])
    assert kinds == {"heat", "convdiff"}
