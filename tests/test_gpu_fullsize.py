"""The benchmark configurations at full size, checked on samples the oracle can compute.

* 3D heat, Q1 127^3 (N_h = 2,048,383), n_t = 512, rank-4 Gaussian load, mixed precision, tol 1e-8
  (the bench's launch configuration): the first two time columns of U = V Y against the oracle's
  block forward substitution with conjugate gradients (forward substitution fixes the first
  columns exactly whatever the later ones are).
* The batched workload (256 2D instances of mixed sizes, mixed precision, through the executor):
  every instance on the 63^2 grid against the oracle's direct solve.
* The served stream (heat and convection-diffusion): the requests of its opening stretch small
  enough for a direct oracle solve, replayed at their arrival times among the others.
Tolerance: 1e-6 relative error for mixed precision (the stated target).
"""

import numpy as np
import pytest
import torch

import paper_1912_10082_gb300 as st
from paper_1912_10082_gb300 import serve
from oracle import fem, kron, timefe
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
    assert status == st.ST_OK and stats["relres"] <= 1e-8
    M, A = fem.tensor_operators(dim, n)
    D, C = timefe.time_matrices(nt, cfg["T"])
    ref = kron.forward_substitution_cg(M, A, D, C, F1, F2, 2, rtol=1e-13)
    err = np.linalg.norm(U2 - ref) / np.linalg.norm(ref)
    assert err <= 1e-6, err


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
