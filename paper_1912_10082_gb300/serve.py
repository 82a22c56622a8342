"""Batched and served space-time solves on one GPU, on top of the native executor.

``run_batch`` submits a set of independent problems at once and waits for all
of them (the batched workload).  ``run_stream`` submits requests at their
arrival times (a Poisson stream) while earlier ones are still running, so the
executor's slots admit new work as earlier solves finish and HBM frees up
(continuous batching); it reports per-request latency = completion - arrival.
Both only marshal requests: the scheduling, admission and every solve run in
libst.so (st_executor_*).
"""

from __future__ import annotations

import time

import numpy as np

from . import (ST_CONVDIFF, ST_FP64, ST_HEAT, ST_METHOD_RKSM, ST_OK, ST_ENOTCONV, ST_SCHED_FIFO, Executor,
               make_desc)


def _desc_of(r, precision, tol, maxit):
    op = ST_CONVDIFF if r.get("op", "heat") == "convdiff" else ST_HEAT
    kappa = float(r.get("kappa", r.get("eps", 1.0))) if op == ST_HEAT else 1.0
    return make_desc(int(r["dim"]), int(r["n"]), int(r["n_t"]), float(r.get("T", 1.0)), kappa, op=op,
                     eps=float(r.get("eps", 0.0)), beta=tuple(r.get("beta", (0.0, 0.0, 0.0))),
                     precision=precision, tol=tol, maxit=maxit)


def run_batch(instances, *, precision=ST_FP64, tol=1e-8, maxit=400, slots=16, method=ST_METHOD_RKSM,
              hbm_budget_bytes=0.0, outputs=None):
    """Solve every instance (dicts with dim, n, n_t, kappa/eps, F1, F2) at once.

    Returns dict(makespan_s, dof, results) where results[i] is the executor's
    result of instance i.  ``outputs[i]``, if given, receives the dense U.
    """
    # largest instances first (longest-processing-time order): the small ones fill the slots at
    # the end instead of one large solve running alone
    order = sorted(range(len(instances)),
                   key=lambda i: (-(int(instances[i]["n"]) ** int(instances[i]["dim"])), -int(instances[i]["n_t"]), i))
    with Executor(slots=slots, hbm_budget_bytes=hbm_budget_bytes) as ex:
        t0 = ex.now()
        for i in order:
            r = instances[i]
            U = outputs[i] if outputs is not None else None
            ex.submit(_desc_of(r, precision, tol, maxit), r["F1"], r["F2"], tag=i, U_out=U, method=method)
        got = {}
        while len(got) < len(instances):
            for res in ex.wait(256, timeout=0.5):
                got[int(res["tag"])] = res
        t1 = max(g["t_end"] for g in got.values())
    dof = sum(int(r["n"]) ** int(r["dim"]) * int(r["n_t"]) for r in instances)
    return dict(makespan_s=t1 - t0, dof=dof, results=[got[i] for i in range(len(instances))])


def run_stream(requests, factors, *, precision=ST_FP64, tol=1e-8, maxit=400, slots=16, hbm_budget_bytes=0.0,
               warmup=0, outputs=None, policy=ST_SCHED_FIFO):
    """Replay a request stream: request i is submitted at its ``arrival_s``.

    ``factors[i]`` = (F1, F2).  The first ``warmup`` requests are run but left
    out of the statistics.  ``outputs`` (optional dict index -> column-major
    n_h x n_t buffer) receives the dense solution of those requests.  Returns
    dict with p50/p99 latency (s), DoF/s over the measured requests' makespan
    and the per-request records.  ``policy`` is the executor's admission order
    (ST_SCHED_FIFO or ST_SCHED_HRRN).
    """
    recs = {}
    with Executor(slots=slots, hbm_budget_bytes=hbm_budget_bytes, policy=policy) as ex:
        start = ex.now()
        i = 0
        n = len(requests)
        while len(recs) < n:
            now = ex.now() - start
            while i < n and requests[i]["arrival_s"] <= now:
                F1, F2 = factors[i]
                U = outputs.get(i) if outputs else None
                ex.submit(_desc_of(requests[i], precision, tol, maxit), F1, F2, tag=i, U_out=U)
                i += 1
            wait = 0.0005
            if i < n:
                wait = max(0.0, min(0.02, requests[i]["arrival_s"] - (ex.now() - start)))
            for res in ex.wait(256, timeout=wait):
                recs[int(res["tag"])] = res
        arrivals = {j: start + requests[j]["arrival_s"] for j in range(n)}
    meas = [j for j in range(warmup, n)]
    lat = np.array([recs[j]["t_end"] - arrivals[j] for j in meas])
    ok = [j for j in meas if recs[j]["status"] in (ST_OK,)]
    t_first = min(arrivals[j] for j in meas)
    t_last = max(recs[j]["t_end"] for j in meas)
    dof = sum(int(requests[j]["n"]) ** int(requests[j]["dim"]) * int(requests[j]["n_t"]) for j in ok)
    return dict(p50_s=float(np.percentile(lat, 50)), p99_s=float(np.percentile(lat, 99)),
                dof_per_s=dof / (t_last - t_first), makespan_s=t_last - t_first, measured=len(meas),
                ok=len(ok), not_converged=sum(recs[j]["status"] == ST_ENOTCONV for j in meas),
                records=recs)
