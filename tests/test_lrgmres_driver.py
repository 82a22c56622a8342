"""The LR-FGMRES host driver (csrc/st_lrgmres.h) against the pinned oracle (oracle/lrfgmres.py), on the CPU.

A dense host backend (tests/lrgmres_check.cpp) stands in for the device one: the driver's Arnoldi process, Givens
least squares and stopping rule must give the oracle's residual history step by step without a preconditioner,
one step with the exact preconditioner, the direct solution at convergence, and the oracle's memory count.
"""

import shutil
import subprocess
from pathlib import Path

import numpy as np
import pytest
import scipy.sparse as sp

import workloads
from oracle import fem, kron, lrfgmres, timefe

ROOT = Path(__file__).resolve().parent.parent
CUDA_INC = Path("/usr/local/cuda/include")


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not (CUDA_INC / "cuda_runtime.h").exists():
        pytest.skip("needs g++ and the CUDA headers")
    out = tmp_path_factory.mktemp("lrgmres") / "check"
    subprocess.run([gxx, "-O2", "-std=c++17", "-pthread", f"-I{ROOT / 'include'}",
                    f"-I{ROOT / 'paper_1912_10082_gb300' / 'csrc'}", f"-I{CUDA_INC}",
                    str(ROOT / "tests" / "lrgmres_check.cpp"),
                    str(ROOT / "paper_1912_10082_gb300" / "csrc" / "st_dense.cpp"), "-o", str(out)],
                   check=True, capture_output=True, text=True)
    return out


def problem(dim, n, nt, p, seed):
    M, A = fem.tensor_operators(dim, n)
    D, C = timefe.time_matrices(nt, 1.0)
    F1, F2 = workloads.gaussian_factors(M.shape[0], nt, p, seed=seed)
    return M.toarray(), A.toarray(), D, C, F1, F2


def run(exe, tmp_path, prob, mode, maxit, tol, trunc):
    M, A, D, C, F1, F2 = prob
    nh, nt, p = M.shape[0], D.shape[0], F1.shape[1]
    path = tmp_path / f"prob_{mode}_{maxit}.txt"
    vals = [M, A, D, C, F1, F2]
    path.write_text(f"{nh} {nt} {p}\n" + "\n".join(" ".join(repr(float(x)) for x in v.reshape(-1, order="F"))
                                                for v in vals) + "\n")
    out = subprocess.run([str(exe), str(path), mode, str(maxit), repr(tol), repr(trunc)], capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    rec = {}
    for ln in out.stdout.splitlines():
        key, *rest = ln.split()
        rec[key] = [float(x) for x in rest]
    X = np.array(rec["X"]).reshape(nh, nt, order="F")
    return dict(its=int(rec["its"][0]), converged=bool(rec["converged"][0]), mu=int(rec["mu"][0]),
                hist=np.array(rec["hist"]), X=X)


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_unpreconditioned_history_matches_oracle(exe, tmp_path):
    prob = problem(1, 7, 5, 2, 3)
    got = run(exe, tmp_path, prob, "identity", 7, 1e-30, 1e-15)
    ref = lrfgmres.lr_fgmres(*prob[:4], prob[4], prob[5], tol=1e-30, maxit=7, precondition=False, trunc=1e-15)
    assert got["its"] == 7 and len(got["hist"]) == len(ref["history"]) == 8
    assert np.allclose(got["hist"], ref["history"], rtol=1e-8, atol=1e-13)


@pytest.mark.parametrize("dim,n,nt,p,seed", [(1, 7, 5, 2, 4), (2, (4, 3), 6, 2, 5)])
def test_converges_to_the_direct_solution(exe, tmp_path, dim, n, nt, p, seed):
    prob = problem(dim, n, nt, p, seed)
    U = kron.solve_sparse(sp.csr_matrix(prob[0]), sp.csr_matrix(prob[1]), prob[2], prob[3], prob[4] @ prob[5].T)
    N = prob[0].shape[0] * nt
    got = run(exe, tmp_path, prob, "identity", N, 1e-12, 1e-14)
    assert got["converged"] and relerr(got["X"], U) <= 1e-9
    ref = lrfgmres.lr_fgmres(*prob[:4], prob[4], prob[5], tol=1e-12, maxit=N, precondition=False, trunc=1e-14)
    assert got["its"] == ref["iterations"]
    assert abs(got["mu"] - ref["mu_mem"]) <= 2   # truncation decisions at 1e-14 may differ by a column


def test_exact_preconditioner_takes_one_step(exe, tmp_path):
    prob = problem(2, (4, 3), 6, 2, 6)
    got = run(exe, tmp_path, prob, "exact", 10, 1e-10, 1e-15)
    assert got["its"] == 1 and got["converged"] and got["hist"][1] <= 1e-12
    M, A, D, C, F1, F2 = prob
    B = np.kron(D, M) + np.kron(C, A)
    U = np.linalg.solve(B, (F1 @ F2.T).reshape(-1, order="F")).reshape(M.shape[0], D.shape[0], order="F")
    assert relerr(got["X"], U) <= 1e-10


def test_zero_load_returns_zero(exe, tmp_path):
    M, A, D, C, F1, F2 = problem(1, 5, 4, 1, 7)
    got = run(exe, tmp_path, (M, A, D, C, 0.0 * F1, F2), "identity", 5, 1e-8, 1e-14)
    assert got["converged"] and got["its"] == 0 and np.all(got["X"] == 0.0)


@pytest.mark.parametrize("nh,nt,r,rank", [(30, 12, 6, 3), (30, 5, 8, 3), (9, 40, 7, 7)])
def test_truncation_core_matches_the_oracle(exe, tmp_path, nh, nt, r, rank):
    """The host half of the device backend's truncation (R_P from a QR of P, then the QR of Q or Q_Q = I when
    r > n_t, the core SVD) against the oracle's truncation and the Eckart-Young error."""
    rng = np.random.default_rng(nh + nt + r)
    s = 10.0 ** -np.arange(rank, dtype=float) * 3.0
    s[-1] = 1e-13 if rank > 1 else s[-1]                       # one value below trunc * largest
    U, _ = np.linalg.qr(rng.standard_normal((nh, rank)))
    V, _ = np.linalg.qr(rng.standard_normal((nt, rank)))
    G = rng.standard_normal((rank, r))                          # r redundant columns of the same product
    P = (U * s) @ G
    Q = V @ np.linalg.pinv(G).T
    X = P @ Q.T
    path = tmp_path / "trunc.txt"
    path.write_text(f"{nh} {nt} {r}\n" + " ".join(repr(float(x)) for x in P.reshape(-1, order="F")) + "\n"
                    + " ".join(repr(float(x)) for x in Q.reshape(-1, order="F")) + "\n")
    out = subprocess.run([str(exe), str(path), "truncate", "1e-12"], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stdout + out.stderr
    rec = {ln.split()[0]: ln.split()[1:] for ln in out.stdout.splitlines()}
    k = int(rec["k"][0])
    Xt = np.array([float(x) for x in rec["X"]]).reshape(nh, nt, order="F")
    Pr, Qr = lrfgmres.lr_truncate(P, Q, 1e-12)
    assert k == Pr.shape[1] == (rank - 1 if rank > 1 else 1)
    assert np.linalg.norm(Xt - Pr @ Qr.T) <= 1e-13 * np.linalg.norm(X)
    assert abs(np.linalg.norm(X - Xt) - (s[-1] if rank > 1 else 0.0)) <= 1e-14 * s[0]


def test_vanishing_preconditioned_direction_is_stagnation_not_convergence(exe, tmp_path):
    """A preconditioner whose output truncates to rank 0 makes h(j,j) and h(j+1,j) vanish together.  The
    least-squares problem is then singular at that step: the driver must report stagnation (not converged,
    the estimate unchanged at |g_j| / beta = 1) and leave the step out of the solution (X = 0)."""
    prob = problem(1, 5, 4, 1, 8)
    got = run(exe, tmp_path, prob, "zero", 5, 1e-8, 1e-14)
    assert not got["converged"]
    assert got["its"] == 0
    assert np.allclose(got["hist"], [1.0, 1.0], rtol=0, atol=1e-15)
    assert np.all(got["X"] == 0.0)
