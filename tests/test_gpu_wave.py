"""The wave equation's three-term space-time system on the GPU (st_wave_solve: GMRES+LYAP, paper Section 4
"Discretized Wave problem", Section 5 Example 2) against the oracle: its direct solve of the assembled system, its
own GMRES+LYAP iteration count, and Example 2's exact solution u = t^2 sin(2 pi x)."""

import numpy as np
import pytest
import torch

import paper_1912_10082_gb300 as st
from oracle import wave
import workloads

pytestmark = pytest.mark.gpu


def example2_load(n_x, n_t, T=1.0):
    return wave.load_factors(n_x, n_t, T, [lambda x: np.sin(2 * np.pi * x)] * 2,
                             [lambda t: 2.0 + 0.0 * t, lambda t: 4.0 * np.pi ** 2 * t ** 2])


@pytest.mark.parametrize("n_x,n_t,T", [(12, 12, 1.0), (10, 17, 1.5), (24, 9, 0.7)])
def test_wave_solve_matches_the_direct_solution_and_the_oracle_gmres(n_x, n_t, T):
    mats = wave.wave_matrices(n_x, n_t, T)
    F1, F2 = example2_load(n_x, n_t, T)
    F1, F2 = np.asfortranarray(F1), np.asfortranarray(F2)
    ref = wave.solve_direct(*mats, F1 @ F2.T)
    U, stats, status = st.wave_solve(n_x, n_t, T, F1, F2, tol=1e-11, maxit=300)
    torch.cuda.synchronize()
    Uh = U.cpu().numpy()
    assert status == st.ST_OK and stats["converged"] == 1
    assert np.linalg.norm(Uh - ref) <= 1e-8 * np.linalg.norm(ref)
    orc = wave.gmres_lyap(*mats, F1 @ F2.T, tol=1e-11, maxit=300)
    assert abs(stats["iterations"] - orc["iterations"]) <= 2, (stats["iterations"], orc["iterations"])
    # the true residual of the returned U, by the oracle's matrix form
    res = np.linalg.norm(wave.apply(*mats, Uh) - F1 @ F2.T) / np.linalg.norm(F1 @ F2.T)
    assert res <= 1e-10, res


def test_wave_solve_random_load_host_output_and_iteration_limit():
    n_x, n_t = 15, 11
    mats = wave.wave_matrices(n_x, n_t, 1.0)
    F1, F2 = workloads.gaussian_factors(n_x + 1, n_t + 1, 3, seed=12)
    F1, F2 = np.asfortranarray(F1), np.asfortranarray(F2)
    ref = wave.solve_direct(*mats, F1 @ F2.T)
    Uh = np.zeros((n_x + 1, n_t + 1), order="F")
    _, stats, status = st.wave_solve(n_x, n_t, 1.0, F1, F2, tol=1e-10, maxit=400, U=Uh)
    assert status == st.ST_OK
    assert np.linalg.norm(Uh - ref) <= 1e-7 * np.linalg.norm(ref)
    U3, s3, st3 = st.wave_solve(n_x, n_t, 1.0, F1, F2, tol=1e-10, maxit=3, ok=(st.ST_ENOTCONV,))
    assert st3 == st.ST_ENOTCONV and s3["iterations"] == 3 and s3["converged"] == 0
    assert np.all(np.isfinite(U3.cpu().numpy()))


def test_example2_solution_from_the_gpu_converges():
    x = np.linspace(0.01, 0.99, 57)
    t = np.linspace(0.01, 0.99, 53)
    exact = t[:, None] ** 2 * np.sin(2 * np.pi * x)[None, :]
    errs = []
    for n in (8, 16, 32):
        F1, F2 = example2_load(n, n)
        U, stats, status = st.wave_solve(n, n, 1.0, np.asfortranarray(F1), np.asfortranarray(F2), tol=1e-12,
                                         maxit=400)
        assert status == st.ST_OK
        errs.append(np.abs(wave.evaluate(U.cpu().numpy(), n, n, 1.0, x, t) - exact).max())
    assert errs[2] <= 5e-3 and errs[0] / errs[1] >= 3.5 and errs[1] / errs[2] >= 3.5, errs
