"""The solver's host algebra (csrc/st_dense.cpp) on the CPU: thread-count independence and accuracy.

The projected problems (Cholesky, multi-right-hand-side solves, the symmetric eigenvalues behind the adaptive
shifts) run on a host thread team whose size depends on how many solves share the host.  Each parallel loop gives
every output element to one thread in the serial summation order, so a solve's numbers must not depend on the
team size: the check program compares one thread with the full team bitwise (Cholesky, its solve, the eigenvalues,
forward substitution), checks L L^T = A and A A^{-1} = I, the LU solves A X = B and A^T X = B (and that a singular
matrix is reported), the Householder QR and the eigenvectors, and prints the eigenvalues of a fixed matrix and the
singular values of two graded matrices, compared here with numpy's.
"""

import shutil
import subprocess
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parent.parent
CUDA_INC = Path("/usr/local/cuda/include")


@pytest.fixture(scope="module")
def run_check(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not (CUDA_INC / "cuda_runtime.h").exists():
        pytest.skip("needs g++ and the CUDA headers")
    exe = tmp_path_factory.mktemp("host_algebra") / "check"
    subprocess.run([gxx, "-O2", "-std=c++17", "-pthread", f"-I{ROOT / 'include'}",
                    f"-I{ROOT / 'paper_1912_10082_gb300' / 'csrc'}", f"-I{CUDA_INC}",
                    str(ROOT / "tests" / "host_algebra_check.cpp"),
                    str(ROOT / "paper_1912_10082_gb300" / "csrc" / "st_dense.cpp"), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    return out


def test_thread_count_independent_and_accurate(run_check):
    assert run_check.returncode == 0, run_check.stdout + run_check.stderr
    assert run_check.stdout.strip().endswith("PASS")


def test_eigenvalues_match_numpy(run_check):
    lines = run_check.stdout.splitlines()
    mat = np.array([float(x) for x in [ln for ln in lines if ln.startswith("mat")][0].split()[1:]])
    got = np.array([float(x) for x in [ln for ln in lines if ln.startswith("eig")][0].split()[1:]])
    m = len(got)
    C = mat.reshape(m, m).T   # column-major
    ref = np.linalg.eigvalsh(C)
    assert np.all(np.diff(got) >= 0)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("shape", [0, 1])
def test_jacobi_svd_matches_numpy(run_check, shape):
    """The one-sided Jacobi SVD behind the rank compression of F: graded singular values 1 .. 1e-14 (tall 15 x 12
    and square 12 x 12) agree with LAPACK's to rounding of the largest."""
    lines = run_check.stdout.splitlines()
    head = [ln for ln in lines if ln.startswith(f"svdmat{shape} ")][0].split()
    m, n = int(head[1]), int(head[2])
    B = np.array([float(x) for x in head[3:]]).reshape(n, m).T
    got = np.array([float(x) for x in [ln for ln in lines if ln.startswith(f"svdval{shape}")][0].split()[1:]])
    ref = np.linalg.svd(B, compute_uv=False)
    assert np.all(np.diff(got) <= 0)
    assert np.max(np.abs(got - ref)) <= 1e-14 * ref[0]
    # the graded values themselves, well above rounding: 1, 10^(-14/11), ...
    exact = 10.0 ** (-14.0 * np.arange(n) / (n - 1))
    big = exact > 1e-10
    assert np.max(np.abs(got[big] - exact[big]) / exact[big]) <= 1e-5
