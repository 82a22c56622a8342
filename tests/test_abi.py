"""The C-ABI library builds, loads without a GPU and exports every declared symbol."""

import ctypes
import re
import subprocess
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def lib():
    from paper_1912_10082_gb300.build import build

    path = build()
    return ctypes.CDLL(str(path))


def declared_functions():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(st_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("st_setup", "st_apply", "st_solve", "st_residual", "st_timestep_cn", "st_destroy",
                     "st_error_string"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    import paper_1912_10082_gb300 as st

    assert set(declared_functions()) <= set(st.ABI_SYMBOLS)


def test_error_strings_without_gpu(lib):
    lib.st_error_string.restype = ctypes.c_char_p
    assert lib.st_error_string(0) == b"ok"
    assert lib.st_error_string(-3).startswith(b"not converged")
    lib.st_setup.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.st_setup(None, None) == -1          # host-side argument check, no GPU call


def test_struct_layouts_match_c(tmp_path):
    """sizeof/offsetof of the ABI structs seen by gcc equal the ctypes mirrors."""
    import paper_1912_10082_gb300 as st

    fields = {"st_desc": st.StDesc, "st_solution": st.StSolution, "st_stats": st.StStats,
              "st_request": st.StRequest, "st_result": st.StResult, "st_kernel_time": st.StKernelTime}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "st.h"', "int main(void){"]
    for cname, cls in fields.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", f"-I{ROOT / 'include'}", str(src), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                          check=True).stdout.splitlines())
    for cname, cls in fields.items():
        assert int(out[cname]) == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert int(out[f"{cname}.{fname}"]) == getattr(cls, fname).offset, (cname, fname)


@pytest.mark.parametrize("dim,n,jitter", [(2, 9, 0.25), (3, 4, 0.25), (2, 6, 0.0)])
def test_p1_mesh_assembly_matches_the_oracle(dim, n, jitter):
    """st_p1_mesh_csr (host code of the library, no GPU) against the oracle's P1 assembly on the same mesh: the
    same pattern, values within rounding."""
    import paper_1912_10082_gb300 as st
    import workloads
    from oracle import fem
    msh = workloads.simplex_mesh(dim, n, seed=2, jitter=jitter)
    rp, col, mv, av = st.p1_mesh_csr(msh["nodes"], msh["elems"], msh["interior"], kappa=0.9)
    M, A = fem.p1_simplex_operators(msh["nodes"], msh["elems"], msh["interior"], kappa=0.9)
    assert np.array_equal(rp, M.indptr) and np.array_equal(col, M.indices)
    assert np.abs(mv - M.data).max() <= 1e-15 * np.abs(M.data).max() * 10
    assert np.abs(av - A.data).max() <= 1e-14 * np.abs(A.data).max()


def test_p1_mesh_assembly_refuses_bad_input():
    import paper_1912_10082_gb300 as st
    nodes = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [2.0, 0.0]])
    inter = np.ones(4, dtype=np.uint8)
    with pytest.raises(st.StError):
        st.p1_mesh_csr(nodes, np.array([[0, 1, 3]]), inter)   # degenerate (collinear) triangle
    with pytest.raises(st.StError):
        st.p1_mesh_csr(nodes, np.array([[0, 1, 7]]), inter)   # index out of range


@pytest.mark.parametrize("nx,nt,T", [(6, 9, 1.0), (13, 5, 2.5)])
def test_wave_matrices_match_the_oracle(nx, nt, T):
    """st_wave_matrices (host code, no GPU) against the oracle's B-spline Gram matrices."""
    import paper_1912_10082_gb300 as st
    from oracle import wave
    mine = st.wave_matrices(nx, nt, T)
    ref = wave.wave_matrices(nx, nt, T)
    for a, b in zip(mine, ref):
        assert a.shape == b.shape
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
