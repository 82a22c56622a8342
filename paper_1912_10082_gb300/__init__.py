"""GB300 space-time Petrov-Galerkin heat solver: Python binding of libst.so.

The binding only marshals arguments; every computation runs in the CUDA library
(``csrc/``), whose C ABI is declared in ``include/st.h``.  Matrices cross the
boundary in column-major layout: an ``(rows, cols)`` torch tensor or numpy array
whose first index is the fastest (``X.stride(0) == 1``).  ``colmajor`` makes
such a copy when needed.

Importing this package never compiles anything; ``build()`` (or
``python -m paper_1912_10082_gb300.build``) builds the library in-tree.  A
missing library raises ``RuntimeError`` at first use: there is no fallback.
"""

from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "_lib" / "libst.so"

ST_OK, ST_EINVAL, ST_ENOMEM, ST_ENOTCONV, ST_EBREAKDOWN, ST_ECUDA, ST_ETIMEOUT, ST_ENOTSUP = 0, -1, -2, -3, -4, -5, -6, -7
ST_FP64, ST_MIXED = 0, 1
ST_F64, ST_F32 = 0, 1
ST_HEAT, ST_CONVDIFF = 0, 1
ST_METHOD_RKSM, ST_METHOD_CN = 0, 1
ST_SCHED_FIFO, ST_SCHED_HRRN = 0, 1

# every symbol include/st.h declares
ABI_SYMBOLS = (
    "st_setup", "st_destroy", "st_problem_info", "st_get_csr", "st_apply", "st_rhs_manufactured",
    "st_shift_solve", "st_solve", "st_residual", "st_residual_lowrank", "st_timestep_cn",
    "st_error_string", "st_last_error", "st_launch_count", "st_profile_begin", "st_profile_end",
    "st_shift_solve_noalloc", "st_shift_solve_noalloc_max", "st_set_coefficients", "st_request_bytes",
    "st_executor_create", "st_executor_submit", "st_executor_wait", "st_executor_pending", "st_executor_now",
    "st_executor_destroy", "st_executor_set_policy", "st_autotune", "st_autotune_reset", "st_autotune_count",
    "st_autotune_save", "st_autotune_load", "st_solve_batch", "st_solve_lrfgmres", "st_p1_mesh_csr",
    "st_wave_matrices", "st_wave_solve",
)


class StDesc(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("n", C.c_int * 3), ("length", C.c_double * 3), ("op", C.c_int),
        ("kappa", C.c_double), ("eps", C.c_double), ("beta", C.c_double * 3), ("n_t", C.c_int),
        ("T", C.c_double), ("n_h", C.c_int), ("nnz", C.c_int), ("row_ptr", C.c_void_p),
        ("col_idx", C.c_void_p), ("m_vals", C.c_void_p), ("a_vals", C.c_void_p),
        ("precision", C.c_int), ("tol", C.c_double), ("maxit", C.c_int), ("max_basis", C.c_int),
        ("stream", C.c_void_p),
    ]


class StSolution(C.Structure):
    _fields_ = [("n_h", C.c_int), ("n_t", C.c_int), ("k", C.c_int), ("V", C.c_void_p), ("Y", C.c_void_p),
                ("U_dense", C.c_void_p), ("ldu", C.c_int)]


class StStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("basis_cols", C.c_int), ("rank", C.c_int), ("p", C.c_int),
                ("converged", C.c_int), ("residual_checks", C.c_int), ("mu_mem", C.c_int),
                ("relres", C.c_double), ("ms_total", C.c_double), ("ms_phase", C.c_double * 8),
                ("shift_min", C.c_double), ("shift_max", C.c_double), ("inner_iterations", C.c_int)]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_ if name != "ms_phase"}
        d["ms_phase"] = list(self.ms_phase)
        return d


class StRequest(C.Structure):
    _fields_ = [("desc", StDesc), ("F1", C.c_void_p), ("ldf1", C.c_int), ("F2", C.c_void_p), ("ldf2", C.c_int),
                ("p", C.c_int), ("U_out", C.c_void_p), ("ldu", C.c_int), ("tag", C.c_ulonglong),
                ("method", C.c_int)]


class StResult(C.Structure):
    _fields_ = [("tag", C.c_ulonglong), ("status", C.c_int), ("slot", C.c_int), ("k", C.c_int),
                ("bytes_reserved", C.c_double), ("t_submit", C.c_double), ("t_start", C.c_double),
                ("t_end", C.c_double), ("stats", StStats), ("message", C.c_char * 160)]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_ if name not in ("stats", "message")}
        d["stats"] = self.stats.as_dict()
        d["message"] = self.message.decode(errors="replace")
        return d


class StBatchStats(C.Structure):
    _fields_ = [("instances", C.c_int), ("grouped", C.c_int), ("rounds", C.c_int), ("grouped_launches", C.c_int),
                ("groups", C.c_int), ("ms_total", C.c_double), ("ms_phase", C.c_double * 8)]

    PHASES = ("compress", "shift_solve_cgs", "block_qr_host", "qr_products", "projected_solve", "residual",
              "output", "shifts")

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_ if name != "ms_phase"}
        d["ms_phase"] = dict(zip(self.PHASES, list(self.ms_phase)))
        return d


class StKernelTime(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("launches", C.c_int), ("ms", C.c_double), ("bytes", C.c_double),
                ("flops", C.c_double)]


_lib = None


def lib() -> C.CDLL:
    """Load libst.so (raises RuntimeError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() or "
                           "python -m paper_1912_10082_gb300.build (no CPU fallback exists)")
    L = C.CDLL(str(LIB_PATH))
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    sig = {
        "st_setup": ([C.POINTER(StDesc), C.POINTER(vp)], i),
        "st_destroy": ([vp], i),
        "st_problem_info": ([vp, C.POINTER(i), C.POINTER(i), C.POINTER(i), C.POINTER(d)], i),
        "st_get_csr": ([vp, vp, vp, vp, vp], i),
        "st_p1_mesh_csr": ([i, i, vp, i, vp, vp, d, vp, vp, vp, vp, C.POINTER(i), C.POINTER(i)], i),
        "st_wave_matrices": ([i, i, d, vp, vp, vp, vp, vp, vp], i),
        "st_wave_solve": ([i, i, d, vp, i, vp, i, i, d, i, vp, i, C.POINTER(StStats), vp], i),
        "st_apply": ([vp, i, vp, i, vp, i], i),
        "st_rhs_manufactured": ([vp, vp, i, vp, i], i),
        "st_shift_solve": ([vp, d, vp, i, i, vp, i, i], i),
        "st_solve": ([vp, vp, i, vp, i, i, C.POINTER(StSolution), C.POINTER(StStats)], i),
        "st_residual": ([vp, vp, i, vp, i, vp, i, i, C.POINTER(d)], i),
        "st_residual_lowrank": ([vp, vp, i, vp, i, i, vp, i, vp, i, i, C.POINTER(d)], i),
        "st_timestep_cn": ([vp, vp, i, vp, i, i, vp, i], i),
        "st_error_string": ([i], C.c_char_p),
        "st_last_error": ([], C.c_char_p),
        "st_launch_count": ([], C.c_ulonglong),
        "st_shift_solve_noalloc": ([vp, d, vp, i, i, vp, i], i),
        "st_shift_solve_noalloc_max": ([], C.c_ulong),
        "st_autotune": ([vp, d, i, i, C.POINTER(i)], i),
        "st_autotune_reset": ([], i),
        "st_autotune_count": ([], i),
        "st_autotune_save": ([C.c_char_p, C.c_char_p], i),
        "st_autotune_load": ([C.c_char_p, C.c_char_p, C.POINTER(i)], i),
        "st_set_coefficients": ([vp, i, d, d, vp], i),
        "st_request_bytes": ([C.POINTER(StDesc), i], d),
        "st_executor_create": ([i, d, C.POINTER(vp)], i),
        "st_executor_submit": ([vp, C.POINTER(StRequest)], i),
        "st_executor_wait": ([vp, C.POINTER(StResult), i, C.POINTER(i), d], i),
        "st_executor_pending": ([vp, C.POINTER(i), C.POINTER(i)], i),
        "st_executor_now": ([vp], d),
        "st_executor_set_policy": ([vp, i], i),
        "st_executor_destroy": ([vp], i),
        "st_profile_begin": ([], i),
        "st_profile_end": ([C.POINTER(StKernelTime), i, C.POINTER(i)], i),
        "st_solve_lrfgmres": ([vp, vp, i, vp, i, i, i, i, d, C.POINTER(StSolution), C.POINTER(StStats)], i),
        "st_solve_batch": ([i, C.POINTER(vp), C.POINTER(vp), C.POINTER(i), C.POINTER(vp), C.POINTER(i),
                            C.POINTER(i), C.POINTER(StSolution), C.POINTER(StStats), C.POINTER(i), vp, i,
                            C.POINTER(StBatchStats)], i),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


class StError(RuntimeError):
    def __init__(self, status: int, where: str):
        L = lib()
        msg = L.st_error_string(status).decode()
        last = L.st_last_error().decode()
        super().__init__(f"{where}: {msg} ({status})" + (f" [{last}]" if last else ""))
        self.status = status


def _check(status: int, where: str, ok=(ST_OK,)):
    if status not in ok:
        raise StError(status, where)
    return status


def colmajor(x):
    """Column-major copy (or the array itself) of a 2D torch tensor or numpy array."""
    if isinstance(x, np.ndarray):
        return np.asfortranarray(x, dtype=np.float64) if x.dtype != np.float32 else np.asfortranarray(x)
    import torch
    if x.dim() == 1:
        x = x[:, None]
    if x.stride(0) == 1 and (x.shape[1] == 1 or x.stride(1) >= x.shape[0]):
        return x
    return x.t().contiguous().t()


def _ptr_ld(x):
    """(pointer, leading dimension, rows, cols) of a column-major 2D array."""
    if isinstance(x, np.ndarray):
        if x.ndim == 1:
            x = x[:, None]
        if not x.flags["F_CONTIGUOUS"]:
            raise ValueError("numpy arrays must be Fortran-ordered (use colmajor)")
        return x.ctypes.data, max(1, x.shape[0]), x.shape[0], x.shape[1]
    if x.dim() == 1:
        return x.data_ptr(), max(1, x.shape[0]), x.shape[0], 1
    if x.stride(0) != 1 and x.shape[0] > 1:
        raise ValueError("tensors must be column-major (stride(0) == 1); use colmajor")
    ld = x.stride(1) if x.shape[1] > 1 else max(1, x.shape[0])
    return x.data_ptr(), max(ld, x.shape[0], 1), x.shape[0], x.shape[1]


class _DevView:
    """__cuda_array_interface__ over library-owned device memory (column-major)."""

    def __init__(self, ptr: int, rows: int, cols: int, ld: int):
        self.__cuda_array_interface__ = {
            "shape": (rows, cols), "typestr": "<f8", "data": (int(ptr or 0), False),
            "strides": (8, 8 * ld), "version": 3,
        }


def empty_colmajor(rows: int, cols: int, dtype=None, device="cuda"):
    import torch
    dtype = dtype or torch.float64
    return torch.empty((cols, rows), dtype=dtype, device=device).t()


def make_desc(dim: int, n, n_t: int, T: float = 1.0, kappa: float = 1.0, *, length=None, op: int = ST_HEAT,
              eps: float = 0.0, beta=(0.0, 0.0, 0.0), precision: int = ST_FP64, tol: float = 1e-8,
              maxit: int = 0, max_basis: int = 0) -> StDesc:
    """An st_desc for a box problem (see include/st.h for every field)."""
    d = StDesc()
    d.dim = int(dim)
    ns = [int(n)] * 3 if np.isscalar(n) else list(n) + [1] * (3 - len(n))
    for i in range(3):
        d.n[i] = int(ns[i]) if i < max(dim, 1) else 1
        d.length[i] = float(length[i]) if length is not None and i < len(length) else 1.0
        d.beta[i] = float(beta[i]) if i < len(beta) else 0.0
    d.op, d.kappa, d.eps = int(op), float(kappa), float(eps)
    d.n_t, d.T = int(n_t), float(T)
    d.precision, d.tol, d.maxit, d.max_basis = int(precision), float(tol), int(maxit), int(max_basis)
    return d


def p1_mesh_csr(nodes, elems, interior, kappa: float = 1.0):
    """st_p1_mesh_csr: P1 mass matrix and heat operator of a simplex mesh on its interior nodes, as the
    (row_ptr, col_idx, m_vals, a_vals) tuple that Problem(0, ..., csr=...) takes.  Host only."""
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    elems = np.ascontiguousarray(elems, dtype=np.int32)
    inter = np.ascontiguousarray(interior, dtype=np.uint8)
    dim = nodes.shape[1]
    nh, nnz = C.c_int(), C.c_int()
    args = (dim, nodes.shape[0], nodes.ctypes.data, elems.shape[0], elems.ctypes.data, inter.ctypes.data,
            float(kappa))
    _check(lib().st_p1_mesh_csr(*args, None, None, None, None, C.byref(nh), C.byref(nnz)), "st_p1_mesh_csr")
    rp = np.empty(nh.value + 1, dtype=np.int32)
    col = np.empty(nnz.value, dtype=np.int32)
    mv = np.empty(nnz.value)
    av = np.empty(nnz.value)
    _check(lib().st_p1_mesh_csr(*args, rp.ctypes.data, col.ctypes.data, mv.ctypes.data, av.ctypes.data,
                                C.byref(nh), C.byref(nnz)), "st_p1_mesh_csr")
    return rp, col, mv, av


def wave_matrices(n_x: int, n_t: int, T: float = 1.0):
    """st_wave_matrices: (Mh, Ah, Qh, Mt, Dt, Qt) of the wave equation's space-time system as numpy arrays."""
    nh, nt = n_x + 1, n_t + 1
    out = [np.zeros((nh, nh), order="F") for _ in range(3)] + [np.zeros((nt, nt), order="F") for _ in range(3)]
    _check(lib().st_wave_matrices(int(n_x), int(n_t), float(T), *[a.ctypes.data for a in out]), "st_wave_matrices")
    return tuple(out)


def wave_solve(n_x: int, n_t: int, T, F1, F2, tol: float = 1e-8, maxit: int = 300, U=None, stream=None,
               ok=(ST_OK,)):
    """st_wave_solve (GMRES+LYAP on the wave equation's three-term system): returns (U, stats, status); U is a
    device tensor (N_h x N_t, column-major) unless one is given (host numpy or device torch)."""
    import torch
    nh, nt = n_x + 1, n_t + 1
    p1, l1, _, m = _ptr_ld(F1)
    p2, l2, _, _ = _ptr_ld(F2)
    if U is None:
        U = empty_colmajor(nh, nt)
    pu, lu, _, _ = _ptr_ld(U)
    stats = StStats()
    sv = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    st = lib().st_wave_solve(int(n_x), int(n_t), float(T), p1, l1, p2, l2, m, float(tol), int(maxit), pu, lu,
                             C.byref(stats), sv)
    _check(st, "st_wave_solve", ok)
    return U, stats.as_dict(), st


class Problem:
    """Owns one st_problem handle (see include/st.h for every argument)."""

    def __init__(self, dim: int, n, n_t: int, T: float = 1.0, kappa: float = 1.0, *, length=None,
                 op: int = ST_HEAT, eps: float = 0.0, beta=(0.0, 0.0, 0.0), precision: int = ST_FP64,
                 tol: float = 1e-8, maxit: int = 0, max_basis: int = 0, stream=None, csr=None):
        L = lib()
        d = make_desc(dim, n, n_t, T, kappa, length=length, op=op, eps=eps, beta=beta, precision=precision,
                      tol=tol, maxit=maxit, max_basis=max_basis)
        self._keep = []
        if csr is not None:
            row_ptr, col, mv, av = (np.ascontiguousarray(csr[0], dtype=np.int32),
                                    np.ascontiguousarray(csr[1], dtype=np.int32),
                                    np.ascontiguousarray(csr[2], dtype=np.float64),
                                    np.ascontiguousarray(csr[3], dtype=np.float64))
            self._keep = [row_ptr, col, mv, av]
            d.dim = 0
            d.n_h, d.nnz = len(row_ptr) - 1, len(col)
            d.row_ptr, d.col_idx = row_ptr.ctypes.data, col.ctypes.data
            d.m_vals, d.a_vals = mv.ctypes.data, av.ctypes.data
        if stream is not None:
            d.stream = int(getattr(stream, "cuda_stream", stream))
        self.desc = d
        h = C.c_void_p()
        _check(L.st_setup(C.byref(d), C.byref(h)), "st_setup")
        self.h = h
        nh, nt, nnz, dt = C.c_int(), C.c_int(), C.c_int(), C.c_double()
        _check(L.st_problem_info(h, C.byref(nh), C.byref(nt), C.byref(nnz), C.byref(dt)), "st_problem_info")
        self.n_h, self.n_t, self.nnz, self.dt = nh.value, nt.value, nnz.value, dt.value

    def close(self):
        if getattr(self, "h", None):
            lib().st_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_coefficients(self, op: int = ST_HEAT, kappa: float = 1.0, eps: float = 0.0, beta=(0.0, 0.0, 0.0)):
        b = (C.c_double * 3)(*[float(x) for x in (list(beta) + [0.0] * 3)[:3]])
        _check(lib().st_set_coefficients(self.h, int(op), float(kappa), float(eps), b), "st_set_coefficients")

    # -- set-up data ---------------------------------------------------------
    def get_csr(self):
        rp = np.empty(self.n_h + 1, dtype=np.int32)
        col = np.empty(self.nnz, dtype=np.int32)
        mv = np.empty(self.nnz)
        av = np.empty(self.nnz)
        _check(lib().st_get_csr(self.h, rp.ctypes.data, col.ctypes.data, mv.ctypes.data, av.ctypes.data),
               "st_get_csr")
        return rp, col, mv, av

    def rhs_manufactured(self, F1=None, F2=None):
        F1 = empty_colmajor(self.n_h, 2) if F1 is None else F1
        F2 = empty_colmajor(self.n_t, 2) if F2 is None else F2
        p1, l1, _, _ = _ptr_ld(F1)
        p2, l2, _, _ = _ptr_ld(F2)
        _check(lib().st_rhs_manufactured(self.h, p1, l1, p2, l2), "st_rhs_manufactured")
        return F1, F2

    # -- hot path ------------------------------------------------------------
    def apply(self, U, Y=None):
        import torch
        dtype = ST_F32 if U.dtype == torch.float32 else ST_F64
        Y = empty_colmajor(self.n_h, self.n_t, dtype=U.dtype, device=U.device) if Y is None else Y
        pu, lu, _, _ = _ptr_ld(U)
        py, ly, _, _ = _ptr_ld(Y)
        _check(lib().st_apply(self.h, dtype, pu, lu, py, ly), "st_apply")
        return Y

    def shift_solve(self, s: float, X, W=None, precision: int = ST_FP64):
        W = empty_colmajor(self.n_h, X.shape[1] if X.dim() > 1 else 1, device=X.device) if W is None else W
        px, lx, _, m = _ptr_ld(X)
        pw, lw, _, _ = _ptr_ld(W)
        _check(lib().st_shift_solve(self.h, float(s), px, lx, m, pw, lw, int(precision)), "st_shift_solve")
        return W

    def autotune(self, s: float, ncols: int, precision: int = ST_FP64) -> int:
        """Times the shifted solve's launch variants for this problem's shapes; returns the shapes added."""
        n = C.c_int(0)
        _check(lib().st_autotune(self.h, float(s), int(ncols), int(precision), C.byref(n)), "st_autotune")
        return n.value

    def solve(self, F1, F2, U_dense=None, ok=(ST_OK,)):
        """Returns (V, Y, stats, status); V, Y are views of library-owned memory."""
        import torch
        p1, l1, _, m = _ptr_ld(F1)
        p2, l2, _, _ = _ptr_ld(F2)
        sol = StSolution()
        if U_dense is not None:
            pu, lu, _, _ = _ptr_ld(U_dense)
            sol.U_dense, sol.ldu = pu, lu
        stats = StStats()
        st = lib().st_solve(self.h, p1, l1, p2, l2, m, C.byref(sol), C.byref(stats))
        _check(st, "st_solve", ok)
        k = sol.k
        if k > 0:
            V = torch.as_tensor(_DevView(sol.V, self.n_h, k, self.n_h), device="cuda")
            Y = torch.as_tensor(_DevView(sol.Y, k, self.n_t, k), device="cuda")
        else:
            V = torch.zeros((self.n_h, 0), dtype=torch.float64, device="cuda")
            Y = torch.zeros((0, self.n_t), dtype=torch.float64, device="cuda")
        return V, Y, stats.as_dict(), st

    def solve_lrfgmres(self, F1, F2, maxit: int = 50, precond_iters: int = 5, trunc: float = 1e-12, U_dense=None,
                       ok=(ST_OK,)):
        """LR-FGMRES+RKSM (st_solve_lrfgmres): returns (V, Y, stats, status) with U = V Y."""
        import torch
        p1, l1, _, m = _ptr_ld(F1)
        p2, l2, _, _ = _ptr_ld(F2)
        sol = StSolution()
        if U_dense is not None:
            pu, lu, _, _ = _ptr_ld(U_dense)
            sol.U_dense, sol.ldu = pu, lu
        stats = StStats()
        st = lib().st_solve_lrfgmres(self.h, p1, l1, p2, l2, m, int(maxit), int(precond_iters), float(trunc),
                                     C.byref(sol), C.byref(stats))
        _check(st, "st_solve_lrfgmres", ok)
        k = sol.k
        if k > 0:
            V = torch.as_tensor(_DevView(sol.V, self.n_h, k, self.n_h), device="cuda")
            Y = torch.as_tensor(_DevView(sol.Y, k, self.n_t, k), device="cuda")
        else:
            V = torch.zeros((self.n_h, 0), dtype=torch.float64, device="cuda")
            Y = torch.zeros((0, self.n_t), dtype=torch.float64, device="cuda")
        return V, Y, stats.as_dict(), st

    def residual(self, U, F1, F2) -> float:
        pu, lu, _, _ = _ptr_ld(U)
        p1, l1, _, m = _ptr_ld(F1)
        p2, l2, _, _ = _ptr_ld(F2)
        out = C.c_double()
        _check(lib().st_residual(self.h, pu, lu, p1, l1, p2, l2, m, C.byref(out)), "st_residual")
        return out.value

    def residual_lowrank(self, V, Y, F1, F2) -> float:
        pv, lv, _, k = _ptr_ld(V)
        py, ly, _, _ = _ptr_ld(Y)
        p1, l1, _, m = _ptr_ld(F1)
        p2, l2, _, _ = _ptr_ld(F2)
        out = C.c_double()
        _check(lib().st_residual_lowrank(self.h, pv, lv, py, max(ly, 1), k, p1, l1, p2, l2, m, C.byref(out)),
               "st_residual_lowrank")
        return out.value

    def timestep_cn(self, F1, F2, U=None):
        U = empty_colmajor(self.n_h, self.n_t) if U is None else U
        p1, l1, _, m = _ptr_ld(F1)
        p2, l2, _, _ = _ptr_ld(F2)
        pu, lu, _, _ = _ptr_ld(U)
        _check(lib().st_timestep_cn(self.h, p1, l1, p2, l2, m, pu, lu), "st_timestep_cn")
        return U


def solve_batch(problems, F1s, F2s, U_dense=None, stream=None, groups=0):
    """st_solve_batch: solve every problem of the list at once (lock-step RKSM, grouped launches).

    ``problems``: distinct Problem objects; ``F1s[i]``, ``F2s[i]``: column-major load factors (host numpy or
    device torch).  ``U_dense`` (optional list, entries may be None) receives dense solutions.  Returns
    (results, batch_stats): results[i] = (V, Y, stats, status) as Problem.solve, V and Y views of the
    problem's own memory; batch_stats a dict of st_batch_stats.  ``groups``: lock-step groups run
    concurrently (0: the library's choice).
    """
    import torch
    n = len(problems)
    hs = (C.c_void_p * n)(*[p.h.value if isinstance(p.h, C.c_void_p) else p.h for p in problems])
    f1p = (C.c_void_p * n)()
    f2p = (C.c_void_p * n)()
    l1 = (C.c_int * n)()
    l2 = (C.c_int * n)()
    nc = (C.c_int * n)()
    for i in range(n):
        p1, ld1, _, m = _ptr_ld(F1s[i])
        p2, ld2, _, _ = _ptr_ld(F2s[i])
        f1p[i], f2p[i], l1[i], l2[i], nc[i] = p1, p2, ld1, ld2, m
    sols = (StSolution * n)()
    if U_dense is not None:
        for i, U in enumerate(U_dense):
            if U is not None:
                pu, lu, _, _ = _ptr_ld(U)
                sols[i].U_dense, sols[i].ldu = pu, lu
    stats = (StStats * n)()
    status = (C.c_int * n)()
    bs = StBatchStats()
    sv = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    _check(lib().st_solve_batch(n, hs, f1p, l1, f2p, l2, nc, sols, stats, status, sv, int(groups), C.byref(bs)),
           "st_solve_batch")
    out = []
    for i, prob in enumerate(problems):
        k = sols[i].k
        if k > 0 and sols[i].V:
            V = torch.as_tensor(_DevView(sols[i].V, prob.n_h, k, prob.n_h), device="cuda")
            Y = torch.as_tensor(_DevView(sols[i].Y, k, prob.n_t, k), device="cuda")
        else:
            V = torch.zeros((prob.n_h, 0), dtype=torch.float64, device="cuda")
            Y = torch.zeros((0, prob.n_t), dtype=torch.float64, device="cuda")
        out.append((V, Y, stats[i].as_dict(), int(status[i])))
    return out, bs.as_dict()


def request_bytes(desc: StDesc, p: int) -> float:
    """Admission estimate of one request's device footprint in bytes."""
    return float(lib().st_request_bytes(C.byref(desc), int(p)))


class Executor:
    """Many independent solves on one GPU (st_executor_*; see include/st.h).

    ``submit`` copies the request; the load factors (and the optional output
    buffer) are kept alive here until their result has been collected by
    ``wait``.
    """

    def __init__(self, slots: int = 16, hbm_budget_bytes: float = 0.0, policy: int = ST_SCHED_FIFO):
        h = C.c_void_p()
        _check(lib().st_executor_create(int(slots), float(hbm_budget_bytes), C.byref(h)), "st_executor_create")
        self.h = h
        self._live = {}
        if policy != ST_SCHED_FIFO:
            self.set_policy(policy)

    def set_policy(self, policy: int):
        _check(lib().st_executor_set_policy(self.h, int(policy)), "st_executor_set_policy")

    def now(self) -> float:
        return float(lib().st_executor_now(self.h))

    def submit(self, desc: StDesc, F1, F2, tag: int, U_out=None, method: int = ST_METHOD_RKSM):
        r = StRequest()
        r.desc = desc
        r.method = int(method)
        p1, l1, _, m = _ptr_ld(F1)
        p2, l2, _, _ = _ptr_ld(F2)
        r.F1, r.ldf1, r.F2, r.ldf2, r.p, r.tag = p1, l1, p2, l2, m, int(tag)
        if U_out is not None:
            pu, lu, _, _ = _ptr_ld(U_out)
            r.U_out, r.ldu = pu, lu
        self._live[int(tag)] = (F1, F2, U_out)
        _check(lib().st_executor_submit(self.h, C.byref(r)), "st_executor_submit")

    def wait(self, max_results: int = 256, timeout: float = 0.05):
        arr = (StResult * max_results)()
        cnt = C.c_int()
        _check(lib().st_executor_wait(self.h, arr, max_results, C.byref(cnt), float(timeout)), "st_executor_wait")
        out = []
        for i in range(cnt.value):
            d = arr[i].as_dict()
            self._live.pop(int(d["tag"]), None)
            out.append(d)
        return out

    def pending(self):
        q, r = C.c_int(), C.c_int()
        _check(lib().st_executor_pending(self.h, C.byref(q), C.byref(r)), "st_executor_pending")
        return q.value, r.value

    def close(self):
        if getattr(self, "h", None):
            lib().st_executor_destroy(self.h)
            self.h = None
            self._live.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(lib().st_launch_count())


def autotune_reset():
    """Forget every tuned launch choice (later launches take the built-in choices)."""
    _check(lib().st_autotune_reset(), "st_autotune_reset")


def autotune_count() -> int:
    """Number of kernel shapes with a tuned launch choice in this process."""
    return int(lib().st_autotune_count())


def device_tag(device=None) -> str:
    """Identity of a CUDA device for the tuning cache: name, compute capability and SM count."""
    import torch
    pr = torch.cuda.get_device_properties(torch.cuda.current_device() if device is None else device)
    return f"{pr.name} sm_{pr.major}{pr.minor} {pr.multi_processor_count}SM"


def autotune_save(path, tag: str | None = None):
    """Write the tuned launch choices to a file (tag: device identity; default: the current CUDA device's)."""
    tag = device_tag() if tag is None else tag
    _check(lib().st_autotune_save(str(path).encode(), tag.encode()), "st_autotune_save")


def autotune_load(path, tag: str | None = None) -> int:
    """Add the choices of a tuning cache written for the same device tag; returns the entries added."""
    tag = device_tag() if tag is None else tag
    n = C.c_int(0)
    _check(lib().st_autotune_load(str(path).encode(), tag.encode(), C.byref(n)), "st_autotune_load")
    return n.value


def profile_begin():
    _check(lib().st_profile_begin(), "st_profile_begin")


def profile_end():
    """Per-kernel totals since profile_begin(): {tag: dict(launches, ms, bytes, flops)}."""
    L = lib()
    arr = (StKernelTime * 64)()
    cnt = C.c_int()
    _check(L.st_profile_end(arr, 64, C.byref(cnt)), "st_profile_end")
    return {arr[i].name.decode(): dict(launches=arr[i].launches, ms=arr[i].ms, bytes=arr[i].bytes,
                                       flops=arr[i].flops) for i in range(min(cnt.value, 64))}


def build(force: bool = False):
    from .build import build as _b
    return _b(force=force)
