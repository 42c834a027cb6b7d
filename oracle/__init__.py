"""ctypes loader for the plain-C FP64 oracle (lpk_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
the CPU-baseline leg of bench.py.  The product path (the CUDA library and its
binding) never imports this package.

Each wrapper takes numpy arrays, checks dtypes, and returns numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lpk_oracle.c")
_LIB = os.path.join(_HERE, "liblpk_oracle.so")

MRNE, CGNE, ABGMRES = 0, 1, 2
# per-iteration trace of lp_solve (orc_lp_solve), one row per step k
TRACE_FIELDS = ("gamma", "mu", "pinf", "dinf", "eps_in", "it_af", "it_cc", "alpha_p", "alpha_d", "sigma",
                "mu_af", "alpha_p_af", "alpha_d_af", "tau", "failed", "rel_gap")
TRACE_COLS = len(TRACE_FIELDS)
STATUS = {0: "OK", 1: "MAX_IPM_ITER", 2: "KRYLOV_STALL", 3: "DIVERGED", 4: "BREAKDOWN",
          6: "EMPTY_ROW_INCONSISTENT", 7: "EMPTY_COL_UNBOUNDED", 8: "INVALID_ARG", 9: "OOM"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags, no FMA contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                              os.path.getmtime(os.path.join(_HERE, "lpk_oracle.h")))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O3", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
                           "-Wall", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


class Options(C.Structure):
    _fields_ = [("tol", C.c_double), ("eta", C.c_double), ("phi", C.c_double),
                ("sigma_max", C.c_double), ("eps_in0", C.c_double), ("omega", C.c_double),
                ("start_tol", C.c_double), ("backtrack", C.c_double),
                ("max_ipm", C.c_int32), ("max_krylov", C.c_int32), ("inner_sweeps", C.c_int32),
                ("method", C.c_int32), ("color_seed", C.c_uint64), ("verbose", C.c_int32),
                ("corrector_ba", C.c_int32), ("max_correctors", C.c_int32), ("pad", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("status", C.c_int32), ("ipm_iters", C.c_int32),
                ("krylov_iters_total", C.c_int64), ("n_colors", C.c_int32),
                ("krylov_failures", C.c_int32), ("gamma", C.c_double), ("rel_gap", C.c_double),
                ("pinf", C.c_double), ("dinf", C.c_double), ("mu", C.c_double),
                ("obj_primal", C.c_double), ("obj_dual", C.c_double), ("correctors", C.c_int32),
                ("pad", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class KrylovInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("restarts", C.c_int32),
                ("breakdown", C.c_int32), ("res0", C.c_double), ("res", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        _lib.orc_color_rows.restype = C.c_int32
        _lib.orc_color_rows.argtypes = [C.c_int32, C.c_int32, P, P, C.c_uint64, P, P, P]
        _lib.orc_splitmix64.restype = C.c_uint64
        _lib.orc_splitmix64.argtypes = [C.c_uint64]
        _lib.orc_scale_rows.restype = None
        _lib.orc_scale_rows.argtypes = [C.c_int32, P, P, P, P, P, P]
        for fn in (_lib.orc_nessor, _lib.orc_nesor):
            fn.restype = None
            fn.argtypes = [C.c_int32, C.c_int32, P, P, P, P, P, C.c_int32, C.c_double, P, P]
        _lib.orc_krylov.restype = C.c_int32
        _lib.orc_krylov.argtypes = [C.c_int32, C.c_int32, C.c_int32, P, P, P, P, P, C.c_int32,
                                    C.c_double, C.c_double, C.c_int32, P, P, P, P]
        _lib.orc_ne_solve.restype = C.c_int32
        _lib.orc_ne_solve.argtypes = [C.c_int32, C.c_int32, P, P, P, P, P, P, C.c_int32,
                                      C.c_double, C.c_int32, C.c_double, C.c_int32, P, P, P]
        _lib.orc_nrsor.restype = None
        _lib.orc_nrsor.argtypes = [C.c_int32, C.c_int32, P, P, P, P, P, C.c_int32, C.c_double, P]
        _lib.orc_ls_krylov.restype = C.c_int32
        _lib.orc_ls_krylov.argtypes = [C.c_int32, C.c_int32, P, P, P, P, P, C.c_int32, C.c_double,
                                       C.c_double, C.c_int32, P, P, P]
        _lib.orc_ls_solve.restype = C.c_int32
        _lib.orc_ls_solve.argtypes = [C.c_int32, C.c_int32, P, P, P, P, P, P, C.c_int32, C.c_double,
                                      C.c_double, C.c_int32, P, P, P]
        _lib.orc_default_options.restype = None
        _lib.orc_default_options.argtypes = [P]
        _lib.orc_lp_solve.restype = C.c_int32
        _lib.orc_lp_solve.argtypes = [C.c_int32, C.c_int32, P, P, P, P, P, P, P, P, P, P, P]
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(C.c_uint64(x)))


def color_rows(m, n, row_ptr, col_idx, seed):
    """Returns (n_colors, color[m], perm[m], color_ptr[n_colors+1])."""
    rp, ci = _c(row_ptr, np.int64), _c(col_idx, np.int32)
    color = np.empty(m, np.int32)
    perm = np.empty(m, np.int32)
    cptr = np.empty(m + 1, np.int32)
    nc = lib().orc_color_rows(m, n, _p(rp), _p(ci), C.c_uint64(seed), _p(color), _p(perm), _p(cptr))
    if nc < 0:
        raise MemoryError("oracle coloring")
    return nc, color, perm, cptr[: nc + 1].copy()


def scale_rows(m, row_ptr, col_idx, val, d2):
    rp, ci, v, d = _c(row_ptr, np.int64), _c(col_idx, np.int32), _c(val, np.float64), _c(d2, np.float64)
    ahat = np.empty(v.size, np.float64)
    rho = np.empty(m, np.float64)
    lib().orc_scale_rows(m, _p(rp), _p(ci), _p(v), _p(d), _p(ahat), _p(rho))
    return ahat, rho


def nessor(m, n, row_ptr, col_idx, a, perm, g, ell=1, omega=1.0):
    """Algorithm 5: returns (z[m], u[n])."""
    args = [_c(row_ptr, np.int64), _c(col_idx, np.int32), _c(a, np.float64), _c(perm, np.int32),
            _c(g, np.float64)]
    z = np.empty(m, np.float64)
    u = np.empty(n, np.float64)
    lib().orc_nessor(m, n, *[_p(x) for x in args], ell, omega, _p(z), _p(u))
    return z, u


def nesor(m, n, row_ptr, col_idx, a, perm, g, ell=1, omega=1.0):
    """Algorithm 6: returns (z[n], y[m]) with z = A^T y."""
    args = [_c(row_ptr, np.int64), _c(col_idx, np.int32), _c(a, np.float64), _c(perm, np.int32),
            _c(g, np.float64)]
    z = np.empty(n, np.float64)
    y = np.empty(m, np.float64)
    lib().orc_nesor(m, n, *[_p(x) for x in args], ell, omega, _p(z), _p(y))
    return z, y


def nrsor(m, n, row_ptr, col_idx, a, perm, c, ell=1, omega=1.0):
    """NR-SOR for min ||A^T y - c||: returns y[m] = B c."""
    args = [_c(row_ptr, np.int64), _c(col_idx, np.int32), _c(a, np.float64), _c(perm, np.int32),
            _c(c, np.float64)]
    y = np.empty(m, np.float64)
    lib().orc_nrsor(m, n, *[_p(x) for x in args], ell, omega, _p(y))
    return y


def ls_krylov(m, n, row_ptr, col_idx, a, perm, r, ell=1, omega=1.0, tol=1e-10, maxit=None):
    """BA-GMRES (NR-SOR) on min ||A^T dy - r|| for a scaled A: (dw[n], dy[m], info)."""
    maxit = m if maxit is None else maxit
    args = [_c(row_ptr, np.int64), _c(col_idx, np.int32), _c(a, np.float64), _c(perm, np.int32),
            _c(r, np.float64)]
    dw = np.empty(n, np.float64)
    dy = np.empty(m, np.float64)
    info = KrylovInfo()
    lib().orc_ls_krylov(m, n, *[_p(x) for x in args], ell, omega, tol, maxit, _p(dw), _p(dy),
                        C.byref(info))
    return dw, dy, info.as_dict()


def ls_solve(m, n, row_ptr, col_idx, val, perm, d2, r, ell=1, omega=1.0, tol=1e-10, maxit=None):
    """Corrector least squares min ||diag(sqrt d2) A^T dy - r|| by BA-GMRES:
    (dy[m], dw[n], info)."""
    maxit = m if maxit is None else maxit
    args = [_c(row_ptr, np.int64), _c(col_idx, np.int32), _c(val, np.float64), _c(perm, np.int32),
            _c(d2, np.float64), _c(r, np.float64)]
    dy = np.empty(m, np.float64)
    dw = np.empty(n, np.float64)
    info = KrylovInfo()
    lib().orc_ls_solve(m, n, *[_p(x) for x in args], ell, omega, tol, maxit, _p(dy), _p(dw),
                       C.byref(info))
    return dy, dw, info.as_dict()


def krylov(method, m, n, row_ptr, col_idx, a, perm, f, ell=1, omega=1.0, tol=1e-10, maxit=None,
           history=False):
    """Krylov solve on an already scaled matrix: returns (dw[n], dy[m], info[, hist])."""
    maxit = m if maxit is None else maxit
    args = [_c(row_ptr, np.int64), _c(col_idx, np.int32), _c(a, np.float64), _c(perm, np.int32),
            _c(f, np.float64)]
    dw = np.empty(n, np.float64)
    dy = np.empty(m, np.float64)
    info = KrylovInfo()
    hist = np.full(maxit + 1, np.nan) if history else None
    lib().orc_krylov(method, m, n, *[_p(x) for x in args], ell, omega, tol, maxit, _p(dw), _p(dy),
                     C.byref(info), _p(hist))
    if history:
        return dw, dy, info.as_dict(), hist[: info.iters + 1]
    return dw, dy, info.as_dict()


def ne_solve(m, n, row_ptr, col_idx, val, perm, d2, f, ell=1, omega=1.0, method=MRNE, tol=1e-10,
             maxit=None):
    """Search-direction solve A diag(d2) A^T dy = f: returns (dy[m], dw[n], info)."""
    maxit = m if maxit is None else maxit
    args = [_c(row_ptr, np.int64), _c(col_idx, np.int32), _c(val, np.float64), _c(perm, np.int32),
            _c(d2, np.float64), _c(f, np.float64)]
    dy = np.empty(m, np.float64)
    dw = np.empty(n, np.float64)
    info = KrylovInfo()
    lib().orc_ne_solve(m, n, *[_p(x) for x in args], ell, omega, method, tol, maxit, _p(dy), _p(dw),
                       C.byref(info))
    return dy, dw, info.as_dict()


def default_options(**kw) -> Options:
    o = Options()
    lib().orc_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def lp_solve(m, n, row_ptr, col_idx, val, b, c, trace=False, **opts):
    """Algorithm 1.  Returns (x, y, s, info dict[, trace array (iters x TRACE_COLS)]);
    the trace columns are TRACE_FIELDS (see lpk_oracle.h)."""
    o = default_options(**opts)
    args = [_c(row_ptr, np.int64), _c(col_idx, np.int32), _c(val, np.float64), _c(b, np.float64),
            _c(c, np.float64)]
    x = np.empty(n, np.float64)
    y = np.empty(m, np.float64)
    s = np.empty(n, np.float64)
    info = Info()
    tr = np.full((max(o.max_ipm, 1), TRACE_COLS), np.nan) if trace else None
    lib().orc_lp_solve(m, n, *[_p(a) for a in args], C.byref(o), _p(x), _p(y), _p(s), C.byref(info),
                       _p(tr))
    d = info.as_dict()
    d["status_name"] = STATUS.get(d["status"], str(d["status"]))
    if trace:
        return x, y, s, d, tr[: info.ipm_iters]
    return x, y, s, d


def lp_solve_lp(lp, trace=False, **opts):
    """lp_solve on a gen.LP-like object (fields m, n, row_ptr, col_idx, val, b, c)."""
    return lp_solve(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, trace=trace, **opts)
