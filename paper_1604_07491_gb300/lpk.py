"""ctypes binding of liblpk.so (include/lpk.h).  Argument marshalling only.

Vectors may be torch tensors (CUDA tensors are passed as device pointers with
on_device=1; CPU tensors as host pointers) or numpy arrays (host pointers).
Every call goes through the C ABI; there is no Python or CPU compute path, and
loading fails loudly when the shared library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblpk.so")

OK, MAX_IPM_ITER, KRYLOV_STALL, DIVERGED, BREAKDOWN, TIMEOUT = 0, 1, 2, 3, 4, 5
EMPTY_ROW_INCONSISTENT, EMPTY_COL_UNBOUNDED, INVALID_ARG, OOM, CUDA_ERROR = 6, 7, 8, 9, 10
STATUS = {0: "OK", 1: "MAX_IPM_ITER", 2: "KRYLOV_STALL", 3: "DIVERGED", 4: "BREAKDOWN", 5: "TIMEOUT",
          6: "EMPTY_ROW_INCONSISTENT", 7: "EMPTY_COL_UNBOUNDED", 8: "INVALID_ARG", 9: "OOM",
          10: "CUDA_ERROR"}
MRNE, CGNE, ABGMRES = 0, 1, 2
EXEC_AUTO, EXEC_GRID, EXEC_CLUSTER, EXEC_BATCH, EXEC_NO_RESIDENT = 0, 1, 2, 3, 4
EXEC_U_SHARED, EXEC_U_GLOBAL = 8, 16
FP64, MIXED = 0, 1
NE_SSOR, NE_SOR = 0, 1

# every symbol include/lpk.h declares
EXPORTS = ["lpk_create", "lpk_destroy", "lpk_last_error", "lpk_default_options", "lpk_get_stats",
           "lpk_reset_stats", "lpk_set_exec", "lpk_set_wait_limit", "lpk_set_phase_timing", "lpk_prepare",
           "lpk_problem_free", "lpk_problem_dims", "lpk_problem_coloring", "lpk_scale_rows",
           "lpk_spmv", "lpk_sweep", "lpk_ne_solve", "lpk_ne_solve_noalloc", "lpk_ls_solve", "lpk_lp_solve",
           "lpk_lp_solve_batch", "lpk_server_default_config", "lpk_server_create", "lpk_server_destroy",
           "lpk_server_now", "lpk_server_submit", "lpk_server_wait", "lpk_server_stats"]


class LpkError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Matrix(C.Structure):
    _fields_ = [("m", C.c_int32), ("n", C.c_int32), ("nnz", C.c_int64), ("row_ptr", C.c_void_p),
                ("col_idx", C.c_void_p), ("val", C.c_void_p), ("on_device", C.c_int32),
                ("reserved", C.c_int32)]


class Options(C.Structure):
    _fields_ = [("tol", C.c_double), ("eta", C.c_double), ("phi", C.c_double),
                ("sigma_max", C.c_double), ("eps_in0", C.c_double), ("omega", C.c_double),
                ("start_tol", C.c_double), ("backtrack", C.c_double), ("max_ipm", C.c_int32),
                ("max_krylov", C.c_int32), ("inner_sweeps", C.c_int32), ("solver", C.c_int32),
                ("precision", C.c_int32), ("verbose", C.c_int32), ("color_seed", C.c_uint64),
                ("corrector", C.c_int32), ("max_correctors", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("status", C.c_int32), ("ipm_iters", C.c_int32), ("krylov_iters_total", C.c_int64),
                ("n_colors", C.c_int32), ("krylov_failures", C.c_int32), ("gamma", C.c_double),
                ("rel_gap", C.c_double), ("pinf", C.c_double), ("dinf", C.c_double),
                ("mu", C.c_double), ("obj_primal", C.c_double), ("obj_dual", C.c_double),
                ("solve_ms", C.c_double), ("correctors", C.c_int32), ("reserved", C.c_int32)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["status_name"] = STATUS.get(d["status"], str(d["status"]))
        return d


class KrylovInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("restarts", C.c_int32),
                ("breakdown", C.c_int32), ("res0", C.c_double), ("res", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(C.Structure):
    _fields_ = [("launches", C.c_int64), ("krylov_launches", C.c_int64), ("krylov_ms", C.c_double),
                ("krylov_iters", C.c_int64), ("sweep_passes", C.c_int64), ("row_passes", C.c_int64),
                ("csc_passes", C.c_int64), ("barriers", C.c_int64), ("last_cluster_size", C.c_int32),
                ("last_resident", C.c_int32), ("basis_passes", C.c_int64), ("spmv_launches", C.c_int64),
                ("spmv_ms", C.c_double), ("phase_ms", C.c_double * 4), ("last_u_global", C.c_int32),
                ("reserved", C.c_int32), ("tune_probes", C.c_int64), ("tune_cache_hits", C.c_int64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "phase_ms"}
        d["phase_ms"] = list(self.phase_ms)
        return d


class ServerConfig(C.Structure):
    _fields_ = [("device", C.c_int32), ("lanes", C.c_int32), ("mem_budget", C.c_int64),
                ("color_seed", C.c_uint64)]


class RequestResult(C.Structure):
    _fields_ = [("info", Info), ("status", C.c_int32), ("lane", C.c_int32), ("t_submit", C.c_double),
                ("t_start", C.c_double), ("t_end", C.c_double), ("mem_bytes", C.c_int64),
                ("error", C.c_char * 256)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("info", "error")}
        d["info"] = self.info.as_dict()
        d["status_name"] = STATUS.get(self.status, str(self.status))
        d["error"] = self.error.decode(errors="replace")
        return d


class ServerStats(C.Structure):
    _fields_ = [("pending", C.c_int64), ("running", C.c_int64), ("completed", C.c_int64),
                ("mem_in_use", C.c_int64), ("mem_peak", C.c_int64), ("mem_budget", C.c_int64),
                ("lanes", C.c_int32), ("reserved", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


_lib = None


def load():
    """Load liblpk.so (built by paper_1604_07491_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run paper_1604_07491_gb300.build.build() first")
    lib = C.CDLL(LIB_PATH)
    P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "lpk_create": (I32, [C.POINTER(P), I32, P]),
        "lpk_destroy": (None, [P]),
        "lpk_last_error": (C.c_char_p, [P]),
        "lpk_default_options": (None, [C.POINTER(Options)]),
        "lpk_get_stats": (I32, [P, C.POINTER(Stats)]),
        "lpk_reset_stats": (I32, [P]),
        "lpk_set_exec": (I32, [P, I32, I32]),
        "lpk_set_wait_limit": (I32, [P, D, I64]),
        "lpk_set_phase_timing": (I32, [P, I32]),
        "lpk_prepare": (I32, [P, C.POINTER(Matrix), C.c_uint64, C.POINTER(P)]),
        "lpk_problem_free": (None, [P]),
        "lpk_problem_dims": (I32, [P, P, P, P, P]),
        "lpk_problem_coloring": (I32, [P, P, P, P, P]),
        "lpk_scale_rows": (I32, [P, P, P, P, P, I32]),
        "lpk_spmv": (I32, [P, P, I32, P, P, I32]),
        "lpk_sweep": (I32, [P, P, P, P, I32, I32, D, I32, P, P, I32]),
        "lpk_ne_solve": (I32, [P, P, P, P, I32, D, I32, I32, D, I32, P, P, C.POINTER(KrylovInfo), I32]),
        "lpk_lp_solve": (I32, [P, P, P, P, C.POINTER(Options), P, P, P, C.POINTER(Info), I32]),
        "lpk_ls_solve": (I32, [P, P, P, P, I32, D, I32, D, I32, P, P, C.POINTER(KrylovInfo), I32]),
        "lpk_ne_solve_noalloc": (I32, [P, P, P, P, I32, D, I32, I32, D, I32, P, P,
                                       C.POINTER(KrylovInfo)]),
        "lpk_lp_solve_batch": (I32, [I32, C.POINTER(P), C.POINTER(P), C.POINTER(P), C.POINTER(Options),
                                     C.POINTER(P), C.POINTER(P), C.POINTER(P), C.POINTER(Info), I32]),
        "lpk_server_default_config": (None, [C.POINTER(ServerConfig)]),
        "lpk_server_create": (I32, [C.POINTER(P), C.POINTER(ServerConfig)]),
        "lpk_server_destroy": (None, [P]),
        "lpk_server_now": (D, [P]),
        "lpk_server_submit": (I32, [P, C.POINTER(Matrix), P, P, C.POINTER(Options), C.POINTER(I64)]),
        "lpk_server_wait": (I32, [P, I64, D, P, P, P, C.POINTER(RequestResult)]),
        "lpk_server_stats": (I32, [P, C.POINTER(ServerStats)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, on_device) of a torch tensor or numpy array (contiguous float64 etc)."""
    if x is None:
        return None, 0
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(x.data_ptr()), int(x.is_cuda)
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be contiguous")
    return C.c_void_p(x.ctypes.data), 0


def _check(ctx, st):
    if st != OK:
        raise LpkError(st, load().lpk_last_error(ctx).decode())


def _like(ref, n, dtype="float64"):
    if _is_torch(ref):
        import torch
        return torch.empty(n, dtype=getattr(torch, dtype), device=ref.device)
    return np.empty(n, dtype=dtype)


def _f64(x):
    if _is_torch(x):
        import torch
        assert x.dtype == torch.float64, "float64 tensor expected"
        return x.contiguous()
    return np.ascontiguousarray(x, dtype=np.float64)


class Context:
    """lpk_create / lpk_destroy.  stream: a cudaStream_t handle (int) or None
    for the current torch stream of `device`."""

    def __init__(self, device: int = 0, stream=None):
        lib = load()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        import weakref
        self.device = device
        self._problems = weakref.WeakSet()
        self._h = C.c_void_p()
        st = lib.lpk_create(C.byref(self._h), device, C.c_void_p(stream))
        if st != OK:
            raise LpkError(st, "lpk_create failed")

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            for p in list(self._problems):   # problems are freed before their context
                p.free()
            load().lpk_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return load().lpk_last_error(self._h).decode()

    def stats(self) -> dict:
        st = Stats()
        load().lpk_get_stats(self._h, C.byref(st))
        return st.as_dict()

    def reset_stats(self):
        load().lpk_reset_stats(self._h)

    def set_wait_limit(self, seconds=5.0, test_stall_barrier=0):
        """Bound of every grid-barrier wait; test_stall_barrier (testing only)
        makes every wait on that grid barrier run out (lpk_set_wait_limit)."""
        _check(self._h, load().lpk_set_wait_limit(self._h, float(seconds), int(test_stall_barrier)))

    def set_phase_timing(self, on=True):
        """Time the persistent kernel's barrier intervals by phase kind
        (stats()["phase_ms"]; lpk_set_phase_timing)."""
        _check(self._h, load().lpk_set_phase_timing(self._h, int(bool(on))))

    def set_exec(self, exec_mode=EXEC_AUTO, cluster_size=0):
        """Krylov kernel path: EXEC_AUTO, EXEC_GRID, EXEC_CLUSTER or EXEC_BATCH
        (cluster size 0/2/4/8/16; or-ing EXEC_NO_RESIDENT disables the row cache,
        EXEC_U_SHARED / EXEC_U_GLOBAL fix where the cluster path keeps u)."""
        _check(self._h, load().lpk_set_exec(self._h, exec_mode, cluster_size))


def default_options(**kw) -> Options:
    o = Options()
    load().lpk_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


class Problem:
    """lpk_prepare: CSR (row_ptr int64, col_idx int32, val float64) on host or device."""

    def __init__(self, ctx: Context, m, n, row_ptr, col_idx, val, color_seed=0x5EED):
        lib = load()
        self.ctx = ctx
        self.m, self.n = int(m), int(n)
        self._keep = (row_ptr, col_idx, val)
        prp, dev = _ptr(row_ptr)
        pci, _ = _ptr(col_idx)
        pv, _ = _ptr(val)
        nnz = int(row_ptr[-1])
        self.nnz = nnz
        A = Matrix(m=self.m, n=self.n, nnz=nnz, row_ptr=prp, col_idx=pci, val=pv, on_device=dev)
        self._h = C.c_void_p()
        _check(ctx.handle, lib.lpk_prepare(ctx.handle, C.byref(A), C.c_uint64(color_seed),
                                           C.byref(self._h)))
        self._keep = None
        ctx._problems.add(self)
        nc = C.c_int32()
        lib.lpk_problem_dims(self._h, None, None, None, C.byref(nc))
        self.n_colors = nc.value

    @classmethod
    def from_lp(cls, ctx, lp, color_seed=0x5EED, device=None):
        """Build from a gen.LP; device=None keeps host arrays."""
        rp, ci, v = lp.row_ptr, lp.col_idx, lp.val
        if device is not None:
            import torch
            rp = torch.from_numpy(rp).to(device)
            ci = torch.from_numpy(ci).to(device)
            v = torch.from_numpy(v).to(device)
        return cls(ctx, lp.m, lp.n, rp, ci, v, color_seed)

    def free(self):
        if self._h:
            load().lpk_problem_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def coloring(self):
        """(color[m] int32, perm[m'] int32, color_ptr[n_colors+1] int32) on the host."""
        color = np.empty(self.m, np.int32)
        mr = C.c_int32()
        perm = np.empty(self.m, np.int32)
        cptr = np.empty(self.n_colors + 1, np.int32)
        _check(self.ctx.handle, load().lpk_problem_coloring(
            self.ctx.handle, self._h, C.c_void_p(color.ctypes.data), C.c_void_p(perm.ctypes.data),
            C.c_void_p(cptr.ctypes.data)))
        del mr
        return color, perm[: int(cptr[-1])], cptr

    def scale_rows(self, d2, with_ahat=False):
        d2 = _f64(d2)
        rho = _like(d2, self.m)
        ahat = _like(d2, self.nnz) if with_ahat else None
        p, dev = _ptr(d2)
        _check(self.ctx.handle, load().lpk_scale_rows(self.ctx.handle, self._h, p, _ptr(rho)[0],
                                                      _ptr(ahat)[0], dev))
        return (rho, ahat) if with_ahat else rho

    def spmv(self, x, transpose=False):
        x = _f64(x)
        y = _like(x, self.n if transpose else self.m)
        p, dev = _ptr(x)
        _check(self.ctx.handle, load().lpk_spmv(self.ctx.handle, self._h, int(bool(transpose)), p,
                                                _ptr(y)[0], dev))
        return y

    def sweep(self, d2, g, kind=NE_SSOR, inner_sweeps=1, omega=1.0, precision=FP64):
        """Returns (z[m], u[n]) of Algorithm 5 (NE_SSOR) or 6 (NE_SOR; u is the
        w-space iterate, z the row corrections)."""
        d2, g = _f64(d2), _f64(g)
        z = _like(g, self.m)
        u = _like(g, self.n)
        p, dev = _ptr(d2)
        _check(self.ctx.handle, load().lpk_sweep(self.ctx.handle, self._h, p, _ptr(g)[0], kind,
                                                 inner_sweeps, omega, precision, _ptr(z)[0],
                                                 _ptr(u)[0], dev))
        return z, u

    def ne_solve(self, d2, f, inner_sweeps=1, omega=1.0, solver=MRNE, precision=FP64, tol=1e-10,
                 max_iter=0):
        """Returns (dy[m], dw[n], info dict)."""
        d2, f = _f64(d2), _f64(f)
        dy = _like(f, self.m)
        dw = _like(f, self.n)
        ki = KrylovInfo()
        p, dev = _ptr(d2)
        _check(self.ctx.handle, load().lpk_ne_solve(self.ctx.handle, self._h, p, _ptr(f)[0],
                                                    inner_sweeps, omega, solver, precision, tol,
                                                    max_iter, _ptr(dy)[0], _ptr(dw)[0],
                                                    C.byref(ki), dev))
        return dy, dw, ki.as_dict()

    def ls_solve(self, d2, r, inner_sweeps=2, omega=1.0, precision=FP64, tol=1e-10, max_iter=0):
        """Corrector least squares min ||diag(sqrt d2) A^T dy - r|| by BA-GMRES
        (NR-SOR): returns (dy[m], dw[n], krylov info dict)."""
        d2, r = _f64(d2), _f64(r)
        dy, dw = _like(r, self.m), _like(r, self.n)
        ki = KrylovInfo()
        p, dev = _ptr(d2)
        _check(self.ctx.handle, load().lpk_ls_solve(self.ctx.handle, self._h, p, _ptr(r)[0], inner_sweeps, omega,
                                                    precision, tol, max_iter, _ptr(dy)[0], _ptr(dw)[0],
                                                    C.byref(ki), dev))
        return dy, dw, ki.as_dict()

    def ne_solve_noalloc(self, d2, f, dy, dw=None, inner_sweeps=1, omega=1.0, solver=MRNE,
                         precision=FP64, tol=1e-10, max_iter=0):
        """lpk_ne_solve_noalloc: device tensors in and out (dy, dw preallocated by
        the caller); the library allocates nothing.  Returns the info dict.
        The C call takes no lengths, so the tensors are checked here: float64,
        contiguous, on the context's GPU, d2/dw of n entries and f/dy of m."""
        import torch
        for name, t, size in (("d2", d2, self.n), ("f", f, self.m), ("dy", dy, self.m), ("dw", dw, self.n)):
            if t is None and name == "dw":
                continue
            if not (_is_torch(t) and t.is_cuda and t.device.index == self.ctx.device):
                raise ValueError(f"{name} must be a CUDA tensor on device {self.ctx.device}")
            if t.dtype != torch.float64 or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous float64 tensor")
            if t.numel() < size:
                raise ValueError(f"{name} has {t.numel()} entries, needs {size}")
        ki = KrylovInfo()
        _check(self.ctx.handle, load().lpk_ne_solve_noalloc(
            self.ctx.handle, self._h, _ptr(d2)[0], _ptr(f)[0], inner_sweeps, omega, solver, precision,
            tol, max_iter, _ptr(dy)[0], _ptr(dw)[0], C.byref(ki)))
        return ki.as_dict()

    def lp_solve(self, b, c, options: Options | None = None, out=None, **kw):
        """Returns (x[n], y[m], s[n], info dict).  Status codes other than OK,
        MAX_IPM_ITER and DIVERGED raise LpkError; those three are in info."""
        b, c = _f64(b), _f64(c)
        o = options if options is not None else default_options(**kw)
        if out is None:
            x, y, s = _like(c, self.n), _like(b, self.m), _like(c, self.n)
        else:
            x, y, s = out
        info = Info()
        p, dev = _ptr(b)
        st = load().lpk_lp_solve(self.ctx.handle, self._h, p, _ptr(c)[0], C.byref(o), _ptr(x)[0],
                                 _ptr(y)[0], _ptr(s)[0], C.byref(info), dev)
        if st not in (OK, MAX_IPM_ITER, DIVERGED):
            _check(self.ctx.handle, st)
        return x, y, s, info.as_dict()


def solve_batch(problems, bs, cs, outs=None, options: Options | None = None, **kw):
    """lpk_lp_solve_batch: LP i = (problems[i], bs[i], cs[i]), each problem on
    its own Context, solved side by side.  Returns a list of (x, y, s, info)."""
    k = len(problems)
    o = options if options is not None else default_options(**kw)
    bs = [_f64(b) for b in bs]
    cs = [_f64(c) for c in cs]
    if outs is None:
        outs = [(_like(cs[i], p.n), _like(bs[i], p.m), _like(cs[i], p.n)) for i, p in enumerate(problems)]
    devs = {_ptr(v)[1] for v in bs + cs + [a for t in outs for a in t]}
    if len(devs) > 1:
        raise ValueError("all vectors must be on the device or all on the host")
    arr = C.c_void_p * max(k, 1)
    infos = (Info * max(k, 1))()
    st = load().lpk_lp_solve_batch(
        k, arr(*[p._h for p in problems]), arr(*[_ptr(b)[0] for b in bs]), arr(*[_ptr(c)[0] for c in cs]),
        C.byref(o), arr(*[_ptr(t[0])[0] for t in outs]), arr(*[_ptr(t[1])[0] for t in outs]),
        arr(*[_ptr(t[2])[0] for t in outs]), infos, devs.pop() if devs else 0)
    res = [(outs[i][0], outs[i][1], outs[i][2], infos[i].as_dict()) for i in range(k)]
    if st not in (OK, MAX_IPM_ITER, DIVERGED, KRYLOV_STALL) and k > 0:
        bad = [i for i in range(k) if infos[i].status == st]
        if bad:   # a solve failed
            _check(problems[bad[0]].ctx.handle, st)
        # rejected before anything ran: the offending context holds the message
        msgs = sorted({p.ctx.last_error() for p in problems} - {""})
        raise LpkError(st, "; ".join(msgs))
    return res


class Server:
    """lpk_server_*: continuous batching of LPs on one GPU (host CSR in,
    host vectors out)."""

    def __init__(self, device=0, lanes=16, mem_budget=0, color_seed=0x5EED):
        lib = load()
        cfg = ServerConfig()
        lib.lpk_server_default_config(C.byref(cfg))
        cfg.device, cfg.lanes, cfg.mem_budget, cfg.color_seed = device, lanes, int(mem_budget), color_seed
        self._h = C.c_void_p()
        st = lib.lpk_server_create(C.byref(self._h), C.byref(cfg))
        if st != OK:
            raise LpkError(st, "lpk_server_create failed")
        self._dims = {}

    def submit(self, m, n, row_ptr, col_idx, val, b, c, options: Options | None = None, **kw) -> int:
        rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        ci = np.ascontiguousarray(col_idx, dtype=np.int32)
        v = np.ascontiguousarray(val, dtype=np.float64)
        b, c = np.ascontiguousarray(b, np.float64), np.ascontiguousarray(c, np.float64)
        A = Matrix(m=int(m), n=int(n), nnz=int(rp[-1]), row_ptr=rp.ctypes.data, col_idx=ci.ctypes.data,
                   val=v.ctypes.data, on_device=0)
        o = options if options is not None else default_options(**kw)
        t = C.c_int64()
        st = load().lpk_server_submit(self._h, C.byref(A), C.c_void_p(b.ctypes.data),
                                      C.c_void_p(c.ctypes.data), C.byref(o), C.byref(t))
        if st != OK:
            raise LpkError(st, "lpk_server_submit failed")
        self._dims[t.value] = (int(m), int(n))
        return t.value

    def submit_lp(self, lp, **kw) -> int:
        return self.submit(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, **kw)

    def wait(self, ticket, timeout=-1.0):
        """(x, y, s, result dict), or None if not ready within timeout seconds."""
        m, n = self._dims[ticket]
        x, y, s = np.empty(n), np.empty(m), np.empty(n)
        r = RequestResult()
        st = load().lpk_server_wait(self._h, ticket, float(timeout), C.c_void_p(x.ctypes.data),
                                    C.c_void_p(y.ctypes.data), C.c_void_p(s.ctypes.data), C.byref(r))
        if st == TIMEOUT:
            return None
        if st != OK:
            raise LpkError(st, "lpk_server_wait failed")
        del self._dims[ticket]
        return x, y, s, r.as_dict()

    def now(self) -> float:
        return load().lpk_server_now(self._h)

    def stats(self) -> dict:
        st = ServerStats()
        load().lpk_server_stats(self._h, C.byref(st))
        return st.as_dict()

    def close(self):
        if self._h:
            load().lpk_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
