"""Python binding of libphipm (include/phipm.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels; this module turns
torch tensors (device memory, streams) and numpy arrays into the plain
pointers and sizes of the C ABI.  If the library is missing or cannot load, the
import of the native library raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import build as _build

c_int32, c_int64, c_double, c_void_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, EMAXSTEPS, ETIMEOUT, EBOUNDS, ETOOLARGE, ENOTRUN = range(10)
F64, F32_MIXED, F64_PAIR = 0, 1, 2
OP_CSR, OP_STENCIL, OP_FUNCTION = 0, 1, 2
FN_VARCOEF_CONVDIFF = 0
CTRL_PAPER, CTRL_LEARNED, CTRL_FIXED_M, CTRL_LEARNED_STEPS = 0, 1, 2, 3      # phipm_controller
M_MAX, P_MAX, NOALLOC_MAX_N = 64, 8, 8192
MLP_PARAMS, CONTROLLER_FLOATS = 4866, 4886


class CsrC(ctypes.Structure):
    _fields_ = [("n", c_int32), ("nnz", c_int32), ("rowptr", c_void_p), ("colind", c_void_p), ("values", c_void_p)]


class StencilC(ctypes.Structure):
    _fields_ = [("ndim", c_int32), ("nx", c_int32), ("ny", c_int32), ("nz", c_int32), ("c_center", c_double),
                ("c_minus", c_double * 3), ("c_plus", c_double * 3)]


class FunctionC(ctypes.Structure):
    _fields_ = [("fn", c_int32), ("ndim", c_int32), ("nx", c_int32), ("ny", c_int32), ("nz", c_int32),
                ("reserved", c_int32), ("field", c_void_p * 4), ("scal", c_double * 6), ("norm_inf", c_double),
                ("cost", c_int64)]


class OperatorC(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("csr", CsrC), ("st", StencilC), ("fn", FunctionC)]


class StatsC(ctypes.Structure):
    _fields_ = [("steps", c_int64), ("rejects", c_int64), ("matvecs", c_int64), ("expms", c_int64),
                ("err_est_sum", c_double), ("krylov_steps", c_int64), ("gs_vectors", c_int64),
                ("kernel_ms", c_double), ("reorth_vectors", c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class TraceRecordC(ctypes.Structure):
    _fields_ = [("problem", c_int32), ("step", c_int32), ("attempt", c_int32), ("accepted", c_int32),
                ("m_req", c_int32), ("m_used", c_int32), ("p", c_int32), ("n", c_int32),
                ("t", c_double), ("t_end", c_double), ("tau", c_double), ("eps", c_double), ("omega", c_double),
                ("norm_a", c_double), ("tol", c_double), ("m_new", c_double), ("source", c_int32),
                ("rejects_prev", c_int32)]


class TuneEntryC(ctypes.Structure):
    _fields_ = [("team", c_int32), ("reserved", c_int32), ("kernel_ms", c_double)]


class ParamsC(ctypes.Structure):
    _fields_ = [("gamma", c_double), ("delta", c_double), ("m_init", c_int32), ("m_max", c_int32),
                ("theta13", c_double), ("breakdown_tol", c_double), ("max_steps", c_int64),
                ("max_rejects", c_int64), ("precision", c_int32), ("controller", c_int32),
                ("timeout_cycles", c_int64), ("stencil_stage", c_int32), ("expm_pade", c_int32),
                ("expm_action", c_int32)]


_LIB = None


def header_functions() -> list:
    """Names of the functions declared in include/phipm.h."""
    hdr = open(os.path.join(_build.ROOT, "include", "phipm.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(phipm_[a-z_]+)\s*\(", hdr)))


def lib(build_if_needed: bool = True):
    """Load libphipm.so (building it first when sources are newer)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.build() if build_if_needed else _build.LIB
    L = ctypes.CDLL(path)
    L.phipm_default_params.argtypes = [ctypes.POINTER(ParamsC)]
    L.phipm_default_params.restype = None
    L.phipm_create.argtypes = [ctypes.POINTER(c_void_p), ctypes.POINTER(ParamsC)]
    L.phipm_create.restype = c_int32
    L.phipm_destroy.argtypes = [c_void_p]
    L.phipm_destroy.restype = None
    L.phipm_last_error.argtypes = [c_void_p]
    L.phipm_last_error.restype = ctypes.c_char_p
    L.phipm_set_params.argtypes = [c_void_p, ctypes.POINTER(ParamsC)]
    L.phipm_set_params.restype = c_int32
    L.phipm_solve.argtypes = [c_void_p, c_double, ctypes.POINTER(OperatorC), c_int32, ctypes.POINTER(c_void_p),
                              c_double, c_int32, c_void_p, ctypes.POINTER(StatsC), c_void_p]
    L.phipm_solve.restype = c_int32
    L.phipm_solve_host.argtypes = L.phipm_solve.argtypes
    L.phipm_solve_host.restype = c_int32
    L.phipm_solve_batched.argtypes = [c_void_p, c_int32, ctypes.POINTER(c_double), ctypes.POINTER(OperatorC),
                                      ctypes.POINTER(c_int32), ctypes.POINTER(ctypes.POINTER(c_void_p)),
                                      ctypes.POINTER(c_double), ctypes.POINTER(c_int32), ctypes.POINTER(c_void_p),
                                      ctypes.POINTER(StatsC), ctypes.POINTER(c_int32), c_void_p]
    L.phipm_solve_batched.restype = c_int32
    L.phipm_solve_noalloc.argtypes = [c_double, ctypes.POINTER(OperatorC), c_int32, ctypes.POINTER(c_void_p),
                                      c_double, c_int32, c_void_p, ctypes.POINTER(StatsC), c_void_p]
    L.phipm_solve_noalloc.restype = c_int32
    L.phipm_trace_enable.argtypes = [c_void_p, c_int64]
    L.phipm_trace_enable.restype = c_int32
    L.phipm_trace_read.argtypes = [c_void_p, ctypes.POINTER(TraceRecordC), c_int64, ctypes.POINTER(c_int64)]
    L.phipm_trace_read.restype = c_int32
    L.phipm_set_controller_weights.argtypes = [c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.c_size_t]
    L.phipm_set_controller_weights.restype = c_int32
    L.phipm_mlp_forward.argtypes = [c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p]
    L.phipm_mlp_forward.restype = c_int32
    L.phipm_mlp_grad.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p]
    L.phipm_mlp_grad.restype = c_int32
    L.phipm_mlp_train.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int32,
                                  c_int64, ctypes.c_float, ctypes.POINTER(ctypes.c_float), c_void_p]
    L.phipm_mlp_train.restype = c_int32
    L.phipm_autotune.argtypes = [c_void_p, c_double, ctypes.POINTER(OperatorC), c_int32, ctypes.POINTER(c_void_p),
                                 c_double, c_int32, c_void_p, ctypes.POINTER(TuneEntryC), c_int32,
                                 ctypes.POINTER(c_int32), c_void_p]
    L.phipm_autotune.restype = c_int32
    L.phipm_autotune_batched.argtypes = [c_void_p, c_int32, ctypes.POINTER(c_double), ctypes.POINTER(OperatorC),
                                         ctypes.POINTER(c_int32), ctypes.POINTER(ctypes.POINTER(c_void_p)),
                                         ctypes.POINTER(c_double), ctypes.POINTER(c_int32), ctypes.POINTER(c_void_p),
                                         ctypes.POINTER(TuneEntryC), c_int32, ctypes.POINTER(c_int32), c_void_p]
    L.phipm_autotune_batched.restype = c_int32
    L.phipm_set_team.argtypes = [c_void_p, c_int32]
    L.phipm_set_team.restype = c_int32
    L.phipm_team_for.argtypes = [c_void_p, c_int32, c_int32, c_int32]
    L.phipm_team_for.restype = c_int32
    L.phipm_batched_team.argtypes = [c_void_p]
    L.phipm_batched_team.restype = c_int32
    L.phipm_tune_save.argtypes = [c_void_p, ctypes.c_char_p]
    L.phipm_tune_save.restype = c_int32
    L.phipm_tune_load.argtypes = [c_void_p, ctypes.c_char_p]
    L.phipm_tune_load.restype = c_int32
    _LIB = L
    return L


class PhipmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"phipm status {status}: {msg}")
        self.status = status


def default_params() -> ParamsC:
    p = ParamsC()
    lib().phipm_default_params(ctypes.byref(p))
    return p


# --------------------------------------------------------------------------------------
# operators
# --------------------------------------------------------------------------------------
class DeviceOperator:
    """A on the device: CSR arrays as torch tensors (int32 / int32 / float64) or stencil coefficients."""

    def __init__(self, op, device="cuda", arrays=None):
        """arrays: optional (rowptr, colind, values) device tensors already holding op's CSR
        arrays (e.g. views of one packed buffer); otherwise they are copied from op."""
        import torch
        self.src = op
        self.c = OperatorC()
        if hasattr(op, "fields"):              # a built-in matrix-free function with its data
            self.fields = [None if f is None else torch.as_tensor(np.ascontiguousarray(f, dtype=np.float64)).to(device)
                           for f in op.fields]
            self.c.kind = OP_FUNCTION
            self.c.fn = function_c(op, [0 if f is None else f.data_ptr() for f in self.fields])
            self.n = int(op.n)
        elif hasattr(op, "rowptr"):
            if arrays is not None:
                self.rowptr, self.colind, self.values = arrays
            else:
                self.rowptr = torch.as_tensor(np.asarray(op.rowptr, dtype=np.int32)).to(device)
                self.colind = torch.as_tensor(np.asarray(op.colind, dtype=np.int32)).to(device)
                self.values = torch.as_tensor(np.asarray(op.values, dtype=np.float64)).to(device)
            self.c.kind = OP_CSR
            self.c.csr = CsrC(int(op.n), int(self.values.numel()), self.rowptr.data_ptr(), self.colind.data_ptr(),
                              self.values.data_ptr())
            self.n = int(op.n)
        else:
            self.c.kind = OP_STENCIL
            self.c.st = stencil_c(op)
            self.n = int(op.n)


def function_c(op, ptrs) -> FunctionC:
    """The C descriptor of a matrix-free operator object (fn id, grid, scalars, optional
    norm bound and cost) with its fields at the given device addresses."""
    c = FunctionC()
    c.fn = int(op.fn)
    c.ndim, c.nx, c.ny, c.nz = int(op.ndim), int(op.nx), int(op.ny), int(op.nz)
    for d in range(4):
        c.field[d] = ptrs[d] if d < len(ptrs) else 0
    for d in range(6):
        c.scal[d] = float(op.scal[d])
    c.norm_inf = float(getattr(op, "norm_bound", 0.0))
    c.cost = int(getattr(op, "cost", 0))
    return c


def stencil_c(st) -> StencilC:
    c = StencilC()
    c.ndim, c.nx, c.ny, c.nz = int(st.ndim), int(st.nx), int(st.ny), int(st.nz)
    c.c_center = float(st.c_center)
    for d in range(3):
        c.c_minus[d] = float(st.c_minus[d])
        c.c_plus[d] = float(st.c_plus[d])
    return c


class HostOperator:
    """A in host memory (for phipm_solve_host)."""

    def __init__(self, op):
        self.c = OperatorC()
        if hasattr(op, "rowptr"):
            self.rowptr = np.ascontiguousarray(op.rowptr, dtype=np.int32)
            self.colind = np.ascontiguousarray(op.colind, dtype=np.int32)
            self.values = np.ascontiguousarray(op.values, dtype=np.float64)
            self.c.kind = OP_CSR
            self.c.csr = CsrC(int(op.n), int(self.values.size), self.rowptr.ctypes.data, self.colind.ctypes.data,
                              self.values.ctypes.data)
        else:
            self.c.kind = OP_STENCIL
            self.c.st = stencil_c(op)
        self.n = int(op.n)


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return c_void_p(s.cuda_stream)


# --------------------------------------------------------------------------------------
# solver handle
# --------------------------------------------------------------------------------------
class Phipm:
    """A library handle: owns the device workspace.

    precision: "f64" (PHIPM_F64, IEEE FP64), "f64pair" (PHIPM_F64_PAIR, FP64-class
    accuracy from float pairs on the FP32 pipe) or "f32" (PHIPM_F32_MIXED); other
    keyword arguments override phipm_params fields (gamma, delta, m_init, ...)."""

    def __init__(self, precision: str = "f64", **overrides):
        L = lib()
        self.params = default_params()
        self.params.precision = {"f64": F64, "f32": F32_MIXED, "f64pair": F64_PAIR}[precision]
        for k, v in overrides.items():
            setattr(self.params, k, v)
        h = c_void_p()
        st = L.phipm_create(ctypes.byref(h), ctypes.byref(self.params))
        if st != OK:
            raise PhipmError(st, "phipm_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().phipm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return lib().phipm_last_error(self.h).decode()

    def _check(self, st):
        if st != OK:
            raise PhipmError(st, self.last_error())

    def solve(self, t_end: float, A: DeviceOperator, b: list, tol: float = 1e-7, symm: int = -1, out=None,
              stream=None, check: bool = True):
        """u(t_end) for device tensors b[k] (float64, length n).  Returns (u, stats dict, status)."""
        import torch
        n = A.n
        p = len(b) - 1
        for x in b:
            if x.dtype != torch.float64 or not x.is_cuda or x.numel() != n or not x.is_contiguous():
                raise ValueError("b[k] must be contiguous float64 CUDA tensors of length n")
        u = out if out is not None else torch.empty(n, dtype=torch.float64, device=b[0].device)
        bp = (c_void_p * (p + 1))(*[x.data_ptr() for x in b])
        stats = StatsC()
        st = lib().phipm_solve(self.h, float(t_end), ctypes.byref(A.c), p, bp, float(tol), int(symm),
                               c_void_p(u.data_ptr()), ctypes.byref(stats), _stream_ptr(stream))
        if check:
            self._check(st)
        return u, stats.as_dict(), st

    def autotune(self, t_end: float, A: DeviceOperator, b: list, tol: float = 1e-7, symm: int = -1, out=None,
                 stream=None) -> list:
        """phipm_autotune: time each candidate team size on this problem and keep the fastest
        for its size class.  Returns [(team, kernel_ms), ...] in the order tried."""
        import torch
        n = A.n
        p = len(b) - 1
        u = out if out is not None else torch.empty(n, dtype=torch.float64, device=b[0].device)
        bp = (c_void_p * (p + 1))(*[x.data_ptr() for x in b])
        rep = (TuneEntryC * 16)()
        cnt = c_int32(0)
        st = lib().phipm_autotune(self.h, float(t_end), ctypes.byref(A.c), p, bp, float(tol), int(symm),
                                  c_void_p(u.data_ptr()), rep, 16, ctypes.byref(cnt), _stream_ptr(stream))
        self._check(st)
        return [(rep[i].team, rep[i].kernel_ms) for i in range(cnt.value)]

    def set_team(self, team: int):
        self._check(lib().phipm_set_team(self.h, int(team)))

    def team_for(self, kind: int, n: int) -> int:
        return lib().phipm_team_for(self.h, self.params.precision, int(kind), int(n))

    def last_batched_team(self) -> int:
        """CTAs per problem of the last batched call (phipm_batched_team)."""
        return int(lib().phipm_batched_team(self.h))

    def tune_save(self, path: str):
        self._check(lib().phipm_tune_save(self.h, str(path).encode()))

    def tune_load(self, path: str):
        self._check(lib().phipm_tune_load(self.h, str(path).encode()))

    def solve_host(self, t_end: float, A: HostOperator, b: list, tol: float = 1e-7, symm: int = -1, out=None,
                   stream=None, check: bool = True):
        """Same with host arrays (numpy float64, or pinned CPU torch tensors)."""
        p = len(b) - 1
        ptrs = [(x.data_ptr() if hasattr(x, "data_ptr") else x.ctypes.data) for x in b]
        if out is None:
            out = np.empty(A.n, dtype=np.float64)
        uptr = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
        bp = (c_void_p * (p + 1))(*ptrs)
        stats = StatsC()
        st = lib().phipm_solve_host(self.h, float(t_end), ctypes.byref(A.c), p, bp, float(tol), int(symm),
                                    c_void_p(uptr), ctypes.byref(stats), _stream_ptr(stream))
        if check:
            self._check(st)
        return out, stats.as_dict(), st

    # ---- attempt traces and the learned controller -------------------------------------
    def trace_enable(self, capacity: int):
        self._check(lib().phipm_trace_enable(self.h, int(capacity)))

    def trace_read(self, max_records: int = 1 << 20) -> list:
        """Attempt records of the last solve call, as dicts."""
        cnt = c_int64()
        lib().phipm_trace_read(self.h, None, 0, ctypes.byref(cnt))
        k = min(int(cnt.value), int(max_records))
        buf = (TraceRecordC * max(k, 1))()
        self._check(lib().phipm_trace_read(self.h, buf, k, ctypes.byref(cnt)))
        return [{f: getattr(buf[i], f) for f, _ in TraceRecordC._fields_} for i in range(k)]

    def set_controller_weights(self, blob):
        blob = np.ascontiguousarray(blob, dtype=np.float32)
        if blob.size == 0:
            self._check(lib().phipm_set_controller_weights(self.h, None, 0))
            return
        self._check(lib().phipm_set_controller_weights(
            self.h, blob.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), blob.size))

    def set_controller(self, kind: int):
        self.params.controller = int(kind)
        self._check(lib().phipm_set_params(self.h, ctypes.byref(self.params)))

    def mlp_forward(self, w, X, stream=None):
        import torch
        Y = torch.empty((X.shape[0], 2), dtype=torch.float32, device=X.device)
        self._check(lib().phipm_mlp_forward(self.h, w.data_ptr(), X.data_ptr(), X.shape[0], Y.data_ptr(),
                                            _stream_ptr(stream)))
        return Y

    def mlp_grad(self, w, X, T, stream=None):
        import torch
        g = torch.empty(MLP_PARAMS, dtype=torch.float32, device=X.device)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        self._check(lib().phipm_mlp_grad(self.h, w.data_ptr(), X.data_ptr(), T.data_ptr(), X.shape[0],
                                         g.data_ptr(), loss.data_ptr(), _stream_ptr(stream)))
        return g, float(loss.item())

    def mlp_train(self, w, m, v, X, T, iters: int, t0: int = 0, lr: float = 1e-3, stream=None):
        losses = (ctypes.c_float * max(iters, 1))()
        self._check(lib().phipm_mlp_train(self.h, w.data_ptr(), m.data_ptr(), v.data_ptr(), X.data_ptr(),
                                          T.data_ptr(), X.shape[0], int(iters), int(t0), float(lr), losses,
                                          _stream_ptr(stream)))
        return [float(losses[i]) for i in range(iters)]

    def batch(self, t_end: list, ops: list, bs: list, tol: list, symm: list, outs: list = None) -> "Batch":
        """Marshal a batch once; Batch.run() then repeats phipm_solve_batched on it (the
        library replays its captured launch graph while nothing baked into it changes)."""
        return Batch(self, t_end, ops, bs, tol, symm, outs)

    def solve_batched(self, t_end: list, ops: list, bs: list, tol: list, symm: list, outs: list = None,
                      stream=None, check: bool = True):
        """count independent problems in one persistent launch.  Returns (us, stats list, statuses)."""
        import torch
        cnt = len(ops)
        if outs is None:
            outs = [torch.empty(A.n, dtype=torch.float64, device="cuda") for A in ops]
        T = (c_double * cnt)(*[float(x) for x in t_end])
        Aa = (OperatorC * cnt)(*[A.c for A in ops])
        P = (c_int32 * cnt)(*[len(b) - 1 for b in bs])
        rows = [(c_void_p * len(b))(*[x.data_ptr() for x in b]) for b in bs]
        B = (ctypes.POINTER(c_void_p) * cnt)(*[ctypes.cast(r, ctypes.POINTER(c_void_p)) for r in rows])
        TOL = (c_double * cnt)(*[float(x) for x in tol])
        SY = (c_int32 * cnt)(*[int(x) for x in symm])
        U = (c_void_p * cnt)(*[u.data_ptr() for u in outs])
        ST = (StatsC * cnt)()
        PS = (c_int32 * cnt)()
        st = lib().phipm_solve_batched(self.h, cnt, T, Aa, P, B, TOL, SY, U, ST, PS, _stream_ptr(stream))
        if check:
            self._check(st)
        return outs, [s.as_dict() for s in ST], list(PS)


class Batch:
    """Prepared arguments of phipm_solve_batched (pointers of the given tensors, which
    the caller keeps alive and in place)."""

    def __init__(self, solver: Phipm, t_end, ops, bs, tol, symm, outs=None):
        import torch
        cnt = len(ops)
        self.solver, self.count, self.ops, self.bs = solver, cnt, ops, bs
        self.outs = outs if outs is not None else [torch.empty(A.n, dtype=torch.float64, device="cuda") for A in ops]
        self.T = (c_double * cnt)(*[float(x) for x in t_end])
        self.A = (OperatorC * cnt)(*[A.c for A in ops])
        self.P = (c_int32 * cnt)(*[len(b) - 1 for b in bs])
        self._rows = [(c_void_p * len(b))(*[x.data_ptr() for x in b]) for b in bs]
        self.B = (ctypes.POINTER(c_void_p) * cnt)(*[ctypes.cast(r, ctypes.POINTER(c_void_p)) for r in self._rows])
        self.TOL = (c_double * cnt)(*[float(x) for x in tol])
        self.SY = (c_int32 * cnt)(*[int(x) for x in symm])
        self.U = (c_void_p * cnt)(*[u.data_ptr() for u in self.outs])
        self.ST = (StatsC * cnt)()
        self.PS = (c_int32 * cnt)()

    def autotune(self, stream=None) -> list:
        """phipm_autotune_batched on this batch: time each cluster size K and keep the
        fastest for its batch class.  Returns [(K, kernel_ms), ...] in the order tried."""
        rep = (TuneEntryC * 8)()
        cnt = c_int32(0)
        st = lib().phipm_autotune_batched(self.solver.h, self.count, self.T, self.A, self.P, self.B, self.TOL, self.SY,
                                          self.U, rep, 8, ctypes.byref(cnt), _stream_ptr(stream))
        self.solver._check(st)
        return [(rep[i].team, rep[i].kernel_ms) for i in range(cnt.value)]

    def run(self, stream=None, check: bool = True) -> int:
        st = lib().phipm_solve_batched(self.solver.h, self.count, self.T, self.A, self.P, self.B, self.TOL, self.SY,
                                       self.U, self.ST, self.PS, _stream_ptr(stream))
        if check:
            self.solver._check(st)
        return st

    def stats(self) -> list:
        return [s.as_dict() for s in self.ST]

    def statuses(self) -> list:
        return list(self.PS)


def solve_noalloc(t_end: float, A: DeviceOperator, b: list, tol: float = 1e-7, symm: int = -1, out=None,
                  stream=None):
    """phipm_solve_noalloc: the FP64 solve with the library's static device scratch
    (no handle, no device allocation inside the call).  Returns (u, stats, status)."""
    import torch
    n = A.n
    p = len(b) - 1
    u = out if out is not None else torch.empty(n, dtype=torch.float64, device=b[0].device)
    bp = (c_void_p * (p + 1))(*[x.data_ptr() for x in b])
    stats = StatsC()
    st = lib().phipm_solve_noalloc(float(t_end), ctypes.byref(A.c), p, bp, float(tol), int(symm),
                                   c_void_p(u.data_ptr()), ctypes.byref(stats), _stream_ptr(stream))
    return u, stats.as_dict(), st
