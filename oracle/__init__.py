"""Python front end of the FP64 CPU oracle (``aar_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the benchmark's
CPU-baseline leg. The CUDA solver package never imports this module.

The oracle is plain sequential C in IEEE FP64 (``-O2 -ffp-contract=off``); see the header of
``aar_oracle.c`` for the equations each function follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aar_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, NOT_CONVERGED, ERR_INVALID_ARG, ERR_OOM, ERR_BREAKDOWN = 0, 1, -1, -2, -4


class _Op(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("radius", C.c_int32), ("periodic", C.c_int32), ("w", C.c_double * 7), ("h", C.c_double), ("shift", C.c_double),
        ("n", C.c_int32), ("nnz", C.c_int64), ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p),
        ("val", C.c_void_p),
    ]


class _ZOp(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("radius", C.c_int32),
        ("periodic", C.c_int32), ("pad", C.c_int32), ("w", C.c_double * 7), ("h", C.c_double),
        ("scale", C.c_double), ("q_re", C.c_double), ("q_im", C.c_double),
    ]


class _Info(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("anderson_steps", C.c_int32), ("status", C.c_int32),
                ("rel_residual", C.c_double)]


class _Trace(C.Structure):
    _fields_ = [("cap", C.c_int64), ("count", C.c_int64), ("k", C.c_void_p), ("r", C.c_void_p),
                ("c", C.c_void_p), ("rank", C.c_void_p), ("fmin", C.c_void_p)]


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to the source (gcc, FP64, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC",
                        "-shared", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            L.orc_op_size.restype = C.c_int64
            L.orc_op_size.argtypes = [C.POINTER(_Op)]
            L.orc_op_apply.restype = None
            L.orc_op_apply.argtypes = [C.POINTER(_Op), C.c_void_p, C.c_void_p]
            L.orc_op_apply_at.restype = C.c_double
            L.orc_op_apply_at.argtypes = [C.POINTER(_Op), C.c_void_p, C.c_int64]
            L.orc_op_diag.restype = None
            L.orc_op_diag.argtypes = [C.POINTER(_Op), C.c_void_p]
            L.orc_sym_eig.restype = C.c_int
            L.orc_sym_eig.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_pinv_solve.restype = C.c_int
            L.orc_pinv_solve.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int)]
            L.orc_aar_solve.restype = C.c_int
            L.orc_aar_solve.argtypes = [C.POINTER(_Op), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_double, C.c_double, C.c_int, C.c_int, C.c_double, C.c_int64,
                                        C.POINTER(_Info), C.POINTER(_Trace)]
            L.orc_rel_residual.restype = C.c_double
            L.orc_rel_residual.argtypes = [C.POINTER(_Op), C.c_void_p, C.c_void_p]
            L.orc_block_apply.restype = C.c_int
            L.orc_block_apply.argtypes = [C.POINTER(_Op), C.c_int, C.c_void_p, C.c_void_p]
            L.orc_aar_solve_block.restype = C.c_int
            L.orc_aar_solve_block.argtypes = [C.POINTER(_Op), C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                              C.c_double, C.c_double, C.c_int, C.c_int, C.c_double, C.c_int64,
                                              C.POINTER(_Info), C.POINTER(_Trace)]
            L.orz_op_size.restype = C.c_int64
            L.orz_op_size.argtypes = [C.POINTER(_ZOp)]
            L.orz_op_apply.restype = None
            L.orz_op_apply.argtypes = [C.POINTER(_ZOp), C.c_void_p, C.c_void_p]
            L.orz_op_apply_at.restype = None
            L.orz_op_apply_at.argtypes = [C.POINTER(_ZOp), C.c_void_p, C.c_int64, C.c_void_p]
            L.orz_op_diag.restype = None
            L.orz_op_diag.argtypes = [C.POINTER(_ZOp), C.c_void_p]
            L.orz_pinv_solve.restype = C.c_int
            L.orz_pinv_solve.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int)]
            L.orz_aar_solve.restype = C.c_int
            L.orz_aar_solve.argtypes = [C.POINTER(_ZOp), C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                        C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, C.c_double,
                                        C.c_int64, C.POINTER(_Info), C.POINTER(_Trace)]
            L.orz_block_apply.restype = C.c_int
            L.orz_block_apply.argtypes = [C.POINTER(_ZOp), C.c_int, C.c_void_p, C.c_void_p]
            L.orz_aar_solve_block.restype = C.c_int
            L.orz_aar_solve_block.argtypes = [C.POINTER(_ZOp), C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                              C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int,
                                              C.c_double, C.c_int64, C.POINTER(_Info), C.POINTER(_Trace)]
            L.orz_rel_residual.restype = C.c_double
            L.orz_rel_residual.argtypes = [C.POINTER(_ZOp), C.c_void_p, C.c_void_p]
            _lib = L
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class Operator:
    """Holds an ``orc_op`` plus references to the numpy arrays it points to."""

    def __init__(self, problem):
        op = _Op()
        self._keep = []
        if hasattr(problem, "radius"):
            op.kind = 0
            op.nx, op.ny, op.nz, op.radius = problem.nx, problem.ny, problem.nz, problem.radius
            for i, v in enumerate(np.asarray(problem.weights, dtype=np.float64)):
                op.w[i] = float(v)
            op.h, op.shift = float(problem.h), float(problem.shift)
            op.periodic = 1 if getattr(problem, "periodic", False) else 0
        else:
            op.kind = 1
            rp = np.ascontiguousarray(problem.row_ptr, dtype=np.int32)
            ci = np.ascontiguousarray(problem.col_idx, dtype=np.int32)
            vv = np.ascontiguousarray(problem.val, dtype=np.float64)
            self._keep += [rp, ci, vv]
            op.n, op.nnz = int(problem.n), int(rp[-1])
            op.row_ptr, op.col_idx, op.val = rp.ctypes.data, ci.ctypes.data, vv.ctypes.data
        self.op = op
        self.n = int(lib().orc_op_size(C.byref(op)))

    def apply(self, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty(self.n)
        lib().orc_op_apply(C.byref(self.op), _ptr(x), _ptr(y))
        return y

    def apply_at(self, x: np.ndarray, idx) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        return np.array([lib().orc_op_apply_at(C.byref(self.op), _ptr(x), int(i)) for i in idx])

    def diag(self) -> np.ndarray:
        d = np.empty(self.n)
        lib().orc_op_diag(C.byref(self.op), _ptr(d))
        return d

    def rel_residual(self, b: np.ndarray, x: np.ndarray) -> float:
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.ascontiguousarray(x, dtype=np.float64)
        return float(lib().orc_rel_residual(C.byref(self.op), _ptr(b), _ptr(x)))

    def block_apply(self, r: np.ndarray, block: int) -> np.ndarray:
        """f = M^{-1} r for the block-Jacobi preconditioner with block x block x block boxes."""
        r = np.ascontiguousarray(r, dtype=np.float64)
        f = np.empty(self.n)
        st = lib().orc_block_apply(C.byref(self.op), int(block), _ptr(r), _ptr(f))
        if st != OK:
            raise ValueError(f"oracle block apply failed (status {st})")
        return f


def sym_eig(S: np.ndarray):
    S = np.ascontiguousarray(S, dtype=np.float64)
    c = S.shape[0]
    lam = np.empty(c)
    V = np.empty((c, c))
    sweeps = lib().orc_sym_eig(c, _ptr(S), _ptr(lam), _ptr(V))
    return lam, V, sweeps


def pinv_solve(G: np.ndarray, g: np.ndarray):
    G = np.ascontiguousarray(G, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    c = G.shape[0]
    gamma = np.zeros(max(c, 1))
    rank = C.c_int(0)
    lib().orc_pinv_solve(c, _ptr(G), _ptr(g), _ptr(gamma), C.byref(rank))
    return gamma[:c], rank.value


class Result:
    def __init__(self, x, info: _Info, trace: dict | None):
        self.x = x
        self.iterations = int(info.iterations)
        self.anderson_steps = int(info.anderson_steps)
        self.status = int(info.status)
        self.rel_residual = float(info.rel_residual)
        self.trace = trace


def solve(problem, omega=0.6, beta=0.6, m=9, p=8, tol=1e-8, max_iter=100000, x0=None, dinv=None,
          trace_cap: int = 0, op: Operator | None = None, block: int = 0) -> Result:
    """Run the FP64 oracle AAR solve (Eq. 2-6) on a workloads.StencilProblem / CsrProblem;
    block >= 2 takes the block-Jacobi preconditioner (block^3 boxes) in place of Jacobi."""
    op = op or Operator(problem)
    b = np.ascontiguousarray(problem.b, dtype=np.float64)
    x = np.empty(op.n)
    info = _Info()
    tr = None
    arrs = None
    if trace_cap:
        arrs = dict(k=np.zeros(trace_cap, np.int64), r=np.zeros(trace_cap), c=np.zeros(trace_cap, np.int32),
                    rank=np.zeros(trace_cap, np.int32), fmin=np.zeros(trace_cap))
        tr = _Trace(trace_cap, 0, arrs["k"].ctypes.data, arrs["r"].ctypes.data, arrs["c"].ctypes.data,
                    arrs["rank"].ctypes.data, arrs["fmin"].ctypes.data)
    x0a = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
    da = None if dinv is None else np.ascontiguousarray(dinv, dtype=np.float64)
    if block and block > 1:
        if dinv is not None:
            raise ValueError("block Jacobi takes no dinv")
        st = lib().orc_aar_solve_block(C.byref(op.op), int(block), _ptr(b), _ptr(x0a), _ptr(x), float(omega),
                                       float(beta), int(m), int(p), float(tol), int(max_iter), C.byref(info),
                                       C.byref(tr) if tr is not None else None)
    else:
        st = lib().orc_aar_solve(C.byref(op.op), _ptr(da), _ptr(b), _ptr(x0a), _ptr(x), float(omega), float(beta),
                                 int(m), int(p), float(tol), int(max_iter), C.byref(info),
                                 C.byref(tr) if tr is not None else None)
    if st == ERR_INVALID_ARG or st == ERR_OOM:
        raise ValueError(f"oracle rejected the arguments (status {st})")
    trace = None
    if tr is not None:
        cnt = int(tr.count)
        trace = {key: v[:cnt].copy() for key, v in arrs.items()}
    return Result(x, info, trace)


# ------------------------------------------------------------------ complex-valued systems

class ZOperator:
    """The complex stencil operator of Eq. 7 (``orz_op``) for a workloads.ComplexStencilProblem."""

    def __init__(self, problem):
        op = _ZOp()
        op.nx, op.ny, op.nz, op.radius = problem.nx, problem.ny, problem.nz, problem.radius
        for i, v in enumerate(np.asarray(problem.weights, dtype=np.float64)):
            op.w[i] = float(v)
        op.h, op.scale = float(problem.h), float(problem.scale)
        q = complex(problem.q)
        op.q_re, op.q_im = q.real, q.imag
        op.periodic = 1 if problem.periodic else 0
        self.op = op
        self.n = int(lib().orz_op_size(C.byref(op)))

    def apply(self, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.complex128)
        y = np.empty(self.n, dtype=np.complex128)
        lib().orz_op_apply(C.byref(self.op), _ptr(x), _ptr(y))
        return y

    def apply_at(self, x: np.ndarray, idx) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.complex128)
        out = np.empty(len(idx), dtype=np.complex128)
        for j, i in enumerate(idx):
            lib().orz_op_apply_at(C.byref(self.op), _ptr(x), int(i), _ptr(out[j:j + 1]))
        return out

    def diag(self) -> complex:
        v = np.empty(1, dtype=np.complex128)
        lib().orz_op_diag(C.byref(self.op), _ptr(v))
        return complex(v[0])

    def rel_residual(self, b: np.ndarray, x: np.ndarray) -> float:
        b = np.ascontiguousarray(b, dtype=np.complex128)
        x = np.ascontiguousarray(x, dtype=np.complex128)
        return float(lib().orz_rel_residual(C.byref(self.op), _ptr(b), _ptr(x)))

    def block_apply(self, r: np.ndarray, block: int) -> np.ndarray:
        """f = M^{-1} r for the block-Jacobi M with block^3 boxes (orz_block_apply)."""
        r = np.ascontiguousarray(r, dtype=np.complex128)
        f = np.empty(self.n, dtype=np.complex128)
        st = lib().orz_block_apply(C.byref(self.op), int(block), _ptr(r), _ptr(f))
        if st != OK:
            raise ValueError(f"orz_block_apply failed (status {st})")
        return f


def zpinv_solve(G: np.ndarray, g: np.ndarray):
    """gamma = pinv(G) g for a Hermitian positive semidefinite complex G (orz_pinv_solve)."""
    G = np.ascontiguousarray(G, dtype=np.complex128)
    g = np.ascontiguousarray(g, dtype=np.complex128)
    c = G.shape[0]
    gamma = np.zeros(max(c, 1), dtype=np.complex128)
    rank = C.c_int(0)
    lib().orz_pinv_solve(c, _ptr(G), _ptr(g), _ptr(gamma), C.byref(rank))
    return gamma[:c], rank.value


def zsolve(problem, omega=0.6, beta=0.6, m=9, p=8, tol=1e-8, max_iter=100000, x0=None, trace_cap: int = 0,
           op: ZOperator | None = None, block: int = 0) -> Result:
    """Run the FP64 complex oracle AAR solve (Eq. 1-6 over C) on a workloads.ComplexStencilProblem;
    omega and beta may be complex. block >= 2: block Jacobi with block^3 boxes in place of Jacobi."""
    op = op or ZOperator(problem)
    b = np.ascontiguousarray(problem.b, dtype=np.complex128)
    x = np.empty(op.n, dtype=np.complex128)
    info = _Info()
    tr = None
    arrs = None
    if trace_cap:
        arrs = dict(k=np.zeros(trace_cap, np.int64), r=np.zeros(trace_cap), c=np.zeros(trace_cap, np.int32),
                    rank=np.zeros(trace_cap, np.int32), fmin=np.zeros(trace_cap))
        tr = _Trace(trace_cap, 0, arrs["k"].ctypes.data, arrs["r"].ctypes.data, arrs["c"].ctypes.data,
                    arrs["rank"].ctypes.data, arrs["fmin"].ctypes.data)
    x0a = None if x0 is None else np.ascontiguousarray(x0, dtype=np.complex128)
    om, be = complex(omega), complex(beta)
    if block >= 2:
        st = lib().orz_aar_solve_block(C.byref(op.op), int(block), _ptr(b), _ptr(x0a), _ptr(x), om.real, om.imag,
                                       be.real, be.imag, int(m), int(p), float(tol), int(max_iter), C.byref(info),
                                       C.byref(tr) if tr is not None else None)
    else:
        st = lib().orz_aar_solve(C.byref(op.op), _ptr(b), _ptr(x0a), _ptr(x), om.real, om.imag, be.real, be.imag,
                                 int(m), int(p), float(tol), int(max_iter), C.byref(info),
                                 C.byref(tr) if tr is not None else None)
    if st == ERR_INVALID_ARG or st == ERR_OOM:
        raise ValueError(f"oracle rejected the arguments (status {st})")
    trace = None
    if tr is not None:
        cnt = int(tr.count)
        trace = {key: v[:cnt].copy() for key, v in arrs.items()}
    return Result(x, info, trace)
