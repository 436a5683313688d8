"""Python binding of ``libaar.so`` (the C ABI in ``include/aar.h``): argument marshalling only.

Every step of a solve runs in the library's CUDA kernels; this module only converts torch
tensors / numpy arrays to pointers and structs. Importing it loads ``libaar.so`` and raises if
the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libaar.so")

OK, NOT_CONVERGED, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_BREAKDOWN, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_COMM = (
    0, 1, -1, -2, -3, -4, -5, -6, -7)
FP64, MIXED = 0, 1
MAX_M, MAX_RADIUS = 16, 6
FLAG_RESTART_HISTORY = 1

EXPORTS = (
    "aar_default_params", "aar_create_stencil", "aar_create_csr", "aar_solve", "aar_apply",
    "aar_rel_residual", "aar_destroy", "aar_status_string", "aar_batch_create", "aar_batch_solve",
    "aar_batch_destroy", "aar_profile_kernel", "aar_rel_residual_noalloc", "aar_tune_stencil",
    "aar_server_create", "aar_server_submit", "aar_server_run", "aar_server_poll", "aar_server_destroy",
    "aar_zdefault_params", "aar_zcreate_stencil", "aar_zsolve", "aar_zapply", "aar_zrel_residual",
    "aar_zprofile_kernel", "aar_zdestroy", "aar_measure_fp64_rate", "aar_dd_create", "aar_dd_solve",
    "aar_dd_destroy",
)
K_SWEEP, K_SWEEP_ANDERSON, K_GRAM, K_UPDATE, K_RESID64, K_FINALIZE, K_BLOCK = 0, 1, 2, 3, 4, 5, 6


class StencilDesc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("radius", C.c_int32),
                ("w", C.c_double * (MAX_RADIUS + 1)), ("h", C.c_double), ("shift", C.c_double),
                ("tile_variant", C.c_int32), ("tile_zc", C.c_int32), ("periodic", C.c_int32),
                ("block", C.c_int32)]


class ZStencilDesc(C.Structure):
    """aar_zstencil_desc (include/aar_complex.h): the complex operator of Eq. 7."""
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("radius", C.c_int32),
                ("w", C.c_double * (MAX_RADIUS + 1)), ("h", C.c_double), ("scale", C.c_double),
                ("q_re", C.c_double), ("q_im", C.c_double), ("periodic", C.c_int32), ("block", C.c_int32)]


class ZParams(C.Structure):
    _fields_ = [("omega_re", C.c_double), ("omega_im", C.c_double), ("beta_re", C.c_double),
                ("beta_im", C.c_double), ("m", C.c_int32), ("p", C.c_int32), ("tol", C.c_double),
                ("max_iter", C.c_int64), ("inner_tol", C.c_double), ("max_refine", C.c_int32),
                ("reserved", C.c_int32)]


class CsrDesc(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64), ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p),
                ("val", C.c_void_p)]


class Params(C.Structure):
    _fields_ = [("omega", C.c_double), ("beta", C.c_double), ("m", C.c_int32), ("p", C.c_int32),
                ("tol", C.c_double), ("max_iter", C.c_int64), ("inner_tol", C.c_double),
                ("max_refine", C.c_int32), ("flags", C.c_int32), ("step_limit", C.c_int64)]


class Info(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("anderson_steps", C.c_int32), ("refinements", C.c_int32),
                ("rel_residual", C.c_double), ("status", C.c_int32), ("last_rank", C.c_int32),
                ("ticks", C.c_int64), ("launches", C.c_int64), ("eigen_steps", C.c_int32),
                ("reserved", C.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


# aar_comm (include/aar_dd.h): the halo-exchange and allreduce callbacks of a domain-decomposed solve
HaloFn = C.CFUNCTYPE(C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p)
AllreduceFn = C.CFUNCTYPE(C.c_int32, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p)


class Comm(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("halo", HaloFn), ("allreduce", AllreduceFn)]


class AARError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} ({status})")
        self.status = status


_lib = None


def lib() -> C.CDLL:
    """Load libaar.so (raises OSError when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"{LIB_PATH} is missing: build it with paper_1606_08740_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.aar_default_params.argtypes = [C.POINTER(Params)]
        L.aar_create_stencil.argtypes = [C.POINTER(StencilDesc), vp, C.c_int32, vp, C.POINTER(vp)]
        L.aar_create_csr.argtypes = [C.POINTER(CsrDesc), vp, C.c_int32, vp, C.POINTER(vp)]
        L.aar_solve.argtypes = [vp, vp, vp, vp, C.POINTER(Params), C.POINTER(Info)]
        L.aar_apply.argtypes = [vp, vp, vp]
        L.aar_rel_residual.argtypes = [vp, vp, vp, C.POINTER(C.c_double)]
        L.aar_destroy.argtypes = [vp]
        L.aar_status_string.argtypes = [C.c_int]
        L.aar_status_string.restype = C.c_char_p
        L.aar_batch_create.argtypes = [C.POINTER(StencilDesc), C.c_int32, C.c_int32, vp, C.POINTER(vp)]
        L.aar_batch_solve.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(Params), C.c_int32,
                                      C.POINTER(Info)]
        L.aar_batch_destroy.argtypes = [vp]
        L.aar_profile_kernel.argtypes = [vp, C.c_int32, C.c_int32, C.POINTER(C.c_float)]
        L.aar_rel_residual_noalloc.argtypes = [vp, vp, vp, C.POINTER(C.c_double)]
        L.aar_server_create.argtypes = [C.c_int32, C.c_int32, C.c_int64, C.c_int32, vp, C.POINTER(vp)]
        L.aar_server_submit.argtypes = [vp, C.POINTER(StencilDesc), vp, vp, C.POINTER(Params), C.POINTER(C.c_int64)]
        L.aar_server_run.argtypes = [vp, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int64)]
        L.aar_server_poll.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(Info), C.c_int32, C.POINTER(C.c_int32)]
        L.aar_server_destroy.argtypes = [vp]
        L.aar_tune_stencil.argtypes = [C.POINTER(StencilDesc), C.c_int32, C.c_int32, vp, C.POINTER(C.c_int32),
                                       C.POINTER(C.c_int32), C.POINTER(C.c_float)]
        L.aar_zdefault_params.argtypes = [C.POINTER(ZParams)]
        L.aar_zcreate_stencil.argtypes = [C.POINTER(ZStencilDesc), C.c_int32, vp, C.POINTER(vp)]
        L.aar_zsolve.argtypes = [vp, vp, vp, vp, C.POINTER(ZParams), C.POINTER(Info)]
        L.aar_zapply.argtypes = [vp, vp, vp]
        L.aar_zrel_residual.argtypes = [vp, vp, vp, C.POINTER(C.c_double)]
        L.aar_zprofile_kernel.argtypes = [vp, C.c_int32, C.c_int32, C.POINTER(C.c_float)]
        L.aar_zdestroy.argtypes = [vp]
        L.aar_measure_fp64_rate.argtypes = [vp, C.c_int32, C.POINTER(C.c_double)]
        L.aar_dd_create.argtypes = [C.POINTER(StencilDesc), C.c_int32, C.c_int32, vp, C.POINTER(vp)]
        L.aar_dd_solve.argtypes = [vp, vp, vp, C.POINTER(Params), C.POINTER(Comm), C.POINTER(Info)]
        L.aar_dd_destroy.argtypes = [vp]
        for name in EXPORTS:
            if name != "aar_status_string":
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().aar_status_string(int(status)).decode()


def params(omega=0.6, beta=0.6, m=9, p=8, tol=1e-8, max_iter=100000, inner_tol=0.1, max_refine=30,
           restart_history=False, step_limit=0) -> Params:
    """Solver parameters; defaults are the paper's {omega, beta, m, p} = {0.6, 0.6, 9, 8}.
    restart_history: mixed form only, start every inner solve from an empty Anderson history.
    step_limit: watchdog on the device loop in device steps (0 = derived from max_iter)."""
    return Params(float(omega), float(beta), int(m), int(p), float(tol), int(max_iter), float(inner_tol),
                  int(max_refine), FLAG_RESTART_HISTORY if restart_history else 0, int(step_limit))


def stencil_desc(nx, ny, nz, radius, weights, h=1.0, shift=0.0, periodic=False, block=0) -> StencilDesc:
    """periodic: every axis wraps (else zero Dirichlet ghosts). block: 0 = Jacobi, 2 = block
    Jacobi with 2 x 2 x 2 boxes."""
    d = StencilDesc()
    d.nx, d.ny, d.nz, d.radius = int(nx), int(ny), int(nz), int(radius)
    w = np.asarray(weights, dtype=np.float64)
    for i in range(min(len(w), MAX_RADIUS + 1)):
        d.w[i] = float(w[i])
    d.h, d.shift = float(h), float(shift)
    d.periodic = 1 if periodic else 0
    d.block = int(block)
    return d


def tune_stencil(desc: StencilDesc, precision: int = MIXED, m: int = 7, stream=None):
    """(tile_variant, tile_zc, ms per sweep) of the fastest tiling for this grid shape."""
    v, z, ms = C.c_int32(0), C.c_int32(0), C.c_float(0.0)
    _check(lib().aar_tune_stencil(C.byref(desc), int(precision), int(m), _stream_ptr(stream), C.byref(v), C.byref(z),
                                  C.byref(ms)), "aar_tune_stencil", allow=(OK,))
    return int(v.value), int(z.value), float(ms.value)


def measure_fp64_rate(op: int = 0, stream=None) -> float:
    """Thread-level FP64 instructions/s of the current device: op 0 = DFMA, 1 = DADD
    (see aar_measure_fp64_rate)."""
    out = C.c_double(0.0)
    _check(lib().aar_measure_fp64_rate(_stream_ptr(stream), int(op), C.byref(out)), "aar_measure_fp64_rate",
           allow=(OK,))
    return float(out.value)


def desc_of(problem, block: int = 0) -> StencilDesc:
    """StencilDesc from any object with nx, ny, nz, radius, weights, h, shift (and optionally
    periodic) attributes; block = 2 selects block Jacobi with 2 x 2 x 2 boxes."""
    return stencil_desc(problem.nx, problem.ny, problem.nz, problem.radius, problem.weights, problem.h, problem.shift,
                        getattr(problem, "periodic", False), block)


def _ptr(a):
    """Device pointer of a torch tensor or host pointer of a numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported buffer type {type(a)}")


def _stream_ptr(stream):
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


def _check(st: int, what: str, allow=(OK, NOT_CONVERGED)) -> int:
    if st not in allow:
        raise AARError(st, what)
    return st


@dataclass
class SolveResult:
    status: int
    iterations: int
    anderson_steps: int
    refinements: int
    rel_residual: float
    last_rank: int
    ticks: int = 0
    launches: int = 0
    eigen_steps: int = 0

    @property
    def converged(self) -> bool:
        return self.status == OK


def _result(info: Info, st: int) -> SolveResult:
    return SolveResult(int(st), int(info.iterations), int(info.anderson_steps), int(info.refinements),
                       float(info.rel_residual), int(info.last_rank), int(info.ticks), int(info.launches),
                       int(info.eigen_steps))


class Solver:
    """A solver handle for one operator (stencil or CSR)."""

    def __init__(self, handle, n: int, keep=()):
        self._h = C.c_void_p(handle)
        self.n = int(n)
        self._keep = list(keep)

    @classmethod
    def stencil(cls, desc: StencilDesc, precision: int = FP64, stream=None, dinv=None) -> "Solver":
        h = C.c_void_p()
        _check(lib().aar_create_stencil(C.byref(desc), _ptr(dinv), int(precision), _stream_ptr(stream), C.byref(h)),
               "aar_create_stencil", allow=(OK,))
        return cls(h.value, desc.nx * desc.ny * desc.nz, keep=[dinv])

    @classmethod
    def csr(cls, row_ptr, col_idx, val, precision: int = FP64, stream=None, dinv=None) -> "Solver":
        d = CsrDesc(int(row_ptr.numel() - 1), int(val.numel()), _ptr(row_ptr), _ptr(col_idx), _ptr(val))
        h = C.c_void_p()
        _check(lib().aar_create_csr(C.byref(d), _ptr(dinv), int(precision), _stream_ptr(stream), C.byref(h)),
               "aar_create_csr", allow=(OK,))
        return cls(h.value, d.n, keep=[row_ptr, col_idx, val, dinv])

    def solve(self, b, x, x0=None, prm: Params | None = None, raise_on_error: bool = True) -> SolveResult:
        """Solve A x = b into ``x`` (torch CUDA float64 tensors, or numpy float64 host arrays)."""
        prm = prm or params()
        info = Info()
        st = lib().aar_solve(self._h, _ptr(b), _ptr(x0), _ptr(x), C.byref(prm), C.byref(info))
        if raise_on_error:
            _check(st, "aar_solve")
        return _result(info, st)

    def apply(self, x, y) -> None:
        _check(lib().aar_apply(self._h, _ptr(x), _ptr(y)), "aar_apply", allow=(OK,))

    def rel_residual(self, b, x) -> float:
        out = C.c_double(math.nan)
        _check(lib().aar_rel_residual(self._h, _ptr(b), _ptr(x), C.byref(out)), "aar_rel_residual", allow=(OK,))
        return float(out.value)

    def rel_residual_noalloc(self, b, x) -> float:
        """||b - A x|| / ||b|| without any device allocation (see aar_rel_residual_noalloc)."""
        out = C.c_double(math.nan)
        _check(lib().aar_rel_residual_noalloc(self._h, _ptr(b), _ptr(x), C.byref(out)), "aar_rel_residual_noalloc",
               allow=(OK,))
        return float(out.value)

    def profile_kernel(self, kernel: int, launches: int = 20) -> float:
        """Mean ms per launch of one solve-loop kernel (see aar_profile_kernel)."""
        ms = C.c_float(0.0)
        _check(lib().aar_profile_kernel(self._h, int(kernel), int(launches), C.byref(ms)), "aar_profile_kernel",
               allow=(OK,))
        return float(ms.value)

    def close(self) -> None:
        if self._h:
            lib().aar_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class DDSolver:
    """This rank's slab [z_lo, z_hi) of a domain-decomposed stencil solve (include/aar_dd.h).

    ``comm`` passed to solve() is any object with two methods taking raw pointers, called from
    inside the library: ``halo(send_lo, send_hi, recv_lo, recv_hi, count, stream)`` and
    ``allreduce(buf, count, stream)`` (device pointers as ints, the stream as an int); see
    ``paper_1606_08740_gb300.dd`` for torch.distributed and in-process implementations. An
    exception raised in a callback makes it return failure, and the solve AAR_ERR_COMM."""

    def __init__(self, desc: StencilDesc, z_lo: int, z_hi: int, stream=None):
        h = C.c_void_p()
        _check(lib().aar_dd_create(C.byref(desc), int(z_lo), int(z_hi), _stream_ptr(stream), C.byref(h)),
               "aar_dd_create", allow=(OK,))
        self._h = h
        self.z_lo, self.z_hi = int(z_lo), int(z_hi)
        self.n = desc.nx * desc.ny * (self.z_hi - self.z_lo)
        self.errors = []  # exceptions raised inside the callbacks of the last solve

    def solve(self, b, x, comm, prm: Params | None = None, raise_on_error: bool = True) -> SolveResult:
        self.errors = []

        def halo(_ctx, slo, shi, rlo, rhi, count, stream):
            try:
                comm.halo(slo or 0, shi or 0, rlo or 0, rhi or 0, int(count), stream or 0)
                return 0
            except Exception as e:  # noqa: BLE001 -- reported through AAR_ERR_COMM
                self.errors.append(e)
                return 1

        def allreduce(_ctx, buf, count, stream):
            try:
                comm.allreduce(buf or 0, int(count), stream or 0)
                return 0
            except Exception as e:  # noqa: BLE001
                self.errors.append(e)
                return 1

        cm = Comm(None, HaloFn(halo), AllreduceFn(allreduce))
        info = Info()
        st = lib().aar_dd_solve(self._h, _ptr(b), _ptr(x), C.byref(prm or params()), C.byref(cm), C.byref(info))
        if raise_on_error:
            _check(st, "aar_dd_solve")
        return _result(info, st)

    def close(self) -> None:
        if self._h:
            lib().aar_dd_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def zparams(omega=0.6, beta=0.6, m=9, p=8, tol=1e-6, max_iter=100000, inner_tol=1e-3, max_refine=30) -> ZParams:
    """Complex-solve parameters (omega, beta may be complex); defaults {0.6, 0.6, 9, 8}, tol 1e-6;
    inner_tol and max_refine apply to the mixed form."""
    om, be = complex(omega), complex(beta)
    return ZParams(om.real, om.imag, be.real, be.imag, int(m), int(p), float(tol), int(max_iter), float(inner_tol),
                   int(max_refine), 0)


def zstencil_desc(nx, ny, nz, radius, weights, h=1.0, scale=1.0, q=0.0, periodic=True, block=0) -> ZStencilDesc:
    """A = scale * (-lap_h) + q I with complex q (Eq. 7: scale = 1/(4 pi), q = Q). block: 0 =
    Jacobi, 2 = block Jacobi with 2 x 2 x 2 boxes."""
    d = ZStencilDesc()
    d.nx, d.ny, d.nz, d.radius = int(nx), int(ny), int(nz), int(radius)
    w = np.asarray(weights, dtype=np.float64)
    for i in range(min(len(w), MAX_RADIUS + 1)):
        d.w[i] = float(w[i])
    d.h, d.scale = float(h), float(scale)
    qq = complex(q)
    d.q_re, d.q_im = qq.real, qq.imag
    d.periodic = 1 if periodic else 0
    d.block = int(block)
    return d


def zdesc_of(problem, block: int = 0) -> ZStencilDesc:
    """ZStencilDesc from an object with nx, ny, nz, radius, weights, h, scale, q, periodic; block = 2
    selects block Jacobi with 2 x 2 x 2 boxes."""
    return zstencil_desc(problem.nx, problem.ny, problem.nz, problem.radius, problem.weights, problem.h,
                         problem.scale, problem.q, problem.periodic, block)


class ZSolver:
    """A complex-valued solver handle (include/aar_complex.h). Vectors are complex128 (torch
    CUDA tensors or numpy host arrays), i.e. interleaved FP64 pairs."""

    def __init__(self, desc: ZStencilDesc, precision: int = FP64, stream=None):
        h = C.c_void_p()
        _check(lib().aar_zcreate_stencil(C.byref(desc), int(precision), _stream_ptr(stream), C.byref(h)),
               "aar_zcreate_stencil", allow=(OK,))
        self._h = h
        self.n = desc.nx * desc.ny * desc.nz

    def solve(self, b, x, x0=None, prm: ZParams | None = None, raise_on_error: bool = True) -> SolveResult:
        prm = prm or zparams()
        info = Info()
        st = lib().aar_zsolve(self._h, _ptr(b), _ptr(x0), _ptr(x), C.byref(prm), C.byref(info))
        if raise_on_error:
            _check(st, "aar_zsolve")
        return _result(info, st)

    def apply(self, x, y) -> None:
        _check(lib().aar_zapply(self._h, _ptr(x), _ptr(y)), "aar_zapply", allow=(OK,))

    def rel_residual(self, b, x) -> float:
        out = C.c_double(math.nan)
        _check(lib().aar_zrel_residual(self._h, _ptr(b), _ptr(x), C.byref(out)), "aar_zrel_residual", allow=(OK,))
        return float(out.value)

    def profile_kernel(self, kernel: int, launches: int = 20) -> float:
        ms = C.c_float(0.0)
        _check(lib().aar_zprofile_kernel(self._h, int(kernel), int(launches), C.byref(ms)), "aar_zprofile_kernel",
               allow=(OK,))
        return float(ms.value)

    def close(self) -> None:
        if self._h:
            lib().aar_zdestroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Many independent stencil systems solved together (shared radius and precision)."""

    def __init__(self, descs, precision: int = FP64, stream=None):
        arr = (StencilDesc * len(descs))(*descs)
        self.nsys = len(descs)
        self.sizes = [d.nx * d.ny * d.nz for d in descs]
        h = C.c_void_p()
        _check(lib().aar_batch_create(arr, self.nsys, int(precision), _stream_ptr(stream), C.byref(h)),
               "aar_batch_create", allow=(OK,))
        self._h = h

    def solve(self, bs, xs, prm: Params | list | None = None, raise_on_error: bool = True):
        if len(bs) != self.nsys or len(xs) != self.nsys:
            raise ValueError("one b and one x per system")
        bp = (C.c_void_p * self.nsys)(*[_ptr(b) for b in bs])
        xp = (C.c_void_p * self.nsys)(*[_ptr(x) for x in xs])
        if isinstance(prm, list):
            parr = (Params * self.nsys)(*prm)
            stride = 1
        else:
            parr = (Params * 1)(prm or params())
            stride = 0
        infos = (Info * self.nsys)()
        st = lib().aar_batch_solve(self._h, bp, xp, parr, stride, infos)
        if raise_on_error:
            _check(st, "aar_batch_solve")
        return [_result(infos[i], infos[i].status) for i in range(self.nsys)]

    def close(self) -> None:
        if self._h:
            lib().aar_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching solve server (see aar_server_* in include/aar.h).

    Host buffers passed to submit() are kept referenced here until their request completes."""

    def __init__(self, radius: int, precision: int = MIXED, budget_bytes: int = 32 << 30, max_active: int = 256,
                 stream=None):
        h = C.c_void_p()
        _check(lib().aar_server_create(int(radius), int(precision), int(budget_bytes), int(max_active),
                                       _stream_ptr(stream), C.byref(h)), "aar_server_create", allow=(OK,))
        self._h = h
        self._keep = {}

    def submit(self, desc: StencilDesc, b: np.ndarray, x: np.ndarray, prm: Params | None = None) -> int:
        rid = C.c_int64(0)
        _check(lib().aar_server_submit(self._h, C.byref(desc), _ptr(b), _ptr(x), C.byref(prm or params()),
                                       C.byref(rid)), "aar_server_submit", allow=(OK,))
        self._keep[rid.value] = (b, x)
        return int(rid.value)

    def run(self, ticks: int = 8):
        a, w, u = C.c_int32(0), C.c_int32(0), C.c_int64(0)
        _check(lib().aar_server_run(self._h, int(ticks), C.byref(a), C.byref(w), C.byref(u)), "aar_server_run",
               allow=(OK,))
        return int(a.value), int(w.value), int(u.value)

    def poll(self, cap: int = 4096):
        ids = (C.c_int64 * cap)()
        infos = (Info * cap)()
        n = C.c_int32(0)
        _check(lib().aar_server_poll(self._h, ids, infos, int(cap), C.byref(n)), "aar_server_poll", allow=(OK,))
        out = []
        for i in range(n.value):
            self._keep.pop(int(ids[i]), None)
            out.append((int(ids[i]), _result(infos[i], infos[i].status)))
        return out

    def close(self) -> None:
        if self._h:
            lib().aar_server_destroy(self._h)
            self._h = C.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
