"""CPU-side checks of the C ABI library: it builds, loads, exports every declared symbol, and
rejects invalid arguments before touching the GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1606_08740_gb300 import build

    build.build()
    from paper_1606_08740_gb300 import aar

    return aar.lib()


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(aar_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 11
    for n in names:
        assert hasattr(lib, n), n


def test_binding_lists_the_declared_symbols(lib):
    from paper_1606_08740_gb300 import aar

    assert set(declared_functions()) == set(aar.EXPORTS)


def test_defaults_and_status_strings(lib):
    from paper_1606_08740_gb300 import aar

    p = aar.Params()
    assert lib.aar_default_params(C.byref(p)) == 0
    assert (p.omega, p.beta, p.m, p.p) == (0.6, 0.6, 9, 8)  # Sec. 2 defaults
    assert (p.inner_tol, p.max_refine, p.flags, p.step_limit) == (0.1, 30, 0, 0)
    assert C.sizeof(aar.Params) == 64  # the C struct: 9 fields of aar_params plus the int64 step_limit
    assert aar.params().flags == 0 and aar.params(restart_history=True).flags == aar.FLAG_RESTART_HISTORY
    for s in [0, 1, -1, -2, -3, -4, -5, -6]:
        assert aar.status_string(s)
    assert lib.aar_default_params(None) == aar.ERR_INVALID_ARG
    # the FP64 rate probe validates its arguments before touching a device
    out = C.c_double(1.0)
    assert lib.aar_measure_fp64_rate(None, 2, C.byref(out)) == aar.ERR_INVALID_ARG
    assert lib.aar_measure_fp64_rate(None, 0, None) == aar.ERR_INVALID_ARG


def test_invalid_descriptors_rejected_without_gpu(lib):
    from paper_1606_08740_gb300 import aar

    h = C.c_void_p()
    for bad in [dict(nx=0), dict(radius=0), dict(radius=7), dict(h=0.0), dict(shift=-1.0)]:
        kw = dict(nx=8, ny=8, nz=8, radius=1, weights=[-2.0, 1.0], h=1.0, shift=0.0)
        kw.update(bad)
        d = aar.stencil_desc(**kw)
        assert lib.aar_create_stencil(C.byref(d), None, aar.FP64, None, C.byref(h)) == aar.ERR_INVALID_ARG
    d = aar.stencil_desc(8, 8, 8, 1, [-2.0, 1.0])
    assert lib.aar_create_stencil(C.byref(d), None, 7, None, C.byref(h)) == aar.ERR_INVALID_ARG
    d = aar.stencil_desc(8, 8, 8, 1, [-2.0, 1.0], periodic=True)
    d.periodic = 2  # only 0 (zero Dirichlet ghosts) and 1 (periodic) are boundary kinds
    assert lib.aar_create_stencil(C.byref(d), None, aar.FP64, None, C.byref(h)) == aar.ERR_INVALID_ARG
    # a positive second-derivative centre weight gives a non-positive diagonal
    d = aar.stencil_desc(8, 8, 8, 1, [2.0, 1.0])
    assert lib.aar_create_stencil(C.byref(d), None, aar.FP64, None, C.byref(h)) == aar.ERR_INVALID_ARG
    assert lib.aar_solve(None, None, None, None, None, None) == aar.ERR_INVALID_ARG
    assert lib.aar_destroy(None) == aar.ERR_INVALID_ARG


def test_complex_defaults_and_invalid_descriptors_without_gpu(lib):
    from paper_1606_08740_gb300 import aar

    p = aar.ZParams()
    assert lib.aar_zdefault_params(C.byref(p)) == 0
    assert (p.omega_re, p.omega_im, p.beta_re, p.beta_im, p.m, p.p) == (0.6, 0.0, 0.6, 0.0, 9, 8)
    assert p.tol == 1e-6  # the tolerance of the paper's Helmholtz runs (Sec. 3.2)
    assert (p.inner_tol, p.max_refine) == (1e-3, 30)
    assert lib.aar_zdefault_params(None) == aar.ERR_INVALID_ARG
    h = C.c_void_p()
    good = dict(nx=8, ny=8, nz=8, radius=3, weights=[-49 / 18, 1.5, -0.15, 1 / 90], h=0.5, scale=0.0796,
                q=complex(-0.135, -0.07), periodic=True)
    for bad in [dict(nx=0), dict(radius=0), dict(radius=7), dict(h=0.0), dict(scale=0.0), dict(scale=-1.0),
                dict(q=complex(float("nan"), 0.0))]:
        kw = dict(good)
        kw.update(bad)
        d = aar.zstencil_desc(**kw)
        assert lib.aar_zcreate_stencil(C.byref(d), aar.FP64, None, C.byref(h)) == aar.ERR_INVALID_ARG, bad
    d = aar.zstencil_desc(**good)
    d.periodic = 2
    assert lib.aar_zcreate_stencil(C.byref(d), aar.FP64, None, C.byref(h)) == aar.ERR_INVALID_ARG
    d = aar.zstencil_desc(**good)
    assert lib.aar_zcreate_stencil(C.byref(d), 7, None, C.byref(h)) == aar.ERR_INVALID_ARG
    # a zero centre coefficient (no Jacobi scaling)
    d = aar.zstencil_desc(8, 8, 8, 1, [-2.0, 1.0], h=1.0, scale=1.0, q=complex(-6.0, 0.0))
    assert lib.aar_zcreate_stencil(C.byref(d), aar.FP64, None, C.byref(h)) == aar.ERR_INVALID_ARG
    assert lib.aar_zsolve(None, None, None, None, None, None) == aar.ERR_INVALID_ARG
    assert lib.aar_zdestroy(None) == aar.ERR_INVALID_ARG


def test_block_jacobi_descriptors_rejected_without_gpu(lib):
    # aar_stencil_desc.block: 0 / 1 Jacobi, 2 = 2 x 2 x 2 boxes (even sides; periodic sides of at
    # least radius + 2); validated before any device work
    from paper_1606_08740_gb300 import aar

    h = C.c_void_p()
    for kw in [dict(nx=9, ny=8, nz=8, radius=1, weights=[-2.0, 1.0]),
               dict(nx=8, ny=8, nz=4, radius=3, weights=[-49 / 18, 1.5, -0.15, 1 / 90], periodic=True),
               dict(nx=8, ny=8, nz=8, radius=1, weights=[-2.0, 1.0], block=3)]:
        kw.setdefault("block", 2)
        d = aar.stencil_desc(**kw)
        assert lib.aar_create_stencil(C.byref(d), None, aar.FP64, None, C.byref(h)) == aar.ERR_INVALID_ARG, kw
    assert aar.K_BLOCK == 6


def test_complex_block_jacobi_descriptors_rejected_without_gpu(lib):
    # aar_zstencil_desc.block: 0 / 1 Jacobi, 2 = 2 x 2 x 2 boxes (even sides; periodic sides of at
    # least radius + 2); validated before any device work
    from paper_1606_08740_gb300 import aar

    h = C.c_void_p()
    w3 = [-49 / 18, 1.5, -0.15, 1 / 90]
    for kw in [dict(nx=9, ny=8, nz=8, radius=1, weights=[-2.0, 1.0]),
               dict(nx=8, ny=8, nz=4, radius=3, weights=w3),
               dict(nx=8, ny=8, nz=8, radius=1, weights=[-2.0, 1.0], block=3)]:
        kw.setdefault("block", 2)
        d = aar.zstencil_desc(h=0.5, scale=0.0796, q=complex(-0.135, -0.07), periodic=True, **kw)
        assert lib.aar_zcreate_stencil(C.byref(d), aar.FP64, None, C.byref(h)) == aar.ERR_INVALID_ARG, kw
    assert aar.zdesc_of(type("P", (), dict(nx=8, ny=8, nz=8, radius=1, weights=[-2.0, 1.0], h=1.0, scale=1.0,
                                            q=0.5, periodic=True))(), block=2).block == 2


def test_desc_of_carries_geometry_and_preconditioner(lib):
    import workloads
    from paper_1606_08740_gb300 import aar

    P = workloads.periodic_modes(16, radius=3, seed=1)
    d = aar.desc_of(P, block=2)
    assert (d.nx, d.ny, d.nz, d.radius, d.periodic, d.block) == (16, 16, 16, 3, 1, 2)
    assert list(d.w)[:4] == list(P.weights) and d.h == P.h and d.shift == P.shift
    assert aar.desc_of(P).block == 0
