"""GPU parity of complex block Jacobi (2 x 2 x 2 boxes, the block Jacobi of Sec. 3.2's Helmholtz
runs with exact block solves; include/aar_complex.h, block = 2) against the complex FP64 oracle's
block-Jacobi solve (orz_aar_solve_block), through the C ABI.

Bar as for every FP64 solve: the same iteration count and a relative solution error <= 1e-9 at
relative residual tol 1e-10, and the iterate after a fixed iteration count to 1e-12 per step;
the mixed form reaches the FP64 tolerance (the oracle's residual) and lies within the bound
2 tol ||b|| / sigma_min(A) of the oracle's solution.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1606_08740_gb300 import aar  # noqa: E402
from tests.test_gpu_complex import sigma_min_periodic  # noqa: E402

DEV = "cuda:0"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).to(DEV)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [
    ("ofdft-al1-h0.486", lambda: workloads.ofdft_helmholtz(1, 0.486, seed=6000), dict(m=9, p=8)),
    ("ofdft-al3-h0.486", lambda: workloads.ofdft_helmholtz(3, 0.486, seed=6000), dict(m=9, p=8)),
    ("uniform-r3-complex-omega", lambda: workloads.complex_uniform(22, 18, 16, 3, seed=6201, q=complex(0.3, 0.2)),
     dict(m=7, p=6, omega=0.5 + 0.1j, beta=0.6 - 0.2j)),
    ("dirichlet-r1", lambda: workloads.complex_uniform(24, 16, 12, 1, seed=6202, q=workloads.OFDFT_Q,
                                                      scale=1 / (4 * math.pi), h=0.486, periodic=False),
     dict(m=5, p=4)),
    ("r6-periodic", lambda: workloads.complex_uniform(16, 16, 10, 6, seed=6203, q=complex(0.8, -0.5)), dict(m=7, p=5)),
]


@pytest.mark.parametrize("name,make,kw", CASES, ids=[c[0] for c in CASES])
def test_block_zsolve_matches_oracle(name, make, kw):
    P = make()
    tol = 1e-10
    ref = oracle.zsolve(P, tol=tol, block=2, **kw)
    assert ref.status == oracle.OK
    x = torch.empty(P.n, dtype=torch.complex128, device=DEV)
    with aar.ZSolver(aar.zdesc_of(P, block=2)) as s:
        res = s.solve(dev(P.b), x, prm=aar.zparams(tol=tol, **kw))
    xg = x.cpu().numpy()
    assert res.status == aar.OK
    assert res.iterations == ref.iterations, (res.iterations, ref.iterations)
    err = rel(xg, ref.x)
    print(f"{name} (block Jacobi): {res.iterations} its, rel err vs oracle {err:.2e}")
    assert err <= 1e-9
    assert oracle.ZOperator(P).rel_residual(P.b, xg) <= tol * 1.0001


@pytest.mark.parametrize("iters", [1, 7, 13])
def test_block_fixed_iterations_match_oracle(iters):
    P = workloads.complex_uniform(14, 12, 10, 2, seed=6204, q=complex(0.5, -0.3))
    kw = dict(m=7, p=6, tol=0.0, max_iter=iters)
    ref = oracle.zsolve(P, block=2, **kw)
    x = torch.empty(P.n, dtype=torch.complex128, device=DEV)
    with aar.ZSolver(aar.zdesc_of(P, block=2)) as s:
        res = s.solve(dev(P.b), x, prm=aar.zparams(**kw), raise_on_error=False)
        assert res.status == aar.NOT_CONVERGED and res.iterations == iters
        if iters >= 6:  # a solve with an Anderson step leaves the state aar_zprofile_kernel times
            assert s.profile_kernel(aar.K_BLOCK, 2) > 0.0
    assert rel(x.cpu().numpy(), ref.x) <= 1e-12 * iters


def test_block_mixed_reaches_fp64_tolerance_and_fewer_iterations():
    # the Sec. 3.2 cell (48^3) at its tolerance 1e-6: the mixed form with block Jacobi reaches the
    # FP64 tolerance, lies within 2 tol ||b|| / sigma_min(A) of the oracle's block-Jacobi solution,
    # and the block preconditioner needs fewer iterations than Jacobi in both forms
    P = workloads.ofdft_helmholtz(3, 0.486, seed=6000)
    tol = 1e-6
    b = dev(P.b)
    x = torch.empty_like(b)
    its = {}
    for blk in (0, 2):
        for prec in (aar.FP64, aar.MIXED):
            with aar.ZSolver(aar.zdesc_of(P, block=blk), prec) as s:
                res = s.solve(b, x, prm=aar.zparams(tol=tol))
            assert res.status == aar.OK
            its[(blk, prec)] = res.iterations
    xg = x.cpu().numpy()  # the last: block Jacobi, mixed
    assert oracle.ZOperator(P).rel_residual(P.b, xg) <= tol * 1.0001
    ref = oracle.zsolve(P, tol=tol, block=2)
    err = rel(xg, ref.x)
    bound = 2 * tol * np.linalg.norm(P.b) / (sigma_min_periodic(P) * np.linalg.norm(ref.x))
    print(f"Eq. 7 cell 48^3: iterations {its}; block mixed error vs oracle {err:.2e} (bound {bound:.2e})")
    assert err <= bound
    assert its[(2, aar.FP64)] < 0.8 * its[(0, aar.FP64)]
    assert its[(2, aar.MIXED)] < 0.8 * its[(0, aar.MIXED)]
