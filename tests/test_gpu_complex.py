"""GPU parity of the complex-valued AAR path (include/aar_complex.h) against the complex FP64
oracle, through the C ABI.

Bar (as for real FP64 solves): the same iteration count and a relative solution error <= 1e-9 at
relative residual tol 1e-10; the operator application agrees to 1e-13 relative (summation order
only). Inputs: the OF-DFT Helmholtz operator of Eq. 7 on periodic aluminium cells
(workloads.ofdft_helmholtz) and seeded uniform complex systems on ragged grids.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1606_08740_gb300 import aar  # noqa: E402

DEV = "cuda:0"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).to(DEV)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def zprob(nx, ny, nz, r, seed, q=complex(0.3, 0.2), scale=1.0, h=1.0, periodic=True):
    return workloads.complex_uniform(nx, ny, nz, r, seed=seed, h=h, scale=scale, q=q, periodic=periodic)


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("r", [1, 3, 6])
@pytest.mark.parametrize("shape", [(37, 29, 23), (5, 70, 9)])
def test_zapply_matches_oracle(r, shape, periodic):
    P = zprob(*shape, r, seed=10 + r, q=workloads.OFDFT_Q, scale=1.0 / (4.0 * math.pi), h=0.486, periodic=periodic)
    g = workloads.rng(200 + r)
    x = g.standard_normal(P.n) + 1j * g.standard_normal(P.n)
    y_ref = oracle.ZOperator(P).apply(x)
    y = torch.empty(P.n, dtype=torch.complex128, device=DEV)
    with aar.ZSolver(aar.zdesc_of(P)) as s:
        s.apply(dev(x), y)
    yg = y.cpu().numpy()
    assert np.max(np.abs(yg - y_ref)) <= 1e-13 * np.max(np.abs(y_ref))


ZCASES = [
    # (name, problem factory, params)
    ("ofdft-al3-h0.486", lambda: workloads.ofdft_helmholtz(3, 0.486, seed=6000), dict(m=9, p=8)),
    ("uniform-r3-ragged-complex-omega", lambda: zprob(21, 19, 17, 3, seed=6101, q=complex(0.3, 0.2)),
     dict(m=7, p=6, omega=0.5 + 0.1j, beta=0.6 - 0.2j)),
    ("dirichlet-r1-eq7", lambda: zprob(33, 20, 14, 1, seed=6102, q=workloads.OFDFT_Q, scale=1 / (4 * math.pi),
                                       h=0.486, periodic=False), dict(m=5, p=4)),
    ("r6-m16", lambda: zprob(20, 18, 16, 6, seed=6103, q=complex(0.8, -0.5)), dict(m=16, p=5)),
    ("p1-m3", lambda: zprob(12, 11, 10, 2, seed=6104, q=complex(0.5, 0.5)), dict(m=3, p=1)),
]


@pytest.mark.parametrize("name,make,kw", ZCASES, ids=[c[0] for c in ZCASES])
def test_zsolve_matches_oracle(name, make, kw):
    P = make()
    tol = 1e-10
    ref = oracle.zsolve(P, tol=tol, **kw)
    assert ref.status == oracle.OK
    x = torch.empty(P.n, dtype=torch.complex128, device=DEV)
    with aar.ZSolver(aar.zdesc_of(P)) as s:
        res = s.solve(dev(P.b), x, prm=aar.zparams(tol=tol, **kw))
    xg = x.cpu().numpy()
    assert res.status == aar.OK
    assert res.iterations == ref.iterations, (res.iterations, ref.iterations)
    assert res.anderson_steps == ref.anderson_steps
    err = rel(xg, ref.x)
    print(f"{name}: {res.iterations} its, rel err vs oracle {err:.2e}, r = {res.rel_residual:.2e}")
    assert err <= 1e-9
    assert oracle.ZOperator(P).rel_residual(P.b, xg) <= tol * 1.0001


def sigma_min_periodic(P) -> float:
    """Smallest singular value of the periodic operator of Eq. 7: it is normal (circulant), so
    this is min |scale * symbol(theta) + q| over the grid's Fourier modes."""
    def axis(n):
        th = 2 * np.pi * np.arange(n) / n
        return -(P.weights[0] + 2 * sum(P.weights[k] * np.cos(k * th) for k in range(1, P.radius + 1))) / P.h ** 2
    lam = axis(P.nx)[None, None, :] + axis(P.ny)[None, :, None] + axis(P.nz)[:, None, None]
    return float(np.min(np.abs(P.scale * lam + P.q)))


def test_zofdft_fine_mesh_reaches_the_oracle_solution():
    # Eq. 7 on one aluminium cell at h = 0.216 (the Jacobi runs of Sec. 3.2's appendix): here the
    # history's Gram matrix is nearly singular and the iteration count moves with rounding (the
    # oracle itself takes 711-743 iterations under 1e-16 perturbations of b), so the unique
    # quantity is compared: both solves converge and their solutions agree within the bound
    # 2 tol ||b|| / sigma_min(A) that two tol-accurate solutions obey
    P = workloads.ofdft_helmholtz(1, 0.216, seed=6000)
    tol = 1e-10
    ref = oracle.zsolve(P, m=9, p=8, tol=tol)
    x = torch.empty(P.n, dtype=torch.complex128, device=DEV)
    with aar.ZSolver(aar.zdesc_of(P)) as s:
        res = s.solve(dev(P.b), x, prm=aar.zparams(m=9, p=8, tol=tol))
    xg = x.cpu().numpy()
    assert res.status == aar.OK and ref.status == oracle.OK
    assert oracle.ZOperator(P).rel_residual(P.b, xg) <= tol * 1.0001
    bound = 2 * tol * np.linalg.norm(P.b) / sigma_min_periodic(P)
    print(f"al1 h=0.216: {res.iterations} its (oracle {ref.iterations}), |x - x_oracle| = "
          f"{np.linalg.norm(xg - ref.x):.2e} <= {bound:.2e}")
    assert np.linalg.norm(xg - ref.x) <= bound
    assert 0.75 * ref.iterations <= res.iterations <= 1.35 * ref.iterations


def test_zm0_fixed_iterations_match_oracle():
    # m = 0, tol = 0: Jacobi-Richardson with omega / beta alternation, exactly max_iter updates
    P = zprob(17, 13, 11, 3, seed=6105, q=complex(0.4, -0.3))
    ref = oracle.zsolve(P, omega=0.5 + 0.2j, beta=0.7 - 0.3j, m=0, p=4, tol=0.0, max_iter=23)
    x = torch.empty(P.n, dtype=torch.complex128, device=DEV)
    with aar.ZSolver(aar.zdesc_of(P)) as s:
        res = s.solve(dev(P.b), x, prm=aar.zparams(omega=0.5 + 0.2j, beta=0.7 - 0.3j, m=0, p=4, tol=0.0, max_iter=23),
                      raise_on_error=False)
    assert res.status == aar.NOT_CONVERGED and res.iterations == 23
    assert rel(x.cpu().numpy(), ref.x) <= 1e-13


def test_zfixed_iterations_with_history_match_oracle():
    # tol = 0: both run exactly max_iter updates through 6 Anderson steps
    P = zprob(23, 16, 12, 3, seed=6106, q=workloads.OFDFT_Q, scale=1 / (4 * math.pi), h=0.486)
    ref = oracle.zsolve(P, m=9, p=8, tol=0.0, max_iter=50)
    x = torch.empty(P.n, dtype=torch.complex128, device=DEV)
    with aar.ZSolver(aar.zdesc_of(P)) as s:
        res = s.solve(dev(P.b), x, prm=aar.zparams(m=9, p=8, tol=0.0, max_iter=50), raise_on_error=False)
    assert res.status == aar.NOT_CONVERGED and res.iterations == 50 and res.anderson_steps == 6
    assert rel(x.cpu().numpy(), ref.x) <= 1e-9


def test_zhost_buffers_x0_and_edge_cases():
    P = zprob(16, 12, 10, 3, seed=6107, q=complex(0.6, 0.1))
    prm = aar.zparams(m=7, p=6, tol=1e-10)
    with aar.ZSolver(aar.zdesc_of(P)) as s:
        xd = torch.empty(P.n, dtype=torch.complex128, device=DEV)
        rd = s.solve(dev(P.b), xd, prm=prm)
        xh = np.empty(P.n, dtype=np.complex128)
        rh = s.solve(np.ascontiguousarray(P.b), xh, prm=prm)
        assert rh.iterations == rd.iterations
        assert np.array_equal(xh, xd.cpu().numpy())
        # a converged x0 stops at the first Anderson step
        x0 = xd.clone()
        r0 = s.solve(dev(P.b), xd, x0=x0, prm=prm)
        assert r0.iterations == prm.p - 1
        ref = oracle.zsolve(P, m=7, p=6, tol=1e-10, x0=x0.cpu().numpy())
        assert ref.iterations == r0.iterations
        # zero right-hand side: x = 0 after 0 iterations
        z = torch.zeros(P.n, dtype=torch.complex128, device=DEV)
        xz = torch.full((P.n,), 1 + 1j, dtype=torch.complex128, device=DEV)
        rz = s.solve(z, xz, prm=prm)
        assert rz.status == aar.OK and rz.iterations == 0 and bool((xz == 0).all())
        # residual entry point against the oracle
        rr = s.rel_residual(dev(P.b), xd)
        assert abs(rr - oracle.ZOperator(P).rel_residual(P.b, xd.cpu().numpy())) <= 1e-6 * rr + 1e-15


def test_zfull_size_sampled_against_oracle():
    # the benchmark's 256^3 OF-DFT cell (16 x 16 x 16 aluminium cells at the paper's h = 0.486):
    # the operator at sampled points against the oracle's one-point evaluation, and a solve to
    # 1e-6 whose FP64 residual is certified on the device and at sampled points
    P = workloads.ofdft_helmholtz(16, 0.486, seed=6000)
    assert P.nx == 256
    op = oracle.ZOperator(P)
    g = workloads.rng(6200)
    x = g.standard_normal(P.n) + 1j * g.standard_normal(P.n)
    idx = np.unique(np.concatenate([g.integers(0, P.n, 300), [0, P.n - 1, P.nx - 1, P.nx * P.ny]]))
    y = torch.empty(P.n, dtype=torch.complex128, device=DEV)
    with aar.ZSolver(aar.zdesc_of(P)) as s:
        s.apply(dev(x), y)
        ys = y.cpu().numpy()[idx]
        ref = op.apply_at(x, idx)
        assert np.max(np.abs(ys - ref)) <= 1e-13 * np.max(np.abs(ref))
        xs = torch.empty(P.n, dtype=torch.complex128, device=DEV)
        res = s.solve(dev(P.b), xs, prm=aar.zparams(tol=1e-6))
        assert res.status == aar.OK
        assert s.rel_residual(dev(P.b), xs) <= 1e-6 * 1.0001
        xh = xs.cpu().numpy()
        rs = P.b[idx] - op.apply_at(xh, idx)
        s.apply(xs, y)
        rg = P.b[idx] - y.cpu().numpy()[idx]
        assert np.max(np.abs(rs - rg)) <= 1e-12 * np.max(np.abs(P.b))


# ------------------------------------------------------------------- mixed precision

ZMIXED = [
    ("ofdft-al3-h0.486", lambda: workloads.ofdft_helmholtz(3, 0.486, seed=6000), dict(m=9, p=8)),
    ("uniform-r3-ragged-complex-omega", lambda: zprob(21, 19, 17, 3, seed=6101, q=complex(0.3, 0.2)),
     dict(m=7, p=6, omega=0.5 + 0.1j, beta=0.6 - 0.2j)),
    ("r6-m16", lambda: zprob(20, 18, 16, 6, seed=6103, q=complex(0.8, -0.5)), dict(m=16, p=5)),
]


@pytest.mark.parametrize("name,make,kw", ZMIXED, ids=[c[0] for c in ZMIXED])
def test_zmixed_reaches_fp64_tolerance(name, make, kw):
    # FP32 inner AAR in FP64 refinement: the FP64 residual (the oracle's) reaches tol and the
    # solution lies within 2 tol ||b|| / sigma_min(A) of the FP64 oracle's
    P = make()
    tol = 1e-10
    ref = oracle.zsolve(P, tol=tol, **kw)
    x = torch.empty(P.n, dtype=torch.complex128, device=DEV)
    with aar.ZSolver(aar.zdesc_of(P), aar.MIXED) as s:
        res = s.solve(dev(P.b), x, prm=aar.zparams(tol=tol, **kw))
        r_dev = s.rel_residual(dev(P.b), x)
    xg = x.cpu().numpy()
    r_true = oracle.ZOperator(P).rel_residual(P.b, xg)
    err = rel(xg, ref.x)
    bound = 2 * tol * np.linalg.norm(P.b) / sigma_min_periodic(P)
    print(f"{name} mixed: {res.iterations} inner its, {res.refinements} refinements (FP64: {ref.iterations} its), "
          f"r = {r_true:.2e}, error vs FP64 oracle {err:.2e}")
    assert res.status == aar.OK and res.refinements >= 1
    assert r_true <= tol * 1.0001 and abs(r_dev - r_true) <= 1e-3 * r_true
    assert abs(res.rel_residual - r_true) <= 1e-3 * r_true
    assert np.linalg.norm(xg - ref.x) <= bound


def test_zmixed_host_buffers_edge_cases_and_profile():
    P = zprob(16, 12, 10, 3, seed=6107, q=complex(0.6, 0.1))
    prm = aar.zparams(m=7, p=6, tol=1e-9)
    with aar.ZSolver(aar.zdesc_of(P), aar.MIXED) as s:
        xd = torch.empty(P.n, dtype=torch.complex128, device=DEV)
        rd = s.solve(dev(P.b), xd, prm=prm)
        xh = np.empty(P.n, dtype=np.complex128)
        rh = s.solve(np.ascontiguousarray(P.b), xh, prm=prm)
        assert rd.status == rh.status == aar.OK and rh.iterations == rd.iterations
        assert np.array_equal(xh, xd.cpu().numpy())
        for k in (aar.K_SWEEP, aar.K_SWEEP_ANDERSON, aar.K_GRAM, aar.K_UPDATE, aar.K_RESID64, aar.K_FINALIZE):
            assert s.profile_kernel(k, 2) > 0.0
        # a solution as x0: no refinement is needed
        r0 = s.solve(dev(P.b), xd, x0=xd.clone(), prm=prm)
        assert r0.status == aar.OK and r0.iterations == 0 and r0.refinements == 0
        z = torch.zeros(P.n, dtype=torch.complex128, device=DEV)
        rz = s.solve(z, xd, prm=prm)
        assert rz.status == aar.OK and rz.iterations == 0 and bool((xd == 0).all())
        # max_iter caps the inner iterations summed over refinements
        rc = s.solve(dev(P.b), xd, prm=aar.zparams(m=7, p=6, tol=1e-14, max_iter=20), raise_on_error=False)
        assert rc.status == aar.NOT_CONVERGED and rc.iterations <= 20


def test_zmixed_full_size_sampled_against_oracle():
    # the benchmark's 256^3 OF-DFT cell in the mixed form: tol 1e-6 reached in FP64, certified on
    # the device and, at sampled points, by the oracle's one-point operator
    P = workloads.ofdft_helmholtz(16, 0.486, seed=6000)
    op = oracle.ZOperator(P)
    g = workloads.rng(6300)
    idx = np.unique(g.integers(0, P.n, 300))
    x = torch.empty(P.n, dtype=torch.complex128, device=DEV)
    with aar.ZSolver(aar.zdesc_of(P), aar.MIXED) as s:
        res = s.solve(dev(P.b), x, prm=aar.zparams(tol=1e-6))
        assert res.status == aar.OK
        r_dev = s.rel_residual(dev(P.b), x)
    assert r_dev <= 1e-6 * 1.0001
    xh = x.cpu().numpy()
    y = torch.empty_like(x)
    with aar.ZSolver(aar.zdesc_of(P)) as s64:
        s64.apply(x, y)
    rs = P.b[idx] - op.apply_at(xh, idx)
    rg = P.b[idx] - y.cpu().numpy()[idx]
    assert np.max(np.abs(rs - rg)) <= 1e-12 * np.max(np.abs(P.b))


_CHILD = r"""
import sys, numpy as np, torch, workloads
from paper_1606_08740_gb300 import aar
out = {}
for name, (nx, ny, nz, r, periodic, q) in enumerate([
        (23, 13, 11, 2, False, complex(0.5, 0.3)),
        (19, 17, 9, 5, True, complex(0.7, -0.2)),
        (33, 9, 14, 6, False, complex(0.9, 0.4)),
        (40, 24, 7, 3, True, complex(0.6, 0.2)),
        (120, 100, 150, 3, False, complex(0.9, 0.3))]):
    P = workloads.complex_uniform(nx, ny, nz, r, seed=6400 + name, q=q, periodic=periodic)
    b = torch.from_numpy(np.ascontiguousarray(P.b)).to("cuda:0")
    x = torch.empty_like(b)
    with aar.ZSolver(aar.zdesc_of(P), aar.MIXED) as s:
        res = s.solve(b, x, prm=aar.zparams(m=7, p=5, tol=1e-9), raise_on_error=False)
    out[f"x{name}"] = x.cpu().numpy()
    out[f"its{name}"] = np.array([res.iterations, res.status])
np.savez(sys.argv[1], **out)
"""


def test_zsweep_staged_matches_register_fed(tmp_path):
    # the staged FP32 sweep of the inner solves (planes in shared memory) forms the same sums in
    # the same order as the register-fed one: whole mixed solves agree bit for bit, on Dirichlet
    # and periodic grids that are ragged against its 32 x 8 tiles, radii 2, 3, 5 and 6, with one
    # plane per CTA (a periodic z side of 2r + 1 planes) up to 12 (longer than its ring of 2r + 3
    # staged planes). The switch is read once per process, so each form runs in a child process.
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    files = []
    for reg in ("0", "1"):
        f = str(tmp_path / f"x{reg}.npz")
        env = dict(os.environ, AAR_ZSWEEP_REG=reg, PYTHONPATH=root + os.pathsep + os.environ.get("PYTHONPATH", ""))
        subprocess.run([sys.executable, "-c", _CHILD, f], check=True, cwd=root, env=env, timeout=600)
        files.append(np.load(f))
    a, b = files
    for k in a.files:
        assert np.array_equal(a[k], b[k]), k
    for i in range(5):
        assert a[f"its{i}"][1] == aar.OK
