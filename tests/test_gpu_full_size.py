"""The workloads at their full sizes, in the configuration bench.py runs them: the 32^3 Poisson
case against the oracle element by element; the 256^3 radius-6 case in FP64 against the oracle
element by element at a fixed iteration count; the 128^3 CSR convection-diffusion case, the
512-system batch and the 256^3 periodic case through properties the oracle checks at any size
(FP64 true residual from the oracle, sampled operator outputs)."""
import numpy as np
import pytest

import dense
import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1606_08740_gb300 import aar  # noqa: E402


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def test_poisson_32_fp64_matches_oracle():
    P = workloads.poisson_uniform(32, radius=1, seed=0)
    prm = dict(omega=0.6, beta=0.6, m=7, p=6, tol=1e-10)
    ref = oracle.solve(P, **prm)
    x = torch.empty(P.n, dtype=torch.float64, device="cuda:0")
    with aar.Solver.stencil(aar.desc_of(P)) as s:
        res = s.solve(_dev(P.b), x, prm=aar.params(**prm))
    assert res.status == aar.OK and res.iterations == ref.iterations
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-9 * np.linalg.norm(ref.x)


def test_r6_256_fp64_matches_oracle_at_fixed_iteration_count():
    # the 256^3 radius-6 workload in FP64 (the full-size tiling of the FP64 register sweep, the
    # FP64 Gram, eigen pseudoinverse and literal update): tol = 0 and two Anderson cycles, so both
    # sides run exactly 12 updates (Anderson steps at k = 5 and 11) and return x_12
    P = workloads.poisson_sine_modes(256, radius=6, seed=1000)
    prm = dict(omega=0.6, beta=0.6, m=7, p=6, tol=0.0, max_iter=12)
    ref = oracle.solve(P, **prm)
    assert ref.status == oracle.NOT_CONVERGED and ref.iterations == 12
    x = torch.empty(P.n, dtype=torch.float64, device="cuda:0")
    with aar.Solver.stencil(aar.desc_of(P), aar.FP64) as s:
        res = s.solve(_dev(P.b), x, prm=aar.params(**prm))
    assert res.status == aar.NOT_CONVERGED and res.iterations == 12 and res.anderson_steps == 2
    xg = x.cpu().numpy()
    err = np.linalg.norm(xg - ref.x) / np.linalg.norm(ref.x)
    print(f"256^3 radius-6 FP64 at k = 12: rel. error vs oracle {err:.3e}")
    assert err <= 1e-9
    assert np.max(np.abs(xg - ref.x)) <= 1e-9 * np.max(np.abs(ref.x))


def test_convection_diffusion_128_csr_full_size():
    P = workloads.convection_diffusion(128, seed=2000)
    op = oracle.Operator(P)
    rp, ci, va = _dev(P.row_ptr), _dev(P.col_idx), _dev(P.val)
    x = torch.empty(P.n, dtype=torch.float64, device="cuda:0")
    with aar.Solver.csr(rp, ci, va) as s:
        xr = workloads.rng(3).standard_normal(P.n)
        y = torch.empty_like(x)
        s.apply(_dev(xr), y)
        idx = workloads.rng(4).integers(0, P.n, 3000)
        ref = op.apply_at(xr, idx)
        assert np.max(np.abs(y.cpu().numpy()[idx] - ref)) <= 1e-13 * np.max(np.abs(ref))
        res = s.solve(_dev(P.b), x, prm=aar.params(omega=0.5, beta=0.5, m=10, p=5, tol=1e-8))
    assert res.status == aar.OK
    assert op.rel_residual(P.b, x.cpu().numpy()) <= 1e-8 * 1.0001


def test_batched_512_full_size_sampled():
    probs = workloads.batched_helmholtz(512, seed_base=3000)
    bt = aar.Batch([aar.desc_of(P) for P in probs], aar.MIXED)
    bs = [_dev(P.b) for P in probs]
    xs = [torch.empty(P.n, dtype=torch.float64, device="cuda:0") for P in probs]
    res = bt.solve(bs, xs, aar.params(omega=0.6, beta=0.6, m=7, p=6, tol=1e-8))
    bt.close()
    assert all(r.status == aar.OK for r in res)
    for i in range(0, 512, 37):
        assert oracle.Operator(probs[i]).rel_residual(probs[i].b, xs[i].cpu().numpy()) <= 1e-8 * 1.0001


def test_periodic_256_mixed_full_size_sampled():
    # the periodic row at the size bench.py runs it (256^3, sixth order, the periodic paired FP32
    # sweep): the mixed solve reaches the FP64 tolerance, and the library's operator agrees with
    # the oracle's one-point evaluation at sampled points of the solution
    P = workloads.periodic_modes(256, radius=3, seed=5000)
    op = oracle.Operator(P)
    b = _dev(P.b)
    x = torch.empty(P.n, dtype=torch.float64, device="cuda:0")
    y = torch.empty_like(x)
    with aar.Solver.stencil(aar.desc_of(P), aar.MIXED) as s:
        res = s.solve(b, x, prm=aar.params(omega=0.6, beta=0.6, m=7, p=6, tol=1e-8))
        s.apply(x, y)
    assert res.status == aar.OK
    xh = x.cpu().numpy()
    # the FP64 relative residual certified by the oracle's own operator at full size
    r = op.rel_residual(P.b, xh)
    assert r <= 1e-8 * 1.0001, r
    assert abs(res.rel_residual - r) <= 1e-3 * r
    # error against the exact zero-mean solution through that residual (an FP64 oracle solve of
    # this size takes tens of minutes on one core)
    xz = xh - xh.mean()
    bound = r * np.linalg.norm(P.b) / (dense.stencil_lambda_min(P, zero_mean=True) * np.linalg.norm(xz))
    print(f"256^3 periodic mixed: r = {r:.3e}, error vs the exact solution <= {bound:.3e}")
    assert bound <= 1e-5
    idx = workloads.rng(5).integers(0, P.n, 3000)
    ref = op.apply_at(xh, idx)
    assert np.max(np.abs(y.cpu().numpy()[idx] - ref)) <= 1e-13 * np.max(np.abs(ref))
