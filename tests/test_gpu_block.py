"""GPU parity of block Jacobi with 2 x 2 x 2 boxes (row f4; aar_stencil_desc.block = 2) against the
oracle's block-Jacobi solve, through the C ABI.

The GPU applies M^{-1} in the cube's Walsh-Hadamard basis; the oracle solves each block's 8 x 8
system read entry by entry from the operator. FP64 solves must stop at the same iteration and
agree to 1e-9 relative at tol 1e-10; mixed-precision solves must reach the FP64 tolerance.
"""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1606_08740_gb300 import aar  # noqa: E402

DEV = "cuda:0"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def prob(nx, ny, nz, r, seed, shift=0.1, periodic=False, h=1.0):
    b = workloads.uniform_rhs(nx * ny * nz, seed)
    if periodic and shift == 0.0:
        b = b - b.mean()
    return workloads.StencilProblem(nx, ny, nz, r, workloads.stencil_weights(r), h, shift, b, periodic=periodic)


def bdesc(P):
    d = aar.desc_of(P)
    d.block = 2
    return d


BCASES = [
    ("r1-dirichlet", lambda: prob(16, 12, 10, 1, seed=7001, shift=0.1), dict(m=7, p=6)),
    ("r3-periodic-helmholtz", lambda: prob(16, 16, 12, 3, seed=7002, shift=0.3, periodic=True), dict(m=7, p=6)),
    ("r6-dirichlet", lambda: prob(20, 16, 14, 6, seed=7003, shift=0.05, h=0.8), dict(m=9, p=8)),
    ("r2-p1-m3", lambda: prob(12, 10, 8, 2, seed=7004, shift=0.2), dict(m=3, p=1)),
]


@pytest.mark.parametrize("name,make,kw", BCASES, ids=[c[0] for c in BCASES])
def test_block_fp64_matches_oracle(name, make, kw):
    P = make()
    tol = 1e-10
    ref = oracle.solve(P, tol=tol, block=2, **kw)
    assert ref.status == oracle.OK
    x = torch.empty(P.n, dtype=torch.float64, device=DEV)
    with aar.Solver.stencil(bdesc(P), aar.FP64) as s:
        res = s.solve(dev(P.b), x, prm=aar.params(tol=tol, **kw))
    xg = x.cpu().numpy()
    err = rel(xg, ref.x)
    print(f"{name}: {res.iterations} its (oracle {ref.iterations}), rel err {err:.2e}")
    assert res.status == aar.OK and res.iterations == ref.iterations
    assert err <= 1e-9
    assert oracle.Operator(P).rel_residual(P.b, xg) <= tol * 1.0001


def test_block_fixed_iterations_match_oracle():
    # tol = 0: both run exactly max_iter updates (Richardson and Anderson steps through M^{-1})
    P = prob(14, 12, 10, 3, seed=7005, shift=0.2)
    ref = oracle.solve(P, m=5, p=4, tol=0.0, max_iter=37, block=2)
    x = torch.empty(P.n, dtype=torch.float64, device=DEV)
    with aar.Solver.stencil(bdesc(P), aar.FP64) as s:
        res = s.solve(dev(P.b), x, prm=aar.params(m=5, p=4, tol=0.0, max_iter=37), raise_on_error=False)
    assert res.status == aar.NOT_CONVERGED and res.iterations == 37
    assert rel(x.cpu().numpy(), ref.x) <= 1e-12


@pytest.mark.parametrize("name,make,kw", BCASES[:3], ids=[c[0] for c in BCASES[:3]])
def test_block_mixed_reaches_fp64_tolerance(name, make, kw):
    P = make()
    tol = 1e-10
    ref = oracle.solve(P, tol=tol, block=2, **kw)
    x = torch.empty(P.n, dtype=torch.float64, device=DEV)
    with aar.Solver.stencil(bdesc(P), aar.MIXED) as s:
        res = s.solve(dev(P.b), x, prm=aar.params(tol=tol, **kw))
    xg = x.cpu().numpy()
    r_true = oracle.Operator(P).rel_residual(P.b, xg)
    print(f"{name} mixed: {res.iterations} inner its, {res.refinements} refinements, r = {r_true:.2e}, "
          f"error vs FP64 oracle {rel(xg, ref.x):.2e}")
    assert res.status == aar.OK and r_true <= tol * 1.0001


def test_block_needs_fewer_iterations_than_jacobi():
    P = workloads.poisson_uniform(24, radius=6, seed=7006)
    prm = aar.params(m=7, p=6, tol=1e-8)
    x = torch.empty(P.n, dtype=torch.float64, device=DEV)
    with aar.Solver.stencil(aar.desc_of(P), aar.MIXED) as s:
        rj = s.solve(dev(P.b), x, prm=prm)
    with aar.Solver.stencil(bdesc(P), aar.MIXED) as s:
        rb = s.solve(dev(P.b), x, prm=prm)
        assert s.profile_kernel(aar.K_BLOCK, 3) > 0.0
    print(f"24^3 radius 6: Jacobi {rj.iterations} inner its, block Jacobi {rb.iterations}")
    assert rb.status == aar.OK and rb.iterations < 0.8 * rj.iterations


def test_block_invalid_configurations():
    ok = prob(8, 8, 8, 1, seed=7007)
    odd_side = prob(9, 8, 8, 1, seed=1)
    short_periodic = prob(8, 8, 4, 3, seed=1, shift=0.2, periodic=True)  # nz = 4 < radius + 2
    for bad in [odd_side, short_periodic]:
        with pytest.raises(aar.AARError) as ei:
            aar.Solver.stencil(bdesc(bad), aar.FP64)
        assert ei.value.status == aar.ERR_INVALID_ARG
    d = bdesc(ok)
    d.block = 3
    with pytest.raises(aar.AARError):
        aar.Solver.stencil(d, aar.FP64)
    dinv = torch.full((ok.n,), 1.0 / 6.1, dtype=torch.float64, device=DEV)
    with pytest.raises(aar.AARError) as ei:
        aar.Solver.stencil(bdesc(ok), aar.FP64, dinv=dinv)
    assert ei.value.status == aar.ERR_INVALID_ARG
    with aar.Solver.stencil(aar.desc_of(ok), aar.MIXED) as s:
        x = torch.empty(ok.n, dtype=torch.float64, device=DEV)
        s.solve(dev(ok.b), x, prm=aar.params(m=5, p=4, tol=1e-8))
        with pytest.raises(aar.AARError) as ei:
            s.profile_kernel(aar.K_BLOCK, 1)
        assert ei.value.status == aar.ERR_UNSUPPORTED


def test_block_full_size_r6_256_mixed():
    # the headline workload (256^3 radius-6 Poisson, sine modes) with block Jacobi: the mixed
    # solve reaches the FP64 tolerance, certified by the library's FP64 residual
    P = workloads.poisson_sine_modes(256, radius=6, seed=1000)
    x = torch.empty(P.n, dtype=torch.float64, device=DEV)
    with aar.Solver.stencil(bdesc(P), aar.MIXED) as s:
        b = dev(P.b)
        res = s.solve(b, x, prm=aar.params(omega=0.6, beta=0.6, m=7, p=6, tol=1e-8))
        r = s.rel_residual(b, x)
    print(f"256^3 r6 block Jacobi: {res.iterations} inner its, {res.refinements} refinements, r = {r:.2e}")
    assert res.status == aar.OK and r <= 1e-8 * 1.0001
    assert oracle.Operator(P).rel_residual(P.b, x.cpu().numpy()) <= 1e-8 * 1.0001


@pytest.mark.parametrize("shape,r,periodic", [((64, 48, 40), 6, False), ((64, 64, 32), 3, True), ((128, 18, 10), 1, False)])
def test_block_fused_sweep_matches_two_pass(shape, r, periodic):
    # the paired sweep with the boxes fused (variants 6, 7) and the register sweep followed by
    # k_block_apply (variant 0, forced through the tile hint) take the same steps. Their tiles sum
    # the FP32 residual norms in different orders, which can move an inner solve's stopping point
    # within the tolerance: both must reach the FP64 tolerance (the oracle's residual), in the
    # same number of inner iterations, and agree to well within what the tolerance allows
    P = prob(*shape, r, seed=7100 + r, shift=0.05, periodic=periodic)
    prm = aar.params(m=7, p=6, tol=1e-8)
    out = {}
    for hint in (0, 1):
        d = bdesc(P)
        d.tile_variant = hint  # 0: automatic (fused for these grids), 1: variant 0 (two-pass)
        x = torch.empty(P.n, dtype=torch.float64, device=DEV)
        with aar.Solver.stencil(d, aar.MIXED) as s:
            res = s.solve(dev(P.b), x, prm=prm)
            fused = hint == 0
            if fused:
                with pytest.raises(aar.AARError):
                    s.profile_kernel(aar.K_BLOCK, 1)  # no separate block pass
        assert res.status == aar.OK
        out[hint] = (x.cpu().numpy(), res.iterations)
    assert out[0][1] == out[1][1]
    op = oracle.Operator(P)
    for hint in (0, 1):
        assert op.rel_residual(P.b, out[hint][0]) <= 1e-8 * 1.0001
    assert rel(out[0][0], out[1][0]) <= 1e-7


def _mixed_problems():
    # two block-Jacobi systems (one paired-sweep sized, one small) and a Jacobi one, radius 3
    return [(prob(64, 32, 16, 3, seed=7201, shift=0.2), 2), (prob(12, 10, 8, 3, seed=7202, shift=0.3), 2),
            (prob(20, 16, 14, 3, seed=7203, shift=0.1), 0)]


def test_block_in_a_batch_equals_the_single_solves():
    # a batch may mix block-Jacobi and Jacobi systems; each system's arithmetic depends on its own
    # size only, so its result equals its single solve bit for bit
    probs = _mixed_problems()
    prm = aar.params(m=7, p=6, tol=1e-8)
    descs = []
    for P, blk in probs:
        d = aar.desc_of(P)
        d.block = blk
        descs.append(d)
    bs = [dev(P.b) for P, _ in probs]
    xs = [torch.empty(P.n, dtype=torch.float64, device=DEV) for P, _ in probs]
    bt = aar.Batch(descs, aar.MIXED)
    res = bt.solve(bs, xs, prm)
    bt.close()
    for (P, blk), d, b, x, r in zip(probs, descs, bs, xs, res):
        assert r.status == aar.OK
        assert oracle.Operator(P).rel_residual(P.b, x.cpu().numpy()) <= 1e-8 * 1.0001
        x1 = torch.empty_like(x)
        with aar.Solver.stencil(d, aar.MIXED) as s:
            r1 = s.solve(b, x1, prm=prm)
        assert r1.iterations == r.iterations and bool(torch.equal(x1, x)), (blk, r1.iterations, r.iterations)


def test_block_requests_in_the_server():
    # the server admits block-Jacobi requests beside Jacobi ones; every result reaches the FP64
    # tolerance and equals the request's solve alone
    probs = _mixed_problems()
    prm = aar.params(m=7, p=6, tol=1e-8)
    sv = aar.Server(3, aar.MIXED, budget_bytes=4 << 30, max_active=8)
    xs = [np.empty(P.n) for P, _ in probs]
    ids = []
    for (P, blk), x in zip(probs, xs):
        d = aar.desc_of(P)
        d.block = blk
        ids.append(sv.submit(d, np.ascontiguousarray(P.b), x, prm))
    done = {}
    for _ in range(1000):
        sv.run(16)
        for rid, r in sv.poll():
            done[rid] = r
        if len(done) == len(ids):
            break
    sv.close()
    assert len(done) == len(ids)
    for rid, (P, blk), x in zip(ids, probs, xs):
        assert done[rid].status == aar.OK
        assert oracle.Operator(P).rel_residual(P.b, x) <= 1e-8 * 1.0001
