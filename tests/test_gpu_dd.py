"""The domain-decomposed solve (include/aar_dd.h) through the C ABI on one GPU: 2 to 4 slabs of
one grid, each with its own handle and stream, driven by one host thread per slab and exchanging
through paper_1606_08740_gb300.dd.LocalGroup (a host barrier, then device copies; no kernel waits
on another). The gathered iterate must match the single-domain FP64 oracle at a fixed iteration
count and stop at the oracle's iteration, as the single-GPU FP64 solve does."""
import threading

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1606_08740_gb300 import aar, dd  # noqa: E402


def _periodic(n, r, seed, shift):
    b = workloads.uniform_rhs(n ** 3, seed)
    return workloads.StencilProblem(n, n, n, r, workloads.stencil_weights(r), 1.0, shift, b - b.mean(), periodic=True)


def run_slabs(P, world, prm):
    """Solve P split into `world` slabs; returns (gathered x, per-slab results, callback errors)."""
    group = dd.LocalGroup(world, P.periodic, timeout=60.0)
    bg = P.b.reshape(P.nz, P.ny, P.nx)
    out = [None] * world

    def run(rank):
        z_lo, z_hi = dd.slab_bounds(P.nz, world, rank, P.radius)
        stream = torch.cuda.Stream()
        b = torch.from_numpy(bg[z_lo:z_hi].ravel().copy()).cuda()
        x = torch.empty_like(b)
        with aar.DDSolver(aar.desc_of(P), z_lo, z_hi, stream=stream) as s:
            res = s.solve(b, x, group.comm(rank), prm=aar.params(**prm), raise_on_error=False)
            out[rank] = (res, x.cpu().numpy(), list(s.errors))

    th = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    assert all(o is not None for o in out)
    return np.concatenate([o[1] for o in out]), [o[0] for o in out], [e for o in out for e in o[2]]


CASES = [
    (2, lambda: workloads.poisson_uniform(32, radius=1, seed=0)),
    (3, lambda: workloads.poisson_uniform(30, radius=6, seed=31, shift=0.1, ny=27, nz=20)),
    (4, lambda: workloads.poisson_sine_modes(36, radius=3, seed=1000)),
    (2, lambda: _periodic(24, 3, 32, 0.2)),
    (3, lambda: _periodic(21, 2, 33, 0.3)),
]


@pytest.mark.parametrize("world,make", CASES, ids=["7pt-2slabs", "r6-ragged-3slabs", "r3-sines-4slabs",
                                                   "r3-periodic-2slabs", "r2-periodic-3slabs"])
def test_slabs_match_the_single_domain_oracle(world, make):
    P = make()
    prm = dict(omega=0.6, beta=0.6, m=7, p=6)
    # fixed iteration count: two Anderson cycles and one Richardson step
    x, res, errs = run_slabs(P, world, dict(prm, tol=0.0, max_iter=13))
    assert not errs, errs
    assert all(r.status == aar.NOT_CONVERGED and r.iterations == 13 for r in res)
    ref = oracle.solve(P, tol=0.0, max_iter=13, **prm)
    # the parity bar; the sine-mode right-hand side (8 modes) makes the Gram matrix nearly singular
    # once the history outgrows the modes, so rounding differences of the sums reach 1e-11 there
    assert np.linalg.norm(x - ref.x) <= 1e-10 * np.linalg.norm(ref.x)
    # to convergence at the parity tolerance: the oracle's stopping iteration, on every slab
    x, res, errs = run_slabs(P, world, dict(prm, tol=1e-10, max_iter=20000))
    assert not errs, errs
    ref = oracle.solve(P, tol=1e-10, max_iter=20000, **prm)
    assert ref.status == oracle.OK
    assert all(r.status == aar.OK and r.iterations == ref.iterations for r in res), (res, ref.iterations)
    assert all(r.rel_residual == res[0].rel_residual for r in res)  # the same reduced values everywhere
    assert np.linalg.norm(x - ref.x) <= 1e-9 * np.linalg.norm(ref.x)


def test_failing_callback_ends_the_solve_with_a_comm_error():
    # a transport failure is made on the host (the allreduce callback raises): the solve returns
    # AAR_ERR_COMM and the handle stays usable
    P = workloads.poisson_uniform(16, radius=1, seed=3)

    class Broken:
        def halo(self, *a):
            pass

        def allreduce(self, *a):
            raise RuntimeError("peer lost")

    b = torch.from_numpy(P.b).cuda()
    x = torch.empty_like(b)
    with aar.DDSolver(aar.desc_of(P), 0, P.nz) as s:
        r = s.solve(b, x, Broken(), raise_on_error=False)
        assert r.status == aar.ERR_COMM and isinstance(s.errors[0], RuntimeError)
        # one slab holding the whole grid with a working (single-rank) exchange: the FP64 solve
        r = s.solve(b, x, dd.LocalGroup(1, False).comm(0), prm=aar.params(m=7, p=6, tol=1e-10))
    ref = oracle.solve(P, m=7, p=6, tol=1e-10)
    assert r.status == aar.OK and r.iterations == ref.iterations
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-9 * np.linalg.norm(ref.x)


def test_invalid_slabs_are_rejected():
    d = aar.desc_of(workloads.poisson_uniform(16, radius=3, seed=0))
    for lo, hi in [(-1, 8), (0, 17), (5, 7), (8, 8)]:  # outside the grid, or thinner than the radius
        with pytest.raises(aar.AARError) as e:
            aar.DDSolver(d, lo, hi)
        assert e.value.status == aar.ERR_INVALID_ARG
