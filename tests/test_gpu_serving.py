"""Serving (continuous batching) through the C ABI: results are the same alone and in the mix,
admission never exceeds the memory budget, requests join while others run, and a failing
request does not disturb the others."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1606_08740_gb300 import aar  # noqa: E402

PRM = dict(omega=0.6, beta=0.6, m=7, p=6)


def _req(side, shift, tol, seed):
    P = workloads.poisson_uniform(side, radius=6, seed=seed, shift=shift)
    return P, aar.params(tol=tol, **PRM)


def _drain(sv, ticks=8, limit=100000):
    done = {}
    for _ in range(limit):
        act, wait, _ = sv.run(ticks)
        for rid, res in sv.poll():
            done[rid] = res
        if act == 0 and wait == 0:
            return done
    raise AssertionError("server did not drain")


def test_results_same_alone_and_in_mix():
    specs = [(24, 0.0, 1e-8, 1), (32, 0.7, 1e-6, 2), (40, 0.0, 1e-10, 3), (48, 1.3, 1e-8, 4),
             (24, 0.2, 1e-10, 5), (36, 0.0, 1e-8, 6)]
    reqs = [_req(*s) for s in specs]
    sv = aar.Server(6, aar.MIXED, budget_bytes=8 << 30, max_active=16)
    xs = [np.empty(P.n) for P, _ in reqs]
    ids = [sv.submit(aar.desc_of(P), P.b, x, prm) for (P, prm), x in zip(reqs, xs)]
    done = _drain(sv)
    sv.close()
    for (P, prm), x, rid, (side, shift, tol, _) in zip(reqs, xs, ids, specs):
        assert done[rid].status == aar.OK
        assert oracle.Operator(P).rel_residual(P.b, x) <= tol * 1.0001
    for i in [0, 2, 3]:
        P, prm = reqs[i]
        alone = aar.Server(6, aar.MIXED, budget_bytes=8 << 30, max_active=4)
        xa = np.empty(P.n)
        alone.submit(aar.desc_of(P), P.b, xa, prm)
        _drain(alone)
        alone.close()
        assert np.array_equal(xa, xs[i])
        xd = torch.empty(P.n, dtype=torch.float64, device="cuda:0")
        with aar.Solver.stencil(aar.desc_of(P), aar.MIXED) as s:
            s.solve(torch.from_numpy(P.b).cuda(), xd, prm=prm)
        assert np.array_equal(xd.cpu().numpy(), xs[i])


def test_mixed_periods_run_full_ticks_with_the_same_results():
    # requests with different Anderson periods: the rounds fall back to full ticks (every kernel
    # every tick); each result still equals its own single solve bit for bit, and a p = 6 request
    # gives the same x whether it shares the server with a p = 4 one or not
    specs = [(28, 0.3, 1e-8, 11, 6), (32, 0.0, 1e-8, 12, 4), (20, 0.9, 1e-10, 13, 5)]
    sv = aar.Server(6, aar.MIXED, budget_bytes=8 << 30, max_active=8)
    reqs, xs, ids = [], [], []
    for side, shift, tol, seed, p in specs:
        P = workloads.poisson_uniform(side, radius=6, seed=seed, shift=shift)
        prm = aar.params(tol=tol, **dict(PRM, p=p))
        x = np.empty(P.n)
        ids.append(sv.submit(aar.desc_of(P), P.b, x, prm))
        reqs.append((P, prm))
        xs.append(x)
    done = _drain(sv, ticks=5)
    sv.close()
    for (P, prm), x, rid in zip(reqs, xs, ids):
        assert done[rid].status == aar.OK
        xd = torch.empty(P.n, dtype=torch.float64, device="cuda:0")
        with aar.Solver.stencil(aar.desc_of(P), aar.MIXED) as s:
            s.solve(torch.from_numpy(P.b).cuda(), xd, prm=prm)
        assert np.array_equal(xd.cpu().numpy(), x)


def test_admission_respects_budget_and_fifo():
    reqs = [_req(32, 0.5, 1e-8, 10 + i) for i in range(6)]
    one = 2 * 8 * 32 ** 3 * 4 + 32 ** 3 * (8 + 8 + 4)  # ring + b + x64 + rhs32, N = 32^3 (multiple of 64)
    sv = aar.Server(6, aar.MIXED, budget_bytes=2 * one + one // 2, max_active=16)
    xs = [np.empty(P.n) for P, _ in reqs]
    ids = [sv.submit(aar.desc_of(P), P.b, x, prm) for (P, prm), x in zip(reqs, xs)]
    order = []
    for _ in range(100000):
        act, wait, used = sv.run(4)
        assert act <= 2 and used <= 2 * one + one // 2
        order += [rid for rid, res in sv.poll()]
        if act == 0 and wait == 0:
            break
    sv.close()
    assert sorted(order) == sorted(ids)


def test_request_joins_while_others_run_and_failure_is_isolated():
    big, pb = _req(64, 0.0, 1e-10, 20)
    small, ps = _req(24, 1.0, 1e-6, 21)
    bad, pbad = _req(24, 0.0, 1e-8, 22)
    bad.b = bad.b.copy()
    bad.b[11] = np.nan
    sv = aar.Server(6, aar.MIXED, budget_bytes=8 << 30, max_active=8)
    xb, xs_, xbad = np.empty(big.n), np.empty(small.n), np.empty(bad.n)
    id_big = sv.submit(aar.desc_of(big), big.b, xb, pb)
    sv.run(8)
    id_small = sv.submit(aar.desc_of(small), small.b, xs_, ps)
    id_bad = sv.submit(aar.desc_of(bad), bad.b, xbad, pbad)
    done = {}
    overlapped = False
    for _ in range(100000):
        act, wait, _ = sv.run(8)
        overlapped = overlapped or act >= 2  # the big solve and the small one resident together
        for rid, res in sv.poll():
            done[rid] = (res, id_big in done)
        if act == 0 and wait == 0:
            break
    sv.close()
    assert overlapped
    assert done[id_small][0].status == aar.OK and not done[id_small][1]  # finished while the big one ran
    assert done[id_bad][0].status == aar.ERR_BREAKDOWN
    assert done[id_big][0].status == aar.OK
    assert oracle.Operator(big).rel_residual(big.b, xb) <= 1e-10 * 1.0001
