"""The allocation-free residual check against the allocating one, through the C ABI.

aar_rel_residual_noalloc serves callers that cannot allocate device memory inside a call (a
latency-critical loop that cannot absorb cudaMalloc's implicit synchronisation, or a process whose
device memory is fully budgeted). It must give the same relative residual as aar_rel_residual, to
rounding, call after call: its scratch is a shared device array that keeps the previous call's
contents, so two calls in a row are checked. This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1606_08740_gb300 import aar  # noqa: E402

TOL = 1e-12  # both are FP64 sums of the same terms in different orders


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


@pytest.mark.parametrize("kind", ["stencil-r6", "stencil-r1", "csr", "stencil-r3-periodic"])
def test_noalloc_matches_allocating_residual_twice(kind):
    if kind == "csr":
        P = workloads.convection_diffusion(21, seed=5)
        s = aar.Solver.csr(_dev(P.row_ptr), _dev(P.col_idx), _dev(P.val))
    elif kind == "stencil-r3-periodic":
        P = workloads.periodic_modes(30, radius=3, seed=5003, shift=0.2)
        s = aar.Solver.stencil(aar.desc_of(P))
    else:
        r = 6 if kind == "stencil-r6" else 1
        P = workloads.poisson_uniform(37, radius=r, seed=3, ny=29, nz=23, shift=0.2)
        s = aar.Solver.stencil(aar.desc_of(P))
    b = _dev(P.b)
    g = workloads.rng(8)
    with s:
        for call in range(2):  # two calls in a row: the second must not see the first's partials
            x = _dev(g.standard_normal(P.n) * (call + 1))
            ref = s.rel_residual(b, x)
            got = s.rel_residual_noalloc(b, x)
            assert abs(got - ref) <= TOL * ref, (call, got, ref)
            # and the oracle's own FP64 residual of the same operator
            orc = oracle.Operator(P).rel_residual(P.b, x.cpu().numpy())
            assert abs(got - orc) <= TOL * orc, (call, got, orc)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    desc = aar.stencil_desc(512, 512, 512, 1, workloads.stencil_weights(1))  # 134M unknowns > 67,108,864
    tiny = torch.zeros(8, dtype=torch.float64, device="cuda:0")
    with aar.Solver.stencil(desc) as s:
        with pytest.raises(aar.AARError) as e:
            s.rel_residual_noalloc(tiny, tiny)
        assert e.value.status == aar.ERR_INVALID_ARG


@pytest.mark.skipif(not torch.cuda.is_available() or torch.cuda.device_count() < 2,
                    reason="needs a second device to make current")
def test_noalloc_rejects_a_call_from_another_device():
    # each device holds its own copy of the scratch array: a call made with a device other than
    # the handle's current would pair the handle's stream with the wrong copy, so it is refused
    P = workloads.poisson_uniform(16, radius=1, seed=3)
    b = _dev(P.b)
    with aar.Solver.stencil(aar.desc_of(P)) as s:
        with torch.cuda.device(1):
            with pytest.raises(aar.AARError) as e:
                s.rel_residual_noalloc(b, b)
        assert e.value.status == aar.ERR_INVALID_ARG
