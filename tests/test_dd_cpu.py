"""Domain decomposition (Sec. 3.2/3.3: subdomains, a halo exchange per sweep, one global reduction
per Anderson step) on CPU gloo ranks, no GPU.

The library runs a slab's iteration on its GPU and calls back for the two exchanges; what runs on
the host is the slab plan (paper_1606_08740_gb300.dd.slab_bounds / neighbours) and the
torch.distributed communication (TorchDistComm). These tests run both on 2 and 3 gloo ranks:

* the plan covers the grid with balanced slabs of at least r planes, and names the neighbours
  (periodic grids wrap; a single slab is its own neighbour);
* the halo exchange delivers the neighbours' boundary planes (zeros stay at Dirichlet ends) and
  the sum over ranks gives every rank the same totals;
* the decomposed iteration, written here step by step with numpy in the library's order (halo
  exchange, local sweep, at an Anderson step one packed reduction of ||b - A x_k||^2, F^T F and
  F^T f_k, then the same pseudoinverse on every rank), reproduces the single-domain oracle: the
  same iterate at a fixed iteration count and the same stopping iteration.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1606_08740_gb300 import dd  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


# ------------------------------------------------------------------------------------ the plan

@pytest.mark.parametrize("nz,world,radius", [(32, 2, 1), (33, 4, 6), (17, 3, 3), (6, 6, 1), (40, 1, 6)])
def test_slabs_cover_the_grid_balanced(nz, world, radius):
    b = [dd.slab_bounds(nz, world, r, radius) for r in range(world)]
    assert b[0][0] == 0 and b[-1][1] == nz
    assert all(b[i][1] == b[i + 1][0] for i in range(world - 1))
    sizes = [hi - lo for lo, hi in b]
    assert max(sizes) - min(sizes) <= 1 and min(sizes) >= radius


def test_slab_plan_rejects_slabs_thinner_than_the_stencil():
    with pytest.raises(ValueError):
        dd.slab_bounds(10, 4, 0, radius=3)
    with pytest.raises(ValueError):
        dd.slab_bounds(10, 2, 2)


def test_neighbours():
    assert dd.neighbours(0, 3, False) == (None, 1)
    assert dd.neighbours(2, 3, False) == (1, None)
    assert dd.neighbours(0, 3, True) == (2, 1)
    assert dd.neighbours(2, 3, True) == (1, 0)
    assert dd.neighbours(0, 1, True) == (0, 0) and dd.neighbours(0, 1, False) == (None, None)


# ------------------------------------------------------------- a slab's arithmetic, in numpy

def _shift(a, k, axis, periodic):
    """b[..., i, ...] = a[..., i + k, ...] along `axis`; zero beyond the ends unless periodic."""
    if periodic:
        return np.roll(a, -k, axis=axis)
    out = np.zeros_like(a)
    n = a.shape[axis]
    if abs(k) < n:
        src = [slice(None)] * a.ndim
        dst = [slice(None)] * a.ndim
        if k > 0:
            src[axis], dst[axis] = slice(k, n), slice(0, n - k)
        else:
            src[axis], dst[axis] = slice(0, n + k), slice(-k, n)
        out[tuple(dst)] = a[tuple(src)]
    return out


def slab_apply(P, xs, glo, ghi):
    """A x on a slab (planes, ny, nx) with the r ghost planes below / above it: the stencil's
    definition, A = -(1/h^2) sum over axes of the 1-D weights + shift I."""
    r = P.radius
    w = np.asarray(P.weights, dtype=np.float64)
    ih2 = 1.0 / (P.h * P.h)
    ext = np.concatenate([glo, xs, ghi], axis=0)  # planes -r .. nzl + r - 1
    nzl = xs.shape[0]
    y = (-3.0 * w[0] * ih2 + P.shift) * xs
    for k in range(1, r + 1):
        s = ext[r - k:r - k + nzl] + ext[r + k:r + k + nzl]
        for axis in (1, 2):
            s = s + _shift(xs, k, axis, P.periodic) + _shift(xs, -k, axis, P.periodic)
        y = y + (-w[k] * ih2) * s
    return y


def _pinv_solve(G, g):
    """Moore-Penrose solve with the cut c 2^-52 lambda_max (Sec. 3.2's pseudoinverse)."""
    c = len(g)
    lam, V = np.linalg.eigh(G)
    lmax = lam.max() if c else 0.0
    keep = lam > c * 2.0 ** -52 * lmax
    return V[:, keep] @ ((V[:, keep].T @ g) / lam[keep])


def decomposed_aar(P, comm, z_lo, z_hi, omega, beta, m, p, tol, max_iter):
    """This rank's slab of the AAR iteration (Eq. 2-6), one exchange per sweep and one packed sum
    per Anderson step, as the library schedules them. Returns (x slab, iterations, status)."""
    nx, ny, r = P.nx, P.ny, P.radius
    b = P.b.reshape(P.nz, ny, nx)[z_lo:z_hi].copy()
    nzl = z_hi - z_lo
    dinv = 1.0 / (-3.0 * P.weights[0] / (P.h * P.h) + P.shift)
    tb = torch.tensor([float(np.sum(b * b))], dtype=torch.float64)
    comm.sum_(tb)
    nb = float(np.sqrt(tb[0]))
    x = np.zeros_like(b)
    xs, fs = [], []  # raw iterates and residuals of the history window
    k = 0
    while True:
        glo = torch.zeros((r, ny, nx), dtype=torch.float64)
        ghi = torch.zeros((r, ny, nx), dtype=torch.float64)
        comm.exchange(torch.from_numpy(x[:r].copy()), torch.from_numpy(x[nzl - r:].copy()), glo, ghi)
        res = b - slab_apply(P, x, glo.numpy(), ghi.numpy())
        f = dinv * res
        xs.append(x.copy())
        fs.append(f.copy())
        xs, fs = xs[-(m + 1):], fs[-(m + 1):]
        if (k + 1) % p != 0:
            x_next = x + omega * f
        else:
            c = min(k, m)
            dX = [(xs[-c + i] - xs[-c - 1 + i]).ravel() for i in range(c)]
            dF = [(fs[-c + i] - fs[-c - 1 + i]).ravel() for i in range(c)]
            packed = [float(np.sum(res * res))]
            packed += [float(dF[i] @ dF[j]) for i in range(c) for j in range(i, c)]
            packed += [float(dF[i] @ f.ravel()) for i in range(c)]
            t = torch.tensor(packed, dtype=torch.float64)
            comm.sum_(t)  # the one reduction of this Anderson step
            t = t.numpy()
            rk = float(np.sqrt(t[0])) / nb
            if rk <= tol:
                return x, k, 0
            G = np.zeros((c, c))
            e = 1
            for i in range(c):
                for j in range(i, c):
                    G[i, j] = G[j, i] = t[e]
                    e += 1
            g = t[e:e + c]
            gam = _pinv_solve(G, g) if c else np.zeros(0)
            upd = beta * f.ravel()
            for i in range(c):
                upd = upd - gam[i] * (dX[i] + beta * dF[i])
            x_next = x + upd.reshape(x.shape)
        x = x_next
        k += 1
        if k >= max_iter:
            return x, k, 1


def _rank_main(rank, world, port, out_dir, case):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import workloads
    from paper_1606_08740_gb300 import dd as ddm

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        P = _problem(workloads, case)
        comm = ddm.TorchDistComm(P.periodic)
        z_lo, z_hi = ddm.slab_bounds(P.nz, world, rank, P.radius)
        if case["kind"] == "exchange":
            g = np.arange(P.nz * P.ny * P.nx, dtype=np.float64).reshape(P.nz, P.ny, P.nx) + 1.0
            xs = g[z_lo:z_hi]
            r = P.radius
            glo = torch.zeros((r, P.ny, P.nx), dtype=torch.float64)
            ghi = torch.zeros((r, P.ny, P.nx), dtype=torch.float64)
            comm.exchange(torch.from_numpy(xs[:r].copy()), torch.from_numpy(xs[-r:].copy()), glo, ghi)
            t = torch.tensor([rank + 1.0, 10.0 * rank], dtype=torch.float64)
            comm.sum_(t)
            np.savez(os.path.join(out_dir, f"r{rank}.npz"), glo=glo.numpy(), ghi=ghi.numpy(), t=t.numpy(),
                     z=np.array([z_lo, z_hi]))
        else:
            x, k, st = decomposed_aar(P, comm, z_lo, z_hi, **case["prm"])
            np.savez(os.path.join(out_dir, f"r{rank}.npz"), x=x, k=np.array(k), st=np.array(st),
                     z=np.array([z_lo, z_hi]))
    finally:
        dist.destroy_process_group()


def _problem(workloads, case):
    if case["periodic"]:
        b = workloads.uniform_rhs(case["n"] ** 3, case["seed"])
        return workloads.StencilProblem(case["n"], case["n"], case["n"], case["r"], workloads.stencil_weights(case["r"]),
                                        1.0, case["shift"], b - b.mean(), periodic=True)
    return workloads.poisson_uniform(case["n"], radius=case["r"], seed=case["seed"], shift=case["shift"])


def _run(world, case, tmp_path):
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path), case)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    return [dict(np.load(os.path.join(str(tmp_path), f"r{r}.npz"))) for r in range(world)]


@pytest.mark.parametrize("world,periodic", [(2, False), (3, True), (2, True)])
def test_halo_exchange_and_sum_over_gloo_ranks(world, periodic, tmp_path):
    import workloads

    case = dict(kind="exchange", n=12, r=3, seed=1, shift=0.2, periodic=periodic)
    out = _run(world, case, tmp_path)
    P = _problem(workloads, case)
    g = np.arange(P.nz * P.ny * P.nx, dtype=np.float64).reshape(P.nz, P.ny, P.nx) + 1.0
    r = P.radius
    for rank, o in enumerate(out):
        z_lo, z_hi = o["z"]
        below = [(z_lo - r + i) for i in range(r)]
        above = [(z_hi + i) for i in range(r)]
        for got, planes in ((o["glo"], below), (o["ghi"], above)):
            for i, z in enumerate(planes):
                if 0 <= z < P.nz or periodic:
                    np.testing.assert_array_equal(got[i], g[z % P.nz])
                else:
                    assert not got[i].any()  # zero Dirichlet ghosts at the grid's ends
        np.testing.assert_array_equal(o["t"], [sum(q + 1.0 for q in range(world)), 10.0 * sum(range(world))])


@pytest.mark.parametrize("world,case", [
    (2, dict(n=14, r=3, seed=21, shift=0.1, periodic=False)),
    (3, dict(n=13, r=1, seed=22, shift=0.0, periodic=False)),
    (2, dict(n=12, r=2, seed=23, shift=0.3, periodic=True)),
    (3, dict(n=18, r=6, seed=24, shift=0.2, periodic=False)),
], ids=["r3-2ranks", "7pt-3ranks", "r2-periodic-2ranks", "r6-3ranks"])
def test_decomposed_iteration_matches_the_single_domain_oracle(world, case, tmp_path):
    import oracle
    import workloads

    P = _problem(workloads, case)
    prm = dict(omega=0.6, beta=0.6, m=7, p=6)
    # a fixed iteration count: the iterate after two Anderson cycles and a Richardson step
    out = _run(world, dict(case, kind="solve", prm=dict(prm, tol=0.0, max_iter=13)), tmp_path)
    x = np.concatenate([o["x"] for o in out], axis=0).ravel()
    ref = oracle.solve(P, tol=0.0, max_iter=13, **prm)
    assert all(int(o["k"]) == 13 for o in out)
    assert np.linalg.norm(x - ref.x) <= 1e-12 * np.linalg.norm(ref.x)
    # to convergence: the same stopping iteration on every rank and in the oracle
    out = _run(world, dict(case, kind="solve", prm=dict(prm, tol=1e-10, max_iter=5000)), tmp_path)
    ref = oracle.solve(P, tol=1e-10, max_iter=5000, **prm)
    assert ref.status == oracle.OK
    assert all(int(o["st"]) == 0 and int(o["k"]) == ref.iterations for o in out)
    x = np.concatenate([o["x"] for o in out], axis=0).ravel()
    assert np.linalg.norm(x - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
