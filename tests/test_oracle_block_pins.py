"""Pins of the oracle's block-Jacobi preconditioner (row f4: the block Jacobi of Sec. 3.2/3.3
with exact block solves) against what the mathematics fixes (no GPU): a dense block-diagonal
inverse built from the dense operator, the closed form of the 2 x 2 x 2 block (cube-graph
eigenbasis), the 1 x 1 x 1 case (Jacobi), block-preconditioned GMRES (Anderson with complete
history minimises over the same Krylov space) and a dense LU solve."""
import itertools

import numpy as np
import pytest

import oracle
import workloads
from tests.dense import block_diagonal_inverse, gmres_iterate, stencil_dense


def prob(nx, ny, nz, r, seed, shift=0.3, periodic=False, h=1.0):
    b = workloads.uniform_rhs(nx * ny * nz, seed)
    return workloads.StencilProblem(nx, ny, nz, r, workloads.stencil_weights(r), h, shift, b, periodic=periodic)


def test_block1_is_jacobi():
    P = prob(6, 4, 8, 2, seed=1)
    op = oracle.Operator(P)
    v = workloads.rng(2).standard_normal(P.n)
    assert np.array_equal(op.block_apply(v, 1), v / op.diag())


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("r,bs,shape", [(1, 2, (6, 4, 8)), (3, 2, (8, 8, 6)), (2, 4, (8, 4, 8)), (3, 2, (2, 4, 6))])
def test_block_apply_matches_dense_block_diagonal(r, bs, shape, periodic):
    # includes a periodic axis of length 2 < 2r + 1 (wrapped taps inside the block add up)
    P = prob(*shape, r, seed=3, periodic=periodic, h=0.8)
    A = stencil_dense(P)
    Minv = block_diagonal_inverse(A, P.nx, P.ny, P.nz, bs)
    v = workloads.rng(4).standard_normal(P.n)
    ref = Minv @ v
    got = oracle.Operator(P).block_apply(v, bs)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("r,periodic", [(1, False), (3, True), (6, False)])
def test_2cube_block_closed_form(r, periodic):
    # a 2 x 2 x 2 block of a stencil with axes longer than r + 1 is d I + c1 Q3 (Q3: the cube
    # graph), with d the centre coefficient and c1 the distance-1 weight; its eigenvectors are the
    # Walsh-Hadamard vectors, eigenvalue d + c1 (3 - 2 |s|) for the sign pattern s
    n = 2 * r + 2
    P = prob(n, n, n, r, seed=5, periodic=periodic, h=0.7)
    w, h = P.weights, P.h
    d = -3.0 * w[0] / h ** 2 + P.shift
    c1 = -w[1] / h ** 2
    v = np.zeros(P.n)
    rng = workloads.rng(6)
    X0, Y0, Z0 = 2, 0, 2  # one block
    pts = [((Z0 + dz) * n + (Y0 + dy)) * n + (X0 + dx) for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)]
    v[pts] = rng.standard_normal(8)
    f = oracle.Operator(P).block_apply(v, 2)
    H = np.array([[(-1) ** bin(a & b_).count("1") for b_ in range(8)] for a in range(8)], dtype=float)
    lam = np.array([d + c1 * (3 - 2 * bin(s).count("1")) for s in range(8)])
    ref = H @ ((H @ v[pts]) / lam) / 8.0
    assert np.max(np.abs(f[pts] - ref)) <= 1e-13 * np.max(np.abs(ref))
    others = np.setdiff1d(np.arange(P.n), pts)
    assert np.all(f[others] == 0.0)


@pytest.mark.parametrize("p", [1, 3, 4])
def test_block_preconditioned_complete_history_is_gmres(p):
    # m >= k: the minimised ||f_k - F gamma|| at every Anderson step equals the residual of GMRES
    # left-preconditioned by the block-Jacobi M, of dimension k
    # (steps whose residual has fallen below 1e-5 of the first are left out: there the history's
    # Gram matrix is too ill-conditioned for FP64 and the pseudoinverse's cut takes over)
    P = prob(6, 6, 4, 1, seed=7, shift=0.0)
    A = stencil_dense(P)
    Minv = block_diagonal_inverse(A, 6, 6, 4, 2)
    f0 = np.linalg.norm(Minv @ P.b)
    res = oracle.solve(P, omega=0.6, beta=0.6, m=50, p=p, tol=0.0, max_iter=12, trace_cap=20, block=2)
    checked = 0
    for k, fmin in zip(res.trace["k"], res.trace["fmin"]):
        if k == 0:
            continue
        _, ref = gmres_iterate(A, Minv, P.b, np.zeros(P.n), int(k))
        if ref < 1e-5 * f0:
            continue
        assert abs(fmin - ref) <= 1e-7 * ref + 1e-12, (k, fmin, ref)
        checked += 1
    assert checked >= 2


@pytest.mark.parametrize("periodic,r", [(False, 1), (False, 3), (True, 3)])
def test_block_lu_brute_force(periodic, r):
    P = prob(8, 8, 8, r, seed=8, shift=0.2, periodic=periodic)
    A = stencil_dense(P)
    ref = np.linalg.solve(A, P.b)
    tol = 1e-10
    res = oracle.solve(P, m=7, p=6, tol=tol, block=2)
    assert res.status == oracle.OK
    assert np.linalg.norm(res.x - ref) <= 2 * np.linalg.cond(A) * tol * np.linalg.norm(ref)
    assert oracle.Operator(P).rel_residual(P.b, res.x) <= tol


def test_block_jacobi_needs_fewer_iterations():
    # the reason for the block preconditioner: radius-6 Poisson, 16^3, 2^3 blocks
    P = workloads.poisson_uniform(16, radius=6, seed=9)
    it_j = oracle.solve(P, m=7, p=6, tol=1e-8).iterations
    it_b = oracle.solve(P, m=7, p=6, tol=1e-8, block=2).iterations
    assert it_b < 0.8 * it_j, (it_b, it_j)


def test_block_rejects_indivisible_grids():
    P = prob(6, 5, 4, 1, seed=10)
    with pytest.raises(ValueError):
        oracle.solve(P, block=2)
