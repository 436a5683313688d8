"""Pins of the oracle's complex block-Jacobi preconditioner (the block Jacobi of Sec. 3.2's Helmholtz
runs, with exact block solves, on the operator of Eq. 7) against what the mathematics fixes (no
GPU): the dense block-diagonal inverse of the dense complex operator, the closed form of a
2 x 2 x 2 block (cube-graph eigenbasis with a complex centre coefficient), 1 x 1 x 1 boxes
(complex Jacobi), complex block-preconditioned GMRES (Anderson with complete history minimises
over the same Krylov space) and a dense complex LU solve."""
import numpy as np
import pytest

import oracle
import workloads
from tests.dense import block_diagonal_inverse, gmres_iterate, zstencil_dense


def zprob(nx, ny, nz, r, seed, q=complex(0.4, -0.3), scale=1.0, periodic=True, h=1.0):
    return workloads.complex_uniform(nx, ny, nz, r, seed=seed, h=h, scale=scale, q=q, periodic=periodic)


def test_block1_is_complex_jacobi():
    P = zprob(6, 4, 8, 2, seed=6601)
    op = oracle.ZOperator(P)
    g = workloads.rng(2)
    v = g.standard_normal(P.n) + 1j * g.standard_normal(P.n)
    ref = v / op.diag()  # complex division: C's and numpy's algorithms may differ in the last bit
    assert np.max(np.abs(op.block_apply(v, 1) - ref)) <= 4e-16 * np.max(np.abs(ref))


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("r,bs,shape", [(1, 2, (6, 4, 8)), (3, 2, (8, 8, 6)), (2, 4, (8, 4, 8)), (3, 2, (2, 4, 6))])
def test_block_apply_matches_dense_complex_block_diagonal(r, bs, shape, periodic):
    # includes a periodic axis of length 2 < 2r + 1 (wrapped taps inside the block add up)
    P = zprob(*shape, r, seed=6602, periodic=periodic, h=0.8, scale=0.3)
    A = zstencil_dense(P)
    Minv = block_diagonal_inverse(A, P.nx, P.ny, P.nz, bs)
    g = workloads.rng(4)
    v = g.standard_normal(P.n) + 1j * g.standard_normal(P.n)
    ref = Minv @ v
    got = oracle.ZOperator(P).block_apply(v, bs)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("r,periodic", [(1, False), (3, True), (6, False)])
def test_2cube_complex_block_closed_form(r, periodic):
    # a 2 x 2 x 2 block of Eq. 7's operator (axes longer than r + 1) is d I + c1 Q3 with the complex
    # centre coefficient d = scale (-3 w0 / h^2) + Q and the real distance-1 coupling
    # c1 = -scale w1 / h^2: Walsh-Hadamard eigenvectors, eigenvalue d + c1 (3 - 2 |s|)
    n = 2 * r + 2
    q = complex(-0.135, -0.07)
    P = zprob(n, n, n, r, seed=6603, periodic=periodic, h=0.7, scale=1.0 / (4 * np.pi), q=q)
    w, h = P.weights, P.h
    d = P.scale * (-3.0 * w[0] / h ** 2) + q
    c1 = -P.scale * w[1] / h ** 2
    v = np.zeros(P.n, dtype=np.complex128)
    g = workloads.rng(6)
    X0, Y0, Z0 = 2, 0, 2
    pts = [((Z0 + dz) * n + (Y0 + dy)) * n + (X0 + dx) for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)]
    v[pts] = g.standard_normal(8) + 1j * g.standard_normal(8)
    f = oracle.ZOperator(P).block_apply(v, 2)
    H = np.array([[(-1) ** bin(a & b_).count("1") for b_ in range(8)] for a in range(8)], dtype=float)
    lam = np.array([d + c1 * (3 - 2 * bin(s).count("1")) for s in range(8)])
    ref = H @ ((H @ v[pts]) / lam) / 8.0
    assert np.max(np.abs(f[pts] - ref)) <= 1e-13 * np.max(np.abs(ref))
    others = np.setdiff1d(np.arange(P.n), pts)
    assert np.all(f[others] == 0.0)


@pytest.mark.parametrize("p", [1, 3])
def test_complex_block_preconditioned_complete_history_is_gmres(p):
    # m >= k: the minimised ||f_k - F gamma|| at every Anderson step equals the residual of complex
    # GMRES left-preconditioned by the block-Jacobi M, of dimension k (F^H in Eq. 3)
    P = zprob(6, 6, 4, 1, seed=6604, q=complex(0.2, 0.5))
    A = zstencil_dense(P)
    Minv = block_diagonal_inverse(A, 6, 6, 4, 2)
    f0 = np.linalg.norm(Minv @ P.b)
    res = oracle.zsolve(P, omega=0.6, beta=0.6, m=50, p=p, tol=0.0, max_iter=12, trace_cap=20, block=2)
    checked = 0
    for k, fmin in zip(res.trace["k"], res.trace["fmin"]):
        if k == 0:
            continue
        _, ref = gmres_iterate(A, Minv, P.b, np.zeros(P.n, dtype=np.complex128), int(k))
        if ref < 1e-5 * f0:
            continue
        assert abs(fmin - ref) <= 1e-7 * ref + 1e-12, (k, fmin, ref)
        checked += 1
    assert checked >= 2


@pytest.mark.parametrize("periodic,r", [(True, 3), (False, 1)])
def test_complex_block_lu_brute_force(periodic, r):
    P = zprob(8, 8, 8, r, seed=6605, periodic=periodic, q=complex(0.3, -0.4), scale=0.5)
    A = zstencil_dense(P)
    ref = np.linalg.solve(A, P.b)
    tol = 1e-10
    res = oracle.zsolve(P, m=7, p=6, tol=tol, block=2)
    assert res.status == oracle.OK
    assert np.linalg.norm(res.x - ref) <= 2 * np.linalg.cond(A) * tol * np.linalg.norm(ref)
    assert oracle.ZOperator(P).rel_residual(P.b, res.x) <= tol


def test_complex_block_jacobi_needs_fewer_iterations_on_the_eq7_cell():
    # the reason for the block preconditioner in Sec. 3.2's runs: the Eq. 7 operator of one FCC
    # aluminium cell at a coarse mesh (16^3), 2^3 blocks
    P = workloads.ofdft_helmholtz(1, 7.78 / 16, seed=6000)
    it_j = oracle.zsolve(P, m=7, p=6, tol=1e-6).iterations
    it_b = oracle.zsolve(P, m=7, p=6, tol=1e-6, block=2).iterations
    assert it_b < 0.8 * it_j, (it_b, it_j)


def test_complex_block_rejects_indivisible_grids():
    P = zprob(6, 5, 4, 1, seed=6606)
    with pytest.raises(ValueError):
        oracle.zsolve(P, block=2)
