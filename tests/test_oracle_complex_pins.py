"""Pins of the complex-valued oracle (Eq. 1-6 over C, the operator of Eq. 7) against what the
mathematics fixes (no GPU): a dense Kronecker-form matrix, the closed-form Fourier eigenvalues of
the periodic operator, numpy's complex least squares and pseudoinverse, the real oracle on real
data, brute-force complex GMRES (Anderson with complete history minimises over the same Krylov
space), Jacobi-Richardson for m = 0, and a dense complex LU solve.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from tests.dense import gmres_iterate, zstencil_dense


def zprob(nx, ny, nz, r, seed, q=complex(0.3, 0.2), scale=1.0, h=1.0, periodic=True):
    return workloads.complex_uniform(nx, ny, nz, r, seed=seed, h=h, scale=scale, q=q, periodic=periodic)


def crand(g, *shape):
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


# ---------------------------------------------------------------- operator

@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("r,shape", [(1, (5, 4, 3)), (3, (7, 6, 5)), (3, (4, 9, 3))])
def test_zapply_matches_dense(r, shape, periodic):
    P = zprob(*shape, r, seed=11, q=complex(-0.135, -0.0702), scale=1.0 / (4.0 * math.pi), h=0.486,
              periodic=periodic)
    A = zstencil_dense(P)
    x = crand(np.random.default_rng(3), P.n)
    y = oracle.ZOperator(P).apply(x)
    assert np.max(np.abs(y - A @ x)) <= 1e-13 * np.max(np.abs(A @ x))
    # Jacobi D: the stencil's centre coefficient (on a periodic axis shorter than 2r + 1 the
    # matrix diagonal also collects wrapped taps; D stays the centre coefficient, as for real data)
    centre = P.scale * (-3.0 * P.weights[0] / P.h ** 2) + P.q
    assert abs(oracle.ZOperator(P).diag() - centre) <= 1e-15 * abs(centre)
    if min(shape) >= 2 * r + 1 or not periodic:
        assert abs(centre - A[0, 0]) <= 1e-14 * abs(centre)
    idx = [0, 7, P.n - 1]
    assert np.max(np.abs(oracle.ZOperator(P).apply_at(x, idx) - (A @ x)[idx])) <= 1e-13 * np.max(np.abs(A @ x))


@pytest.mark.parametrize("r", [1, 3])
def test_zperiodic_fourier_mode_eigenvalue(r):
    # periodic: e^{i theta . j} is an eigenvector with eigenvalue
    # scale (-1/h^2) sum_axes (w0 + 2 sum_k w_k cos(k theta_axis)) + q
    nx, ny, nz = 9, 8, 7
    h, scale, q = 0.3, 1.0 / (4.0 * math.pi), complex(-0.134992, -0.070225)
    P = zprob(nx, ny, nz, r, seed=1, q=q, scale=scale, h=h)
    w = P.weights
    a, b, c = 2, 3, 1
    th = [2 * math.pi * a / nx, 2 * math.pi * b / ny, 2 * math.pi * c / nz]
    ix = np.arange(nx)[None, None, :]
    iy = np.arange(ny)[None, :, None]
    iz = np.arange(nz)[:, None, None]
    x = np.exp(1j * (th[0] * ix + th[1] * iy + th[2] * iz)).reshape(-1)
    lam = scale * (-1.0 / h ** 2) * sum(w[0] + 2 * sum(w[k] * math.cos(k * t) for k in range(1, r + 1)) for t in th) + q
    y = oracle.ZOperator(P).apply(x)
    assert np.max(np.abs(y - lam * x)) <= 1e-12 * abs(lam)


# ---------------------------------------------------------------- pseudoinverse

def test_zpinv_full_rank_is_least_squares():
    g = np.random.default_rng(5)
    F = crand(g, 40, 6)
    f = crand(g, 40)
    G = F.conj().T @ F
    gamma, rank = oracle.zpinv_solve(G, F.conj().T @ f)
    ref, *_ = np.linalg.lstsq(F, f, rcond=None)
    assert rank == 6
    assert np.max(np.abs(gamma - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_zpinv_rank_deficient_is_minimum_norm():
    # a column that is a complex multiple of another: rank c - 1, the minimum-norm solution
    g = np.random.default_rng(6)
    F = crand(g, 30, 5)
    F[:, 3] = (0.3 + 0.7j) * F[:, 1]
    f = crand(g, 30)
    G = F.conj().T @ F
    gvec = F.conj().T @ f
    gamma, rank = oracle.zpinv_solve(G, gvec)
    assert rank == 4
    ref = np.linalg.pinv(F) @ f
    assert np.max(np.abs(gamma - ref)) <= 1e-9 * np.max(np.abs(ref))
    assert np.max(np.abs(gamma - np.linalg.pinv(G, hermitian=True) @ gvec)) <= 1e-9 * np.max(np.abs(ref))


def test_zpinv_zero_matrix_gives_zero():
    gamma, rank = oracle.zpinv_solve(np.zeros((3, 3), complex), np.ones(3, complex))
    assert rank == 0 and np.all(gamma == 0)


# ---------------------------------------------------------------- the solve

@pytest.mark.parametrize("m,p", [(5, 4), (9, 8), (3, 1)])
def test_zsolve_on_real_data_equals_real_oracle(m, p):
    # q, b, omega, beta real: the complex loop takes the real loop's steps (the Hermitian Gram is
    # the real Gram, its 2c x 2c form two copies of it)
    Z = zprob(8, 7, 6, 3, seed=21, q=0.4, scale=1.0, periodic=False)
    Z.b = Z.b.real.astype(np.complex128)
    R = workloads.StencilProblem(8, 7, 6, 3, Z.weights, 1.0, 0.4, Z.b.real.copy())
    rz = oracle.zsolve(Z, 0.6, 0.6, m=m, p=p, tol=1e-10)
    rr = oracle.solve(R, 0.6, 0.6, m=m, p=p, tol=1e-10)
    assert rz.status == rr.status == oracle.OK
    assert rz.iterations == rr.iterations
    assert np.max(np.abs(rz.x.imag)) == 0.0
    assert np.linalg.norm(rz.x.real - rr.x) <= 1e-12 * np.linalg.norm(rr.x)


@pytest.mark.parametrize("omega,beta", [(0.6, 0.6), (0.5 + 0.2j, 0.7 - 0.3j)])
def test_zm0_is_jacobi_richardson(omega, beta):
    P = zprob(5, 6, 4, 1, seed=31, q=complex(0.5, -0.4))
    op = oracle.ZOperator(P)
    A = zstencil_dense(P)
    dinv = 1.0 / A[0, 0]
    x = np.zeros(P.n, complex)
    for k in range(17):
        x = x + (beta if (k + 1) % 4 == 0 else omega) * dinv * (P.b - A @ x)
    res = oracle.zsolve(P, omega, beta, m=0, p=4, tol=0.0, max_iter=17, op=op)
    assert res.status == oracle.NOT_CONVERGED and res.iterations == 17
    assert np.linalg.norm(res.x - x) <= 1e-13 * np.linalg.norm(x)


@pytest.mark.parametrize("p,beta", [(3, 0.6), (5, 0.7 - 0.3j)])
def test_zfirst_anderson_step_is_gmres(p, beta):
    # x_p = xbar + beta f(xbar), xbar the complex GMRES iterate of dimension p - 1
    P = zprob(4, 4, 3, 1, seed=41, q=complex(0.2, 0.5))
    A = zstencil_dense(P)
    dinv = np.full(P.n, 1.0 / A[0, 0])
    res = oracle.zsolve(P, omega=0.45 + 0.1j, beta=beta, m=20, p=p, tol=0.0, max_iter=p, trace_cap=4)
    xbar, fnorm = gmres_iterate(A, dinv, P.b, np.zeros(P.n, complex), p - 1)
    expect = xbar + beta * dinv * (P.b - A @ xbar)
    assert np.linalg.norm(res.x - expect) <= 1e-10 * np.linalg.norm(expect)
    assert abs(res.trace["fmin"][0] - fnorm) <= 1e-9 * fnorm


@pytest.mark.parametrize("p,omega", [(1, 0.6), (3, 0.6 + 0.3j), (4, 1.1)])
def test_zcomplete_history_minimises_over_krylov(p, omega):
    # m >= k: the minimised ||f_k - F gamma|| at every Anderson step equals the complex GMRES
    # residual of dimension k (a plain transpose in place of F^H fails this)
    P = zprob(4, 3, 3, 1, seed=51, q=complex(-0.3, 0.4))
    A = zstencil_dense(P)
    dinv = np.full(P.n, 1.0 / A[0, 0])
    res = oracle.zsolve(P, omega=omega, beta=0.6, m=50, p=p, tol=0.0, max_iter=12, trace_cap=20)
    for k, fmin in zip(res.trace["k"], res.trace["fmin"]):
        if k == 0:
            continue
        _, ref = gmres_iterate(A, dinv, P.b, np.zeros(P.n, complex), int(k))
        assert abs(fmin - ref) <= 1e-7 * ref + 1e-12, (k, fmin, ref)


@pytest.mark.parametrize("periodic", [True, False])
def test_zdense_lu_brute_force(periodic):
    # Eq. 7's constants on a small periodic (or Dirichlet) grid: the AAR solution against a dense LU
    q, scale = workloads.OFDFT_Q, 1.0 / (4.0 * math.pi)
    P = zprob(6, 6, 6, 3, seed=61, q=q, scale=scale, h=0.486, periodic=periodic)
    A = zstencil_dense(P)
    ref = np.linalg.solve(A, P.b)
    tol = 1e-10
    res = oracle.zsolve(P, m=9, p=8, tol=tol)
    assert res.status == oracle.OK
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(res.x - ref) <= 2 * kappa * tol * np.linalg.norm(ref)
    assert oracle.ZOperator(P).rel_residual(P.b, res.x) <= tol


def test_ofdft_density_carries_the_valence_charge():
    # the stand-in density integrates to 3 electrons per atom, 4 atoms per FCC cell
    for cells, n in [(1, 36), (2, 40)]:
        rho = workloads.ofdft_density(cells, n, seed=6000)
        hh = cells * 7.78 / n
        assert abs(rho.sum() * hh ** 3 - 12.0 * cells ** 3) <= 1e-3 * 12.0 * cells ** 3
        assert rho.min() >= 0.0


def test_zzero_rhs_and_max_iter():
    P = zprob(4, 4, 4, 1, seed=71)
    P.b = np.zeros(P.n, complex)
    res = oracle.zsolve(P)
    assert res.status == oracle.OK and res.iterations == 0 and np.all(res.x == 0)
    P = zprob(4, 4, 4, 1, seed=72)
    res = oracle.zsolve(P, tol=0.0, max_iter=5)
    assert res.status == oracle.NOT_CONVERGED and res.iterations == 5


@pytest.mark.parametrize("r", [1, 3])
def test_zsolve_single_fourier_mode_closed_form(r):
    # periodic Eq. 7 operator, b = e^{i theta . j}: the exact solution is b / lambda(theta), and the
    # AAR solve must reach it within kappa-free accuracy (A is normal: ||x - x*|| <= ||r|| / |lambda|)
    nx, ny, nz = 12, 10, 8
    h, scale, q = 0.486, 1.0 / (4.0 * math.pi), workloads.OFDFT_Q
    P = zprob(nx, ny, nz, r, seed=1, q=q, scale=scale, h=h)
    w = P.weights
    a, b, c = 1, 2, 3
    th = [2 * math.pi * a / nx, 2 * math.pi * b / ny, 2 * math.pi * c / nz]
    ix = np.arange(nx)[None, None, :]
    iy = np.arange(ny)[None, :, None]
    iz = np.arange(nz)[:, None, None]
    P.b = np.exp(1j * (th[0] * ix + th[1] * iy + th[2] * iz)).reshape(-1)
    lam = scale * (-1.0 / h ** 2) * sum(w[0] + 2 * sum(w[k] * math.cos(k * t) for k in range(1, r + 1)) for t in th) + q
    exact = P.b / lam
    tol = 1e-12
    res = oracle.zsolve(P, m=9, p=8, tol=tol)
    assert res.status == oracle.OK
    # one mode: Richardson and Anderson act on it alone, so the residual bound gives the error
    assert np.linalg.norm(res.x - exact) <= 2 * tol * np.linalg.norm(P.b) / abs(lam)
