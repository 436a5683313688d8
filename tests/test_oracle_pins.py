"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: textbook finite-difference
weights, a dense matrix built from the operator's definition, library eigen/least-squares
routines, closed-form solutions of the Dirichlet Laplacian, brute-force left-preconditioned
GMRES (Sec. 2: AAR with complete history minimises over the same Krylov space), a dense LU
solve, and the special cases m = 0 (Jacobi-Richardson) and p = 1 (Anderson-Richardson).
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import workloads
from tests.dense import dense, gmres_iterate, stencil_dense


# ---------------------------------------------------------------- operator pins

FORNBERG = {  # centred second-derivative weights, Fornberg (1988) table, w[0..r]
    1: [Fraction(-2), Fraction(1)],
    2: [Fraction(-5, 2), Fraction(4, 3), Fraction(-1, 12)],
    3: [Fraction(-49, 18), Fraction(3, 2), Fraction(-3, 20), Fraction(1, 90)],
    4: [Fraction(-205, 72), Fraction(8, 5), Fraction(-1, 5), Fraction(8, 315), Fraction(-1, 560)],
}


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_stencil_weights_textbook(r):
    w = workloads.stencil_weights(r)
    assert np.array_equal(w, np.array([float(v) for v in FORNBERG[r]]))


@pytest.mark.parametrize("r", [1, 2, 3, 4, 5, 6])
def test_stencil_weights_exact_on_polynomials(r):
    # sum_k w_|k| k^(2j) = 2 for j == 1, 0 otherwise (j <= r): exact second derivative of x^(2j)
    w = workloads.stencil_weights(r)
    for j in range(0, r + 1):
        s = w[0] * (1.0 if j == 0 else 0.0) + sum(2.0 * w[k] * float(k) ** (2 * j) for k in range(1, r + 1))
        assert abs(s - (2.0 if j == 1 else 0.0)) < 1e-9 * (1 + float(r) ** (2 * j)), (r, j, s)


@pytest.mark.parametrize("r,shape,h,shift", [(1, (5, 6, 7), 1.0, 0.0), (3, (7, 5, 6), 0.5, 0.7),
                                              (6, (9, 8, 7), 1.0, 0.3), (6, (4, 13, 5), 2.0, 0.0)])
def test_stencil_apply_matches_dense(r, shape, h, shift):
    nx, ny, nz = shape
    P = workloads.poisson_uniform(nx, radius=r, seed=5, h=h, shift=shift, ny=ny, nz=nz)
    op = oracle.Operator(P)
    x = workloads.rng(11).standard_normal(P.n)
    y_dense = stencil_dense(P) @ x
    y = op.apply(x)
    assert np.max(np.abs(y - y_dense)) <= 1e-12 * np.max(np.abs(y_dense))
    idx = [0, 3, P.n // 2, P.n - 1]
    assert np.array_equal(op.apply_at(x, idx), y[idx])
    assert np.array_equal(op.diag(), np.diag(stencil_dense(P)))


def test_csr_apply_and_diag_match_scipy():
    P = workloads.convection_diffusion(6, seed=7)
    op = oracle.Operator(P)
    M = sp.csr_matrix((P.val, P.col_idx, P.row_ptr), shape=(P.n, P.n))
    x = workloads.rng(3).standard_normal(P.n)
    assert np.allclose(op.apply(x), M @ x, rtol=0, atol=1e-12 * np.abs(M @ x).max())
    assert np.array_equal(op.diag(), M.diagonal())


def test_convection_diffusion_structure():
    n = 5
    P = workloads.convection_diffusion(n, seed=9)
    A = dense(P)
    # 7-point structure, nnz = 7N - 6 n^2, M-matrix (upwind), weakly diagonally dominant
    assert P.nnz == 7 * n ** 3 - 6 * n * n
    off = A - np.diag(np.diag(A))
    assert (off <= 0).all()
    assert (np.diag(A) >= np.abs(off).sum(axis=1) - 1e-12).all()
    assert not np.allclose(A, A.T)  # nonsymmetric


# ---------------------------------------------------------------- m x m solve pins

def test_sym_eig_matches_numpy():
    g = workloads.rng(1)
    for c in [1, 2, 5, 7, 10, 16]:
        F = g.standard_normal((40, c))
        S = F.T @ F
        lam, V, _ = oracle.sym_eig(S)
        ref = np.linalg.eigvalsh(S)
        assert np.allclose(np.sort(lam), ref, rtol=1e-12, atol=1e-12 * ref.max())
        assert np.allclose(V @ np.diag(lam) @ V.T, S, atol=1e-12 * np.abs(S).max())
        assert np.allclose(V.T @ V, np.eye(c), atol=1e-13)


def test_pinv_well_conditioned_equals_normal_equations_and_lstsq():
    g = workloads.rng(2)
    F = g.standard_normal((200, 7))
    f = g.standard_normal(200)
    G, gv = F.T @ F, F.T @ f
    gamma, rank = oracle.pinv_solve(G, gv)
    assert rank == 7
    assert np.allclose(gamma, np.linalg.solve(G, gv), rtol=1e-11)
    assert np.allclose(gamma, np.linalg.lstsq(F, f, rcond=None)[0], rtol=1e-10)


def test_pinv_rank_deficient_is_minimum_norm():
    g = workloads.rng(3)
    B = g.standard_normal((100, 3))
    F = np.concatenate([B, B @ g.standard_normal((3, 2))], axis=1)  # rank 3, 5 columns
    f = g.standard_normal(100)
    G, gv = F.T @ F, F.T @ f
    gamma, rank = oracle.pinv_solve(G, gv)
    assert rank == 3
    ref = np.linalg.pinv(G, rcond=5 * 2.0 ** -52, hermitian=True) @ gv
    assert np.allclose(gamma, ref, rtol=1e-7, atol=1e-9 * np.abs(ref).max())
    ref_ls = np.linalg.lstsq(F, f, rcond=None)[0]  # minimum-norm least squares
    assert np.allclose(F @ gamma, F @ ref_ls, atol=1e-8 * np.linalg.norm(f))
    assert np.linalg.norm(gamma) <= np.linalg.norm(ref_ls) * (1 + 1e-6)


def test_pinv_zero_matrix_gives_zero():
    gamma, rank = oracle.pinv_solve(np.zeros((4, 4)), np.ones(4))
    assert rank == 0 and np.array_equal(gamma, np.zeros(4))


# ---------------------------------------------------------------- solver pins

def _jacobi_richardson(P, omega, beta, p, iters):
    op = oracle.Operator(P)
    dinv = 1.0 / op.diag()
    x = np.zeros(P.n)
    for k in range(iters):
        f = dinv * (P.b - op.apply(x))
        x = x + (beta if (k + 1) % p == 0 else omega) * f
    return x


@pytest.mark.parametrize("omega,beta,p", [(0.6, 0.6, 6), (0.6, 0.9, 4), (0.5, 0.3, 1)])
def test_m0_is_jacobi_richardson(omega, beta, p):
    # Eq. 3 with an empty history: B_k = omega I, or beta I at Anderson steps (p -> inf: Richardson)
    P = workloads.poisson_uniform(6, radius=1, seed=21, ny=7, nz=5)
    res = oracle.solve(P, omega, beta, m=0, p=p, tol=0.0, max_iter=23)
    assert res.status == oracle.NOT_CONVERGED and res.iterations == 23
    assert np.array_equal(res.x, _jacobi_richardson(P, omega, beta, p, 23))


@pytest.mark.parametrize("p", [2, 3, 4, 6])
def test_first_anderson_step_is_gmres(p):
    # x_p = xbar + beta f(xbar), xbar the GMRES iterate of dimension p-1 (Sec. 2, complete history)
    P = workloads.poisson_uniform(6, radius=1, seed=31, shift=0.2)
    A = dense(P)
    dinv = 1.0 / np.diag(A)
    beta = 0.7
    res = oracle.solve(P, omega=0.45, beta=beta, m=20, p=p, tol=0.0, max_iter=p, trace_cap=4)
    xbar, fnorm = gmres_iterate(A, dinv, P.b, np.zeros(P.n), p - 1)
    expect = xbar + beta * dinv * (P.b - A @ xbar)
    assert np.linalg.norm(res.x - expect) <= 1e-10 * np.linalg.norm(expect)
    assert abs(res.trace["fmin"][0] - fnorm) <= 1e-9 * fnorm
    assert res.trace["k"][0] == p - 1 and res.trace["c"][0] == p - 1


@pytest.mark.parametrize("p,omega", [(1, 0.6), (3, 0.6), (3, 1.1), (5, 0.3)])
def test_complete_history_minimises_over_krylov(p, omega):
    # m >= k: at every Anderson step k the minimised residual ||f_k - F gamma|| equals the
    # GMRES residual of dimension k, independent of omega and p (Sec. 2, GMRES equivalence)
    P = workloads.convection_diffusion(4, seed=41)
    A = dense(P)
    dinv = 1.0 / np.diag(A)
    res = oracle.solve(P, omega=omega, beta=0.6, m=50, p=p, tol=0.0, max_iter=12, trace_cap=20)
    for k, fmin in zip(res.trace["k"], res.trace["fmin"]):
        if k == 0:
            continue
        _, ref = gmres_iterate(A, dinv, P.b, np.zeros(P.n), int(k))
        assert abs(fmin - ref) <= 1e-7 * ref + 1e-12, (k, fmin, ref)
    assert np.all(np.diff(res.trace["fmin"][1:]) <= 1e-12)  # nested spaces: non-increasing


def test_ar_p1_has_anderson_every_step():
    P = workloads.poisson_uniform(5, radius=1, seed=51)
    res = oracle.solve(P, 0.6, 0.6, m=3, p=1, tol=0.0, max_iter=9, trace_cap=20)
    assert list(res.trace["k"]) == list(range(9))
    assert list(res.trace["c"]) == [0, 1, 2, 3, 3, 3, 3, 3, 3]


def test_sine_mode_closed_form():
    # 7-point Dirichlet Laplacian: sin modes are eigenvectors, lambda = sum_d (2 - 2 cos(pi a_d/(n+1)))/h^2
    n, h = 12, 0.5
    P = workloads.poisson_uniform(n, radius=1, seed=0, h=h)
    a, b, c = 2, 3, 1
    s = workloads.sine_mode_grid(n, n, n, a, b, c)
    lam = sum(2 - 2 * np.cos(np.pi * q / (n + 1)) for q in (a, b, c)) / h ** 2
    P.b = s
    res = oracle.solve(P, 0.6, 0.6, m=7, p=6, tol=1e-11, trace_cap=4)
    u = s / lam
    assert res.status == oracle.OK
    # one mode spans a one-dimensional Krylov space: F has rank 1 (pinv truncation path) and the
    # first extrapolation (k = 5) lands on the solution; r is only measured at the next
    # Anderson step, k = 11, where it is at round-off
    # (eigenvalues at the rounding level may sit either side of the threshold, so only bound it)
    assert 1 <= res.trace["rank"][0] < res.trace["c"][0]
    assert res.trace["fmin"][0] <= 1e-13 * np.linalg.norm(s)
    assert res.iterations == 11
    assert np.linalg.norm(res.x - u) <= 1e-11 * np.linalg.norm(u)


def test_k_modes_converge_at_first_anderson_step():
    n = 10
    P = workloads.poisson_uniform(n, radius=1, seed=0)
    modes = [(1, 1, 1), (2, 1, 3), (4, 2, 2)]
    P.b = sum((i + 1) * workloads.sine_mode_grid(n, n, n, *md) for i, md in enumerate(modes))
    res = oracle.solve(P, 0.6, 0.6, m=7, p=6, tol=1e-10, trace_cap=4)
    # 3 modes with distinct eigenvalues: Krylov dimension 3 <= c = 5, so x_6 is exact
    assert res.status == oracle.OK and res.iterations == 11
    assert 3 <= res.trace["rank"][0] < res.trace["c"][0]
    A = dense(P)
    x_ref = np.linalg.solve(A, P.b)
    assert np.linalg.norm(res.x - x_ref) <= 1e-10 * np.linalg.norm(x_ref)


@pytest.mark.parametrize("kind", ["7pt", "r6", "upwind"])
def test_dense_lu_brute_force(kind):
    if kind == "7pt":
        P = workloads.poisson_uniform(6, radius=1, seed=61)
        params = dict(m=7, p=6, omega=0.6, beta=0.6)
    elif kind == "r6":
        P = workloads.poisson_uniform(6, radius=6, seed=62, shift=0.1)
        params = dict(m=7, p=6, omega=0.6, beta=0.6)
    else:
        P = workloads.convection_diffusion(6, seed=63)
        params = dict(m=10, p=5, omega=0.5, beta=0.5)
    tol = 1e-10
    res = oracle.solve(P, tol=tol, **params)
    A = dense(P)
    x_lu = np.linalg.solve(A, P.b)
    kappa = np.linalg.cond(A)
    assert res.status == oracle.OK
    assert (res.iterations + 1) % params["p"] == 0
    assert np.linalg.norm(res.x - x_lu) <= kappa * tol * np.linalg.norm(x_lu)
    assert np.linalg.norm(P.b - A @ res.x) <= tol * np.linalg.norm(P.b) * (1 + 1e-6)
    assert abs(res.rel_residual - np.linalg.norm(P.b - A @ res.x) / np.linalg.norm(P.b)) < 1e-6 * tol


# ------------------------------------------------------ periodic boundaries (Sec. 3.2/3.3)

def periodic_symbol(w, n_axes, waves, h=1.0, shift=0.0):
    """Eigenvalue of the periodic operator on the Fourier mode with wave numbers ``waves``: each
    axis contributes w[0] + 2 sum_k w[k] cos(2 pi k a / n)."""
    lam = 0.0
    for n, a in zip(n_axes, waves):
        lam += w[0] + 2 * sum(w[k] * np.cos(2 * np.pi * k * a / n) for k in range(1, len(w)))
    return -lam / h ** 2 + shift


@pytest.mark.parametrize("r,shape", [(1, (8, 6, 5)), (3, (12, 10, 9)), (6, (16, 13, 14)), (6, (5, 7, 4))])
def test_periodic_fourier_modes_are_eigenvectors(r, shape):
    # circulant operators are diagonalised by Fourier modes for any stencil radius; (5, 7, 4) with
    # radius 6 makes taps wrap more than once
    nx, ny, nz = shape
    w = workloads.stencil_weights(r)
    P = workloads.StencilProblem(nx, ny, nz, r, w, 0.7, 0.3, np.zeros(nx * ny * nz), periodic=True)
    op = oracle.Operator(P)
    for waves, ph in [((1, 0, 0), 0.0), ((2, 3, 1), 0.4), ((nx - 1, 1, nz // 2), 1.3)]:
        v = workloads.fourier_mode_grid(nx, ny, nz, *waves, phase=ph)
        lam = periodic_symbol(w, (nx, ny, nz), waves, h=0.7, shift=0.3)
        assert np.allclose(op.apply(v), lam * v, rtol=0, atol=1e-12 * abs(lam) * np.abs(v).max() + 1e-13)


@pytest.mark.parametrize("r,shape,shift", [(3, (6, 5, 7), 0.0), (6, (5, 7, 4), 0.2), (1, (4, 4, 3), 1.0)])
def test_periodic_apply_matches_circulant_kronecker(r, shape, shift):
    nx, ny, nz = shape
    P = workloads.StencilProblem(nx, ny, nz, r, workloads.stencil_weights(r), 1.3, shift,
                                 np.zeros(nx * ny * nz), periodic=True)
    A = stencil_dense(P)
    x = workloads.rng(5).standard_normal(P.n)
    assert np.allclose(oracle.Operator(P).apply(x), A @ x, rtol=0, atol=1e-12 * np.abs(A @ x).max())


def test_periodic_single_mode_closed_form():
    # -lap u = cos mode on the periodic grid: u = mode / lambda(mode), reached at the first
    # Anderson step (one mode spans a one-dimensional Krylov space)
    n, r = 12, 3
    w = workloads.stencil_weights(r)
    v = workloads.fourier_mode_grid(n, n, n, 2, 1, 3, 0.5)
    P = workloads.StencilProblem(n, n, n, r, w, 1.0, 0.0, v.copy(), periodic=True)
    lam = periodic_symbol(w, (n, n, n), (2, 1, 3))
    res = oracle.solve(P, 0.6, 0.6, m=7, p=6, tol=1e-11)
    assert res.status == oracle.OK and res.iterations == 11
    assert np.linalg.norm(res.x - v / lam) <= 1e-11 * np.linalg.norm(v / lam)


@pytest.mark.parametrize("shift", [0.0, 0.4])
def test_periodic_dense_brute_force(shift):
    # Helmholtz (shift > 0) is nonsingular: dense LU. Periodic Poisson is singular (constants span
    # the null space); with a zero-mean right-hand side and x0 = 0 every iterate keeps zero mean,
    # so AAR converges to the minimum-norm least-squares solution
    P = workloads.periodic_modes(6, radius=3, seed=64, shift=shift)
    A = dense(P)
    tol = 1e-10
    res = oracle.solve(P, m=7, p=6, omega=0.6, beta=0.6, tol=tol)
    assert res.status == oracle.OK
    if shift > 0:
        x_ref = np.linalg.solve(A, P.b)
        kappa = np.linalg.cond(A)
    else:
        x_ref = np.linalg.lstsq(A, P.b, rcond=None)[0]
        ev = np.linalg.eigvalsh(A)
        kappa = ev[-1] / ev[np.abs(ev) > 1e-9].min()
        assert abs(res.x.mean()) <= 1e-12 * np.abs(res.x).max()
    assert np.linalg.norm(res.x - x_ref) <= kappa * tol * np.linalg.norm(x_ref)
    assert np.linalg.norm(P.b - A @ res.x) <= tol * np.linalg.norm(P.b) * (1 + 1e-6)


def test_zero_rhs_and_breakdown_and_max_iter():
    P = workloads.poisson_uniform(4, radius=1, seed=0)
    P.b = np.zeros(P.n)
    res = oracle.solve(P, tol=1e-8)
    assert res.status == oracle.OK and res.iterations == 0 and not res.x.any()
    P = workloads.poisson_uniform(4, radius=1, seed=0)
    P.b[5] = np.nan
    res = oracle.solve(P, m=3, p=2, tol=1e-8)
    assert res.status == oracle.ERR_BREAKDOWN and res.iterations == 1
    P = workloads.poisson_uniform(8, radius=1, seed=0)
    res = oracle.solve(P, m=3, p=4, tol=1e-12, max_iter=10)
    assert res.status == oracle.NOT_CONVERGED and res.iterations == 10


def test_x0_is_used():
    P = workloads.poisson_uniform(6, radius=1, seed=71)
    ref = oracle.solve(P, m=5, p=3, tol=1e-12)
    res = oracle.solve(P, m=5, p=3, tol=1e-6, x0=ref.x)
    assert res.status == oracle.OK and res.iterations == 2  # first Anderson step already converged
