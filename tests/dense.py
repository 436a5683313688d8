"""Dense test-side constructions of the operators, written from their definitions.

These do not call the oracle or the CUDA path: they are the independent reference the oracle's
operator application is pinned against, and the brute-force direct solves.
"""
import numpy as np


def second_derivative_1d(n: int, w: np.ndarray) -> np.ndarray:
    """Banded Toeplitz n x n matrix with entries w[|i-j|] for |i-j| <= r, truncated at the ends
    (zero Dirichlet ghosts)."""
    r = len(w) - 1
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(max(0, i - r), min(n, i + r + 1)):
            D[i, j] = w[abs(i - j)]
    return D


def second_derivative_1d_periodic(n: int, w: np.ndarray) -> np.ndarray:
    """Circulant n x n matrix: row i gets w[|k|] at column (i + k) mod n for every k in -r..r
    (taps that wrap onto the same column add up, as when n < 2r + 1)."""
    r = len(w) - 1
    D = np.zeros((n, n))
    for i in range(n):
        for k in range(-r, r + 1):
            D[i, (i + k) % n] += w[abs(k)]
    return D


def stencil_dense(P) -> np.ndarray:
    """A = -(1/h^2)(Dxx + Dyy + Dzz) + shift I with index (z*ny + y)*nx + x (Kronecker form);
    circulant factors for a periodic problem."""
    w = np.asarray(P.weights, dtype=np.float64)
    d1 = second_derivative_1d_periodic if getattr(P, "periodic", False) else second_derivative_1d
    Dx = d1(P.nx, w)
    Dy = d1(P.ny, w)
    Dz = d1(P.nz, w)
    Ix, Iy, Iz = np.eye(P.nx), np.eye(P.ny), np.eye(P.nz)
    lap = np.kron(Iz, np.kron(Iy, Dx)) + np.kron(Iz, np.kron(Dy, Ix)) + np.kron(Dz, np.kron(Iy, Ix))
    return -lap / (P.h * P.h) + P.shift * np.eye(P.n)


def zstencil_dense(P) -> np.ndarray:
    """Complex A = scale * (-(1/h^2)(Dxx + Dyy + Dzz)) + q I (Eq. 7's operator) in Kronecker form."""
    w = np.asarray(P.weights, dtype=np.float64)
    d1 = second_derivative_1d_periodic if P.periodic else second_derivative_1d
    Dx, Dy, Dz = d1(P.nx, w), d1(P.ny, w), d1(P.nz, w)
    Ix, Iy, Iz = np.eye(P.nx), np.eye(P.ny), np.eye(P.nz)
    lap = np.kron(Iz, np.kron(Iy, Dx)) + np.kron(Iz, np.kron(Dy, Ix)) + np.kron(Dz, np.kron(Iy, Ix))
    return (P.scale * (-lap / (P.h * P.h))).astype(np.complex128) + complex(P.q) * np.eye(P.n)


def csr_dense(P) -> np.ndarray:
    A = np.zeros((P.n, P.n))
    for i in range(P.n):
        for e in range(P.row_ptr[i], P.row_ptr[i + 1]):
            A[i, P.col_idx[e]] += P.val[e]
    return A


def dense(P) -> np.ndarray:
    return stencil_dense(P) if hasattr(P, "radius") else csr_dense(P)


def gmres_iterate(A: np.ndarray, dinv: np.ndarray, b: np.ndarray, x0: np.ndarray, dim: int):
    """Left-preconditioned GMRES iterate of dimension ``dim`` by brute force (real or complex): minimise
    ||D^{-1}(b - A y)|| over y in x0 + K_dim(D^{-1}A, D^{-1}(b - A x0)) with an Arnoldi
    (modified Gram-Schmidt) basis and a dense least-squares solve."""
    if np.ndim(dinv) == 2:  # a dense preconditioner matrix M^{-1}
        M = dinv @ A
        f0 = dinv @ (b - A @ x0)
    else:
        M = dinv[:, None] * A
        f0 = dinv * (b - A @ x0)
    n = len(b)
    V = np.zeros((n, dim), dtype=np.result_type(M, f0))
    v = f0 / np.linalg.norm(f0)
    for j in range(dim):
        V[:, j] = v
        w = M @ v
        for i in range(j + 1):  # Hermitian inner products (plain dot for real data)
            w -= (np.conj(V[:, i]) @ w) * V[:, i]
        for i in range(j + 1):  # re-orthogonalise once
            w -= (np.conj(V[:, i]) @ w) * V[:, i]
        nw = np.linalg.norm(w)
        if nw == 0:
            V = V[:, : j + 1]
            break
        v = w / nw
    y, *_ = np.linalg.lstsq(M @ V, f0, rcond=None)
    xbar = x0 + V @ y
    if np.ndim(dinv) == 2:
        return xbar, np.linalg.norm(dinv @ (b - A @ xbar))
    return xbar, np.linalg.norm(dinv * (b - A @ xbar))


def block_diagonal_inverse(A: np.ndarray, nx: int, ny: int, nz: int, bs: int) -> np.ndarray:
    """Dense inverse of the block-diagonal part of A for the tiling of the grid by bs^3 boxes."""
    idx = np.arange(nx * ny * nz).reshape(nz, ny, nx)
    Minv = np.zeros_like(A)
    for Z in range(0, nz, bs):
        for Y in range(0, ny, bs):
            for X in range(0, nx, bs):
                bl = idx[Z:Z + bs, Y:Y + bs, X:X + bs].reshape(-1)
                Minv[np.ix_(bl, bl)] = np.linalg.inv(A[np.ix_(bl, bl)])
    return Minv


def stencil_lambda_min(P, zero_mean: bool = False) -> float:
    """Smallest eigenvalue of the symmetric stencil operator A = -(1/h^2)(Dxx + Dyy + Dzz) + shift I.

    A is a Kronecker sum of three 1-D matrices, so its eigenvalues are the sums mu_x + mu_y + mu_z
    of their eigenvalues (scaled by -1/h^2) plus the shift: the smallest one needs only three
    small symmetric eigenproblems. zero_mean: the smallest eigenvalue on the zero-mean subspace
    (periodic Poisson, whose constant mode has eigenvalue 0), i.e. the smallest sum other than
    the one of the three constant modes."""
    w = np.asarray(P.weights, dtype=np.float64)
    d1 = second_derivative_1d_periodic if getattr(P, "periodic", False) else second_derivative_1d
    mus = [np.sort(np.linalg.eigvalsh(-d1(n, w))) / (P.h * P.h) for n in (P.nx, P.ny, P.nz)]
    if not zero_mean:
        return float(sum(m[0] for m in mus) + P.shift)
    # the constant mode is the first of each axis; the next smallest sum raises one axis only
    base = sum(m[0] for m in mus)
    return float(min(base - m[0] + m[1] for m in mus) + P.shift)


def mixed_error_bound(lam_min: float, b_norm: float, x_norm: float, r_a: float, r_b: float) -> float:
    """Bound on ||x_a - x_b|| / ||x_b|| for two approximate solutions of A x = b with relative
    residuals r_a, r_b (symmetric A, smallest eigenvalue lam_min on the space both live in):
    ||x - A^{-1} b|| <= ||b - A x|| / lam_min for each, and the triangle inequality."""
    return (r_a + r_b) * b_norm / (lam_min * x_norm)
