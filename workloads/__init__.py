"""Seeded synthetic inputs for the AAR solver: operators, right-hand sides, batches, request streams.

This module is shared by the CUDA path, the CPU oracle, the tests and the benchmark. It holds
only problem generation (grids, stencil coefficients, right-hand sides, sparse operators and
request streams); none of the AAR method's arithmetic lives here. Every generator draws from
``numpy.random.Generator(PCG64(seed))`` with ``seed = workload_index * 1000 + system_index``.

The paper's own inputs (Matrix Market matrices, DFT electron densities and pseudocharges,
Sec. 3) are not available; these generators produce stand-ins with the same structure:
3-D finite-difference Poisson/Helmholtz operators with zero Dirichlet boundaries and a
nonsymmetric sparse operator (first-order upwind convection-diffusion).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from fractions import Fraction

import numpy as np

__all__ = [
    "rng",
    "stencil_weights",
    "StencilProblem",
    "CsrProblem",
    "uniform_rhs",
    "sine_modes_rhs",
    "sine_mode_grid",
    "poisson_uniform",
    "poisson_sine_modes",
    "convection_diffusion",
    "batched_helmholtz",
    "serving_requests",
    "ComplexStencilProblem",
    "complex_uniform",
    "ofdft_density",
    "ofdft_helmholtz",
    "OFDFT_P",
    "OFDFT_Q",
    "OFDFT_ALPHA",
]


def rng(seed: int) -> np.random.Generator:
    """The one generator every workload draws from (PCG64, seeded)."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def stencil_weights(radius: int) -> np.ndarray:
    """Centred finite-difference weights w[0..r] of d^2/dx^2 with accuracy order 2r (h = 1).

    Closed form for the centred 2r-th order second derivative:
    w_k = 2 (-1)^(k+1) (r!)^2 / (k^2 (r-k)! (r+k)!) for k >= 1 and w_0 = -2 sum_k w_k.
    radius 1 gives [-2, 1]; radius 3 gives the sixth-order weights the paper's Poisson and
    Helmholtz discretisations use (Sec. 3.2, 3.3). Computed in exact rationals, then rounded.
    """
    r = int(radius)
    if not 1 <= r <= 6:
        raise ValueError("radius must be in [1, 6]")
    fr = math.factorial(r)
    w = [Fraction(0)] * (r + 1)
    for k in range(1, r + 1):
        w[k] = Fraction(2 * (-1) ** (k + 1) * fr * fr, k * k * math.factorial(r - k) * math.factorial(r + k))
    w[0] = -2 * sum(w[1:])
    return np.array([float(v) for v in w], dtype=np.float64)


@dataclass
class StencilProblem:
    """(-lap_h + shift) u = b on an nx*ny*nz grid, x fastest; zero Dirichlet ghosts, or periodic
    in every axis when ``periodic`` is set."""

    nx: int
    ny: int
    nz: int
    radius: int
    weights: np.ndarray  # w[0..radius], 1-D second-derivative weights for h = 1
    h: float
    shift: float
    b: np.ndarray  # float64, length nx*ny*nz, index (z*ny + y)*nx + x
    periodic: bool = False

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz


@dataclass
class ComplexStencilProblem:
    """(scale (-lap_h) + q) u = b with complex q and b (Eq. 7's operator: scale = 1/(4 pi), q = Q),
    x fastest; zero Dirichlet ghosts, or periodic in every axis when ``periodic`` is set."""

    nx: int
    ny: int
    nz: int
    radius: int
    weights: np.ndarray  # w[0..radius], 1-D second-derivative weights for h = 1
    h: float
    scale: float
    q: complex
    b: np.ndarray  # complex128, length nx*ny*nz, index (z*ny + y)*nx + x
    periodic: bool = True

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz


@dataclass
class CsrProblem:
    """A x = b with A in CSR (int32 indices, float64 values)."""

    n: int
    row_ptr: np.ndarray  # int32[n+1]
    col_idx: np.ndarray  # int32[nnz]
    val: np.ndarray  # float64[nnz]
    b: np.ndarray  # float64[n]

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


def uniform_rhs(n: int, seed: int) -> np.ndarray:
    """b_i i.i.d. uniform[-1, 1]."""
    return rng(seed).uniform(-1.0, 1.0, size=int(n))


def sine_mode_grid(nx: int, ny: int, nz: int, a: int, b: int, c: int) -> np.ndarray:
    """prod_d sin(pi a_d i_d / (n_d + 1)) on interior indices i_d = 1..n_d, flattened x fastest."""
    sx = np.sin(np.pi * a * np.arange(1, nx + 1) / (nx + 1))
    sy = np.sin(np.pi * b * np.arange(1, ny + 1) / (ny + 1))
    sz = np.sin(np.pi * c * np.arange(1, nz + 1) / (nz + 1))
    return (sz[:, None, None] * sy[None, :, None] * sx[None, None, :]).reshape(-1)


def sine_modes_rhs(n: int, seed: int, n_modes: int = 8, max_wave: int = 16, noise: float = 1e-3):
    """Sum of random Dirichlet sine modes plus small uniform noise on an n^3 grid.

    Wave numbers uniform over {1..max_wave}^3, amplitudes uniform[-1, 1], noise
    ``noise * uniform[-1, 1]``. Returns (b, modes) with modes = [(a, b, c, amplitude), ...].
    """
    g = rng(seed)
    waves = g.integers(1, max_wave + 1, size=(n_modes, 3))
    amps = g.uniform(-1.0, 1.0, size=n_modes)
    b = np.zeros(n * n * n)
    for (wa, wb, wc), amp in zip(waves, amps):
        b += amp * sine_mode_grid(n, n, n, int(wa), int(wb), int(wc))
    if noise:
        b += noise * g.uniform(-1.0, 1.0, size=b.size)
    modes = [(int(w[0]), int(w[1]), int(w[2]), float(a)) for w, a in zip(waves, amps)]
    return b, modes


def poisson_uniform(n: int, radius: int = 1, seed: int = 0, h: float = 1.0, shift: float = 0.0,
                    ny: int | None = None, nz: int | None = None) -> StencilProblem:
    """-lap u = f (or Helmholtz with ``shift``) with f i.i.d. uniform[-1, 1]."""
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    return StencilProblem(n, ny, nz, radius, stencil_weights(radius), float(h), float(shift),
                          uniform_rhs(n * ny * nz, seed))


def fourier_mode_grid(nx: int, ny: int, nz: int, a: int, b: int, c: int, phase: float = 0.0) -> np.ndarray:
    """cos(2 pi (a i/nx + b j/ny + c k/nz) + phase) on the periodic grid, flattened x fastest."""
    i = np.arange(nx)[None, None, :]
    jj = np.arange(ny)[None, :, None]
    kk = np.arange(nz)[:, None, None]
    return np.cos(2 * np.pi * (a * i / nx + b * jj / ny + c * kk / nz) + phase).reshape(-1)


def periodic_modes_rhs(n: int, seed: int, n_modes: int = 8, max_wave: int = 16, noise: float = 1e-3):
    """Sum of random periodic Fourier modes plus small uniform noise on an n^3 periodic grid, with
    zero mean (the periodic Poisson system is consistent only for a zero-mean right-hand side).

    Wave numbers uniform over {0..max_wave}^3 without (0, 0, 0), amplitudes uniform[-1, 1],
    phases uniform[0, 2 pi), noise ``noise * uniform[-1, 1]`` with its mean removed. Returns
    (b, modes) with modes = [(a, b, c, amplitude, phase), ...].
    """
    g = rng(seed)
    modes = []
    b = np.zeros(n * n * n)
    while len(modes) < n_modes:
        w = g.integers(0, max_wave + 1, size=3)
        amp, ph = g.uniform(-1.0, 1.0), g.uniform(0.0, 2 * np.pi)
        if not w.any():
            continue
        b += amp * fourier_mode_grid(n, n, n, int(w[0]), int(w[1]), int(w[2]), ph)
        modes.append((int(w[0]), int(w[1]), int(w[2]), float(amp), float(ph)))
    if noise:
        e = noise * g.uniform(-1.0, 1.0, size=b.size)
        b += e - e.mean()
    return b, modes


def periodic_modes(n: int, radius: int = 3, seed: int = 5000, h: float = 1.0, shift: float = 0.0) -> StencilProblem:
    """-lap u = f (or Helmholtz with ``shift``) on an n^3 periodic grid with the 2r-th order
    stencil (radius 3: the paper's sixth order, Sec. 3.2/3.3), f = 8 random Fourier modes plus
    1e-3 noise, zero mean."""
    b, _ = periodic_modes_rhs(n, seed)
    return StencilProblem(n, n, n, radius, stencil_weights(radius), float(h), float(shift), b, periodic=True)


def poisson_sine_modes(n: int, radius: int = 6, seed: int = 1000, h: float = 1.0) -> StencilProblem:
    """-lap u = f with f = 8 random sine modes + 1e-3 uniform noise (the 256^3 radius-6 workload)."""
    b, _ = sine_modes_rhs(n, seed)
    return StencilProblem(n, n, n, radius, stencil_weights(radius), float(h), 0.0, b)


def convection_diffusion(n: int, seed: int = 2000, peclet: float = 5.0, n_modes: int = 16,
                         h: float = 1.0) -> CsrProblem:
    """-lap u + v . grad u = f on an n^3 grid, 7-point Laplacian, first-order upwind convection.

    v_d(x) = sum_q A_qd cos(2 pi k_q . x / (n+1) + phi_qd) over 16 wave vectors k_q drawn from
    {0..3}^3 minus the origin, A uniform[-1, 1], phi uniform[0, 2 pi); v is scaled so that
    max |v_d| h / 2 = peclet (unit diffusion). Upwind rows add
    v_d^+ (u_i - u_{i-1})/h + v_d^- (u_{i+1} - u_i)/h with v^+ = max(v, 0), v^- = min(v, 0).
    Zero Dirichlet ghosts. f uniform[-1, 1]. Column indices in each row are ascending.
    """
    g = rng(seed)
    ks = []
    while len(ks) < n_modes:
        k = g.integers(0, 4, size=3)
        if k.any():
            ks.append(k)
    ks = np.array(ks, dtype=np.float64)
    amp = g.uniform(-1.0, 1.0, size=(n_modes, 3))
    phi = g.uniform(0.0, 2.0 * np.pi, size=(n_modes, 3))
    idx = np.arange(1, n + 1, dtype=np.float64)
    Z, Y, X = np.meshgrid(idx, idx, idx, indexing="ij")
    coords = np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)], axis=1)  # x, y, z per point
    phase = 2.0 * np.pi * coords @ ks.T / (n + 1)  # [N, q]
    v = np.zeros((coords.shape[0], 3))
    for d in range(3):
        v[:, d] = np.cos(phase + phi[None, :, d]) @ amp[:, d]
    vmax = np.abs(v).max()
    v *= peclet * 2.0 / (h * vmax)
    inv_h2 = 1.0 / (h * h)
    N = n ** 3
    strides = (1, n, n * n)
    pos = np.stack([coords[:, 0] - 1, coords[:, 1] - 1, coords[:, 2] - 1], axis=1).astype(np.int64)
    rows = np.arange(N, dtype=np.int64)
    diag = np.full(N, 6.0 * inv_h2)
    entries_c = []
    entries_v = []
    for d in range(3):
        vp = np.maximum(v[:, d], 0.0) / h
        vm = np.minimum(v[:, d], 0.0) / h
        diag += vp - vm
        lo_ok = pos[:, d] > 0
        hi_ok = pos[:, d] < n - 1
        lo_val = -inv_h2 - vp
        hi_val = -inv_h2 + vm
        entries_c.append(np.where(lo_ok, rows - strides[d], -1))
        entries_v.append(lo_val)
        entries_c.append(np.where(hi_ok, rows + strides[d], -1))
        entries_v.append(hi_val)
    entries_c.append(rows)
    entries_v.append(diag)
    C = np.stack(entries_c, axis=1)
    V = np.stack(entries_v, axis=1)
    order = np.argsort(np.where(C < 0, np.iinfo(np.int64).max, C), axis=1, kind="stable")
    C = np.take_along_axis(C, order, axis=1)
    V = np.take_along_axis(V, order, axis=1)
    keep = C >= 0
    counts = keep.sum(axis=1)
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(counts)
    col_idx = C[keep].astype(np.int32)
    val = V[keep].astype(np.float64)
    b = g.uniform(-1.0, 1.0, size=N)
    return CsrProblem(N, row_ptr.astype(np.int32), col_idx, val, b)


def batched_helmholtz(count: int = 512, seed_base: int = 3000, side_lo: int = 16, side_hi: int = 96,
                      radius: int = 1):
    """Independent Helmholtz systems (-lap + c) u = f: side log-uniform in [lo, hi], c in [0.1, 2].

    System i draws from seed ``seed_base + i``: side = round(exp(U[ln lo, ln hi])), c, then f.
    """
    out = []
    for i in range(count):
        g = rng(seed_base + i)
        side = int(round(math.exp(g.uniform(math.log(side_lo), math.log(side_hi)))))
        c = float(g.uniform(0.1, 2.0))
        b = g.uniform(-1.0, 1.0, size=side ** 3)
        out.append(StencilProblem(side, side, side, radius, stencil_weights(radius), 1.0, c, b))
    return out


@dataclass
class Request:
    """One solve request of the serving stream."""

    rid: int
    arrival_s: float
    side: int
    tol: float
    shift: float  # 0 for Poisson, c > 0 for Helmholtz
    seed: int


def serving_requests(rate_hz: float = 2000.0, duration_s: float = 30.0, seed: int = 4000,
                     sides=(32, 48, 64, 96, 128, 192), tols=(1e-6, 1e-8, 1e-10), max_requests=None):
    """Poisson-process arrivals; side, tolerance uniform over the given sets; 50/50 Poisson/Helmholtz.

    Request j's right-hand side is ``uniform_rhs(side**3, seed * 1000 + j + 1)`` (drawn lazily
    by the consumer so the stream itself stays small).
    """
    g = rng(seed)
    t = 0.0
    out = []
    j = 0
    while True:
        t += g.exponential(1.0 / rate_hz)
        if t >= duration_s or (max_requests is not None and j >= max_requests):
            break
        side = int(sides[g.integers(0, len(sides))])
        tol = float(tols[g.integers(0, len(tols))])
        helm = bool(g.integers(0, 2))
        c = float(g.uniform(0.1, 2.0)) if helm else 0.0
        out.append(Request(j, t, side, tol, c, seed * 1000 + j + 1))
        j += 1
    return out


# ------------------------------------------------------------------ complex Helmholtz (Eq. 7)

# Constants of the OF-DFT kernel-potential equation (Eq. 7): P and Q complex, alpha = 5/6 + sqrt(5)/6
OFDFT_P = complex(0.003277, -0.009081)
OFDFT_Q = complex(-0.134992, -0.070225)
OFDFT_ALPHA = 5.0 / 6.0 + math.sqrt(5.0) / 6.0


def complex_uniform(nx: int, ny: int, nz: int, radius: int = 3, seed: int = 6000, h: float = 1.0,
                    scale: float = 1.0, q: complex = complex(0.3, 0.2), periodic: bool = True) -> ComplexStencilProblem:
    """Complex Helmholtz-type system with b = U[-1, 1] + i U[-1, 1] (real parts drawn first)."""
    g = rng(seed)
    n = nx * ny * nz
    re = g.uniform(-1.0, 1.0, size=n)
    im = g.uniform(-1.0, 1.0, size=n)
    return ComplexStencilProblem(nx, ny, nz, radius, stencil_weights(radius), float(h), float(scale), complex(q),
                                 re + 1j * im, periodic)


def ofdft_density(cells: int, n: int, seed: int, lattice: float = 7.78, sigma: float = 1.0, valence: float = 3.0,
                  max_shift: float = 0.25) -> np.ndarray:
    """Stand-in electron density of an aluminium supercell of cells^3 FCC unit cells (lattice
    constant 7.78 Bohr, the cell of Sec. 3.2), atoms displaced by U[-max_shift, max_shift] Bohr per
    coordinate: a sum of normalised Gaussians (width sigma, charge = valence) around the atoms,
    periodic (nearest image, cut at 6 sigma), sampled on an n^3 grid of spacing L / n. float64, x fastest.
    """
    g = rng(seed)
    L = cells * lattice
    hh = L / n
    basis = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
    cellpos = np.array([[i, j, k] for k in range(cells) for j in range(cells) for i in range(cells)], dtype=np.float64)
    atoms = ((cellpos[:, None, :] + basis[None, :, :]) * lattice).reshape(-1, 3)
    atoms = atoms + g.uniform(-max_shift, max_shift, size=atoms.shape)
    rho = np.zeros((n, n, n))  # [z, y, x]
    w = min((n - 1) // 2, int(math.ceil(6.0 * sigma / hh)))  # 2w + 1 <= n: no index twice in a box
    norm = valence / (math.pi ** 1.5 * sigma ** 3)
    offs = np.arange(-w, w + 1)
    for a in atoms:
        c = np.rint(a / hh).astype(np.int64)
        gauss = []
        idx = []
        for ax in range(3):
            pts = c[ax] + offs
            d = pts * hh - a[ax]
            gauss.append(np.exp(-(d * d) / (sigma * sigma)))
            idx.append(np.mod(pts, n))
        blk = norm * gauss[2][:, None, None] * gauss[1][None, :, None] * gauss[0][None, None, :]
        rho[np.ix_(idx[2], idx[1], idx[0])] += blk
    return rho.reshape(-1)


def ofdft_helmholtz(cells: int = 1, h: float = 0.216, seed: int = 6000, radius: int = 3) -> ComplexStencilProblem:
    """Eq. 7 on a periodic aluminium supercell: -(1/(4 pi)) lap V + Q V = P rho^alpha, sixth-order
    stencil (radius 3), n = round(7.78 cells / h) points per side at spacing L / n (Sec. 3.2 cell:
    cells = 3, h = 0.486, n = 48; the Jacobi runs of its appendix: cells = 1, h = 0.216 / 0.108,
    n = 36 / 72), rho from ofdft_density."""
    L = cells * 7.78
    n = int(round(L / h))
    rho = ofdft_density(cells, n, seed)
    b = OFDFT_P * np.power(rho, OFDFT_ALPHA)
    return ComplexStencilProblem(n, n, n, radius, stencil_weights(radius), L / n, 1.0 / (4.0 * math.pi), OFDFT_Q,
                                 b.astype(np.complex128), True)
