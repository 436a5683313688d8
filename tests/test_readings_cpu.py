"""CPU checks of the arithmetic behind two readings of the GPU path (no GPU needed).

* The certified LDL^T solve of the FP64 form (the pseudoinverse of Sec. 3.2): trace(G) trace(G^-1)
  bounds the condition number of a symmetric positive definite G, so trace(G) trace(G^-1) c < 2^42
  puts every eigenvalue at least 2^10 above the cut c 2^-52 lambda_max, where pinv(G) = G^-1.
* The finalize computes trace(G^-1) from the factors, as sum_k ||row k of L^-1||^2 / d_k.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore")


def _spd(rng, c, cond, lam=None):
    q, _ = np.linalg.qr(rng.standard_normal((c, c)))
    if lam is None:
        lam = np.geomspace(1.0, 1.0 / cond, c)
    return (q * lam) @ q.T


@pytest.mark.parametrize("c", [1, 2, 7, 10, 16])
def test_trace_product_bounds_the_condition_number(c):
    # eigenvalues fixed by construction, so the traces and the condition number are exact up to
    # the rounding of G itself; spreads from even to clustered at both ends
    rng = np.random.default_rng(100 + c)
    for cond in (1.0, 1e3, 1e8, 1e12, 1e15):
        for shape in ("geom", "one_small", "one_large"):
            lam = np.geomspace(1.0, 1.0 / cond, c)
            if shape == "one_small":
                lam = np.r_[np.ones(c - 1), 1.0 / cond][:c]
            elif shape == "one_large":
                lam = np.r_[cond, np.ones(c - 1)][:c] / cond
            g = _spd(rng, c, cond, lam)
            kappa = lam.max() / lam.min()
            bound = np.trace(g) * np.sum(1.0 / lam)
            assert kappa <= bound * (1 + 1e-9)
            certified = bound * c < 2.0 ** 42
            if certified:
                cut = c * 2.0 ** -52 * lam.max()
                assert lam.min() >= 2.0 ** 10 * cut * (1 - 1e-9)
            if c > 1 and cond >= 1e15:
                assert not certified  # near the cut, the eigen-decomposition decides


@pytest.mark.parametrize("c", [3, 7, 12])
def test_trace_of_inverse_from_ldl_factors(c):
    # G = L D L^T (L unit lower triangular): G^-1 = L^-T D^-1 L^-1, so
    # trace(G^-1) = sum_k (1/d_k) ||row k of L^-1||^2
    rng = np.random.default_rng(200 + c)
    g = _spd(rng, c, 1e6)
    ch = np.linalg.cholesky(g)
    d = np.diag(ch) ** 2
    lmat = ch / np.diag(ch)
    linv = np.linalg.inv(lmat)
    tr = sum((linv[k] ** 2).sum() / d[k] for k in range(c))
    assert abs(tr - np.trace(np.linalg.inv(g))) <= 1e-9 * np.trace(np.linalg.inv(g))


def _bits(x):
    return np.asarray(x, dtype=np.float64).view(np.int64)


def test_bit_pattern_comparisons_of_the_eigensolver():
    # the Jacobi rounds compare through bit patterns: for non-negative operands, apq^2 <= bound is
    # lhs_bits <= rhs_bits with the bound not a NaN; apq != 0 is (bits << 1) != 0; d >= 0 (with
    # -0 counted as non-negative) is not (bits < 0 and (bits << 1) != 0). Each must agree with the
    # FP64 comparison wherever that comparison decides the rotation.
    rng = np.random.default_rng(7)
    special = np.array([0.0, -0.0, 5e-324, 1e-300, 1e-200, 1.0, 1.5, 2.0 ** 60, 1e300, np.inf, np.nan])
    mags = np.concatenate([special, np.abs(rng.standard_normal(200)) * 10.0 ** rng.integers(-30, 30, 200)])
    lhs = np.abs(mags)[:, None] ** 2
    rhs = np.abs(mags)[None, :] * 2.0 ** -104
    with np.errstate(all="ignore"):
        lhs = np.broadcast_to(lhs, (len(mags), len(mags)))
        rhs = np.broadcast_to(rhs, (len(mags), len(mags)))
        want = lhs <= rhs  # False whenever either side is NaN
    lb, rb = _bits(lhs), _bits(rhs)
    got = (lb <= rb) & (rb <= _bits(np.inf))
    decided = ~np.isnan(lhs)  # a NaN apq gives a NaN rotation either way
    assert np.array_equal(got[decided], want[decided])
    vals = np.concatenate([special, -special, rng.standard_normal(100)])
    b = _bits(vals)
    assert np.array_equal((b << 1) != 0, (vals != 0.0) | np.isnan(vals))
    neg = (b < 0) & ((b << 1) != 0)
    ok = ~np.isnan(vals)
    assert np.array_equal(neg[ok], ~(vals[ok] >= 0.0))
