"""CPU model of the complex Anderson update's coefficient forms (no GPU needed).

Eq. 3 with the differences of Eq. 4/5 expanded over the raw iterates x_{k-c..k}, f_{k-c..k}:
x_{k+1} = x_k + beta f_k - sum_j (ax_j x_j + af_j f_j), ax_j = gamma_{j-1} - gamma_j,
af_j = beta ax_j (gamma_{-1} = gamma_c = 0). The FP32 (mixed-form) update takes every window
difference made by a Richardson step as x_{i+1} - x_i = omega f_i (Eq. 2 with B = omega I) and
moves it into the coefficient of f_i; only differences made by an Anderson step ((s + 1) mod p = 0
for step s = k - c + i) keep their two x columns. The model builds windows that obey that
relation, applies the kernel's coefficient rules and checks both forms against the
difference form of Eq. 3 itself.
"""
import numpy as np
import pytest


def crand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def window(rng, k, c, p, omega, n):
    """x_{k-c..k} and f_{k-c..k} for steps k-c .. k: Richardson steps obey x_{s+1} = x_s + omega f_s,
    steps with (s + 1) mod p == 0 (Anderson steps) produce an arbitrary x_{s+1}."""
    f = crand(rng, c + 1, n)
    x = np.empty((c + 1, n), dtype=complex)
    x[0] = crand(rng, n)
    for i in range(c):
        s = k - c + i
        x[i + 1] = crand(rng, n) if (s + 1) % p == 0 else x[i] + omega * f[i]
    return x, f


def eq3(x, f, gamma, beta):
    # x_{k+1} = x_k + beta f_k - (dX + beta dF) gamma, dX_i = x_{i+1} - x_i
    dx, df = np.diff(x, axis=0), np.diff(f, axis=0)
    return x[-1] + beta * f[-1] - ((dx + beta * df).T @ gamma)


def literal(x, f, gamma, beta):
    c = len(gamma)
    g = np.concatenate([[0], gamma, [0]])  # g[j + 1] = gamma_j
    ax = np.array([g[j] - g[j + 1] for j in range(c + 1)])
    af = beta * ax
    return x[-1] + beta * f[-1] - (ax @ x + af @ f), ax, af


def compressed(x, f, gamma, beta, omega, k, p):
    """The FP32 kernel's rules: cx_j from Anderson-made differences only, cf_j = af_j + gamma_j omega
    for a Richardson-made difference j; returns the update and the x columns it reads."""
    c = len(gamma)
    _, ax, af = literal(x, f, gamma, beta)
    made_by_anderson = [((k - c + i + 1) % p == 0) for i in range(c)]
    cx = np.zeros(c + 1, dtype=complex)
    cf = af.astype(complex).copy()
    for j in range(c + 1):
        if j > 0 and made_by_anderson[j - 1]:
            cx[j] += gamma[j - 1]
        if j < c:
            if made_by_anderson[j]:
                cx[j] -= gamma[j]
            else:
                cf[j] += gamma[j] * omega
    used = [j for j in range(c + 1) if cx[j] != 0]
    out = x[-1] + beta * f[-1] - (sum(cx[j] * x[j] for j in used) + cf @ f)
    return out, used


@pytest.mark.parametrize("c,p", [(1, 2), (3, 2), (7, 6), (9, 8), (9, 3), (16, 5), (5, 1)])
def test_compressed_update_equals_eq3(c, p):
    rng = np.random.default_rng(1000 + 17 * c + p)
    omega, beta = 0.6 - 0.2j, 0.5 + 0.3j
    for k in range(p - 1, p - 1 + 6 * p, p):  # Anderson steps k, (k + 1) mod p = 0
        if k < c:
            continue
        x, f = window(rng, k, c, p, omega, 64)
        gamma = crand(rng, c)
        ref = eq3(x, f, gamma, beta)
        lit, _, _ = literal(x, f, gamma, beta)
        cmp_, used = compressed(x, f, gamma, beta, omega, k, p)
        scale = np.abs(ref).max()
        assert np.abs(lit - ref).max() <= 1e-12 * scale
        assert np.abs(cmp_ - ref).max() <= 1e-12 * scale
        # the x columns read: those of the Anderson-made differences (at most two each)
        n_and = sum(((k - c + i + 1) % p == 0) for i in range(c))
        assert len(used) <= 2 * n_and
        if p > 1 and c >= p:
            assert len(used) < c + 1


def test_compressed_form_needs_the_richardson_relation():
    # a planted slip: a window whose Richardson steps used another omega breaks the compressed
    # form (but not the literal one), so the model does test the relation it relies on
    rng = np.random.default_rng(5)
    c, p, k = 9, 8, 15
    omega, beta = 0.6, 0.6
    x, f = window(rng, k, c, p, omega * 1.01, 32)
    gamma = crand(rng, c)
    ref = eq3(x, f, gamma, beta)
    cmp_, _ = compressed(x, f, gamma, beta, omega, k, p)
    lit, _, _ = literal(x, f, gamma, beta)
    assert np.abs(lit - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(cmp_ - ref).max() > 1e-6 * np.abs(ref).max()
