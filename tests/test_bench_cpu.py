"""Host-side arithmetic of bench.py (no GPU): the whole-solve algorithmic byte count."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Info:
    def __init__(self, iterations, anderson_steps, refinements):
        self.iterations, self.anderson_steps, self.refinements = iterations, anderson_steps, refinements


def test_update_words_of_the_mixed_and_fp64_forms():
    n = 256 ** 3
    # one Anderson step and nothing else: 3 words of the Anderson sweep + (c + 1) Gram + update
    one = _Info(1, 1, 0)
    lit = bench.alg_bytes_per_solve(n, one, 7, 6, 4, False) / (4 * n) - 3 - 8
    # the mixed form adds the first FP64 residual (8 + 8 + 4 bytes = 5 words) at no refinement
    cmp_ = bench.alg_bytes_per_solve(n, one, 7, 6, 4, True) / (4 * n) - 3 - 8 - 5
    assert lit == 2 * 7 + 3
    # m = 7, p = 6: 8 residual columns, x_k, the two x columns of the one difference made by an
    # Anderson step, x_{k+1} written: 12 words, the 805 MB per launch of the 256^3 launch list
    assert cmp_ == 12
    assert 12 * 4 * n == 805306368


def test_solve_bytes_of_the_headline_counts():
    n = 256 ** 3
    info = _Info(1019, 177, 8)
    got = bench.alg_bytes_per_solve(n, info, 7, 6, 4, True)
    want = n * ((1019 - 177) * 16 + 177 * (12 + 32 + 48) + 9 * 20 + 8 * 20)
    assert got == want
