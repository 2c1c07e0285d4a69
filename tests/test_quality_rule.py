"""The single-precision route of the mapping quality (Section "Postprocessing": quality
min(-10 log10(Pr), 255), Pr = (rank - 1) / n), checked on the CPU against the double expression
the oracle uses (its integer part after adding 1e-9, clamped to 0..255).

The ranking kernels first take 10 log10(n) - 10 log10(rank - 1) in single precision and keep its
integer part when the value lies more than 1e-3 from an integer; otherwise they evaluate the double
expression.  Here the single-precision arithmetic is numpy's float32 (a log10 correctly rounded or
nearly so; the GPU's log10f is within 2 ulp, about 1e-5 on these values), and the test checks that
every value the fast route keeps has the double expression's integer part, with the error of the
float value well inside the margin, over ranks 2 .. 2^32 - 1 and reference sizes from 1 kbp to
3.1 Gbp, including ratios at exact powers of ten.
"""
import math

import numpy as np


def _exact(R, n):
    v = math.floor(-10.0 * math.log10((R - 1) / n) + 1e-9)
    return max(0, min(255, v))


def _fast(R, n):
    """(value kept by the fast route or None, the float value)."""
    l10n = np.float32(10.0 * math.log10(n))
    vf = np.float32(l10n - np.float32(10.0) * np.log10(np.float32(R - 1)))
    fl = np.floor(vf)
    fr = vf - fl
    if fr > np.float32(1e-3) and fr < np.float32(1.0 - 1e-3):
        return max(0, min(255, int(fl))), float(vf)
    return None, float(vf)


def test_fast_route_keeps_only_exact_integer_parts():
    rng = np.random.default_rng(19)
    sizes = [1_000, 4_096, 1_000_000, 400_000_000, 3_100_000_000, 10 ** 9]
    ranks = set(range(2, 3000)) | {10 ** e + 1 for e in range(10)} | {2 ** e + 1 for e in range(32)}
    ranks |= set(int(x) for x in rng.integers(2, 2 ** 32 - 1, 20_000))
    kept = fell_back = 0
    worst = 0.0
    for n in sizes:
        for R in sorted(ranks):
            got, vf = _fast(R, n)
            exact_v = -10.0 * math.log10((R - 1) / n)
            worst = max(worst, abs(vf - exact_v))
            if got is None:
                fell_back += 1
                continue
            kept += 1
            assert got == _exact(R, n), (R, n, vf)
    assert worst < 1e-4, worst  # the margin of 1e-3 is ten times this
    assert fell_back < 0.01 * (kept + fell_back)  # the double route stays rare
    # ratios at exact powers of ten land on an integer and take the double route
    for n in (1_000, 10 ** 9):
        for e in range(1, 4):
            R = n // 10 ** e + 1
            assert _fast(R, n)[0] is None and _exact(R, n) == 10 * e
