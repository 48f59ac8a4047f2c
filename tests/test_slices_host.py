"""Host replay of the exact-slice FP64 contraction (kernels_os.cu) in Python
integers: the 56-bit scaling, the balanced base-2^8 digits, the level sums and
their bounds, and the final rounding, against the exact rational product.

This pins the arithmetic the kernel is built on (Ozaki, Ogita & Oishi 2012:
error-free splitting of a matrix product) independently of the GPU: digits
reconstruct the scaled integers exactly, every level sum of a 55-term
contraction stays below 2^23 (so an FP32 accumulator holds it exactly), and
the result is within the final FP64 rounding plus the 56-bit input rounding
(at most 2^-55 of max|W| max|D| per term) of the exact value.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

BETA, SLICES, LEVELS = 8, 7, range(2, 10)


def biased_exponent(x: float) -> int:
    if x == 0.0:
        return 0
    return math.frexp(abs(x))[1] + 1022  # frexp: x = m 2^e with 0.5 <= m < 1


def fixed56(x: float, emax: int) -> int:
    """x * 2^(56 - e) with e = emax - 1022, rounded to nearest (ties up), as the kernel."""
    if x == 0.0:
        return 0
    m, e = math.frexp(abs(x))
    M = int(m * (1 << 53))  # 53-bit significand
    E = e + 1022  # biased exponent of x
    sh = emax - E - 3
    F = M << (-sh) if sh <= 0 else ((M + (1 << (sh - 1))) >> sh if sh < 60 else 0)
    return -F if x < 0 else F


def digits(F: int):
    G = F + 0x808080808080
    m = [G >> 48]
    for k in range(5, -1, -1):
        m.append(((G >> (8 * k)) & 0xFF) - 128)
    return m


def slice_contract(W: np.ndarray, D: np.ndarray) -> np.ndarray:
    """G[P, I] = sum_q W[P, q] D[I, q] the way the kernel computes it."""
    npair = W.shape[1]
    fP = [max(biased_exponent(w) for w in W[P]) for P in range(W.shape[0])]
    eI = [max(biased_exponent(d) for d in D[I]) for I in range(D.shape[0])]
    wd = [[digits(fixed56(W[P, q], fP[P])) if fP[P] else [0] * SLICES for q in range(npair)] for P in range(W.shape[0])]
    dd = [[digits(fixed56(D[I, q], eI[I])) if eI[I] else [0] * SLICES for q in range(npair)] for I in range(D.shape[0])]
    G = np.zeros((W.shape[0], D.shape[0]))
    worst = 0
    for P in range(W.shape[0]):
        for I in range(D.shape[0]):
            acc = 0
            for L in LEVELS:
                v = sum(dd[I][q][s - 1] * wd[P][q][L - s - 1]
                        for s in range(1, SLICES + 1) if 1 <= L - s <= SLICES for q in range(npair))
                worst = max(worst, abs(v))
                sh = 56 - BETA * L
                acc += v << sh if sh >= 0 else v >> (-sh)
            if acc and eI[I] and fP[P]:
                G[P, I] = float(Fraction(acc) * Fraction(2) ** ((eI[I] - 1022) + (fP[P] - 1022) - 56))
    return G, worst


@pytest.mark.parametrize("seed,spread", [(0, 0.0), (1, 8.0), (2, 30.0)])
def test_slice_contraction_against_exact(seed, spread):
    rng = np.random.default_rng(seed)
    npair, ndet, nout = 55, 6, 4
    W = rng.standard_normal((nout, npair)) * 10.0 ** rng.uniform(-spread, 0, (nout, npair))
    D = rng.standard_normal((ndet, npair)) * 10.0 ** rng.uniform(-spread, 0, (ndet, npair))
    G, worst = slice_contract(W, D)
    assert worst < 2 ** 23  # exact in an FP32 accumulator
    for P in range(nout):
        for I in range(ndet):
            exact = sum(Fraction(W[P, q]) * Fraction(D[I, q]) for q in range(npair))
            scale = Fraction(max(abs(W[P])) * max(abs(D[I])))
            # the final rounding (2^-53 relative, 2^-52 with the level truncation),
            # the inputs rounded to 56 bits below their row maxima (at most
            # 2^-55 of the scale per term) and the dropped levels (2^-56)
            bound = Fraction(2) ** -52 * abs(exact) + (npair + 1) * Fraction(2) ** -55 * scale
            assert abs(Fraction(G[P, I]) - exact) <= bound


def test_worst_case_level_sum_below_2_23():
    """All digits at their extremes (|m_1| = 256, |m_s| = 128 with equal signs):
    the largest level sum over 55 terms is 55 (2 * 2^15 + 5 * 2^14) < 2^23."""
    worst = 0
    for L in LEVELS:
        v = 0
        for s in range(1, SLICES + 1):
            t = L - s
            if 1 <= t <= SLICES:
                v += 55 * (256 if s == 1 else 128) * (256 if t == 1 else 128)
        worst = max(worst, v)
    assert worst == 55 * (2 * 2 ** 15 + 5 * 2 ** 14) and worst < 2 ** 23


def test_digits_reconstruct_and_stay_in_range():
    rng = np.random.default_rng(3)
    for F in list(rng.integers(-(2 ** 56) + 1, 2 ** 56 - 1, 2000)) + [0, 1, -1, 2 ** 56 - 1, -(2 ** 56) + 1]:
        F = int(F)
        m = digits(F)
        assert sum(d << (56 - BETA * (s + 1)) for s, d in enumerate(m)) == F
        assert abs(m[0]) <= 256 and all(-128 <= d <= 127 for d in m[1:])
