"""Pins for the oracle's parameter sampler (Philox4x32-10 + Normal32).

The paper passes "the current random seed" to the GPU every sampling time
(Sect. II-D, "Fourth") and samples theta unconstrained in R^{n_theta}
(Sect. V-A, item (iii)); the generator itself is this library's choice:
Philox4x32-10 (Salmon et al., SC'11) and an FP32 Box-Muller transform.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

# Known-answer vectors published with the Philox generator (Random123
# distribution, kat_vectors: philox4x32 with 10 rounds): (ctr, key, output).
KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,want", KAT)
def test_philox_known_answers(orc, ctr, key, want):
    assert tuple(int(x) for x in orc.philox(ctr, key)) == want


def test_u24_exact(orc):
    rng = np.random.default_rng(0)
    for w in list(rng.integers(0, 2 ** 32, 2000)) + [0, 511, 512, 2 ** 32 - 1]:
        u = orc.u24(int(w))
        assert Fraction(u) == Fraction(2 * (int(w) >> 9) + 1, 2 ** 24)
        assert 0.0 < u < 1.0


def _ulp32(x):
    x = abs(float(x))
    return float(np.spacing(np.float32(x)))


def test_ln32_accuracy(orc):
    """ln32 within 2 ulp of the FP64 logarithm over the whole input grid's
    range (random odd multiples of 2^-24, plus the extremes)."""
    rng = np.random.default_rng(1)
    ws = list(rng.integers(0, 2 ** 32, 20000)) + [0, 2 ** 32 - 1, 0x3504F3 << 9, 0x3504F4 << 9]
    worst = 0.0
    for w in ws:
        u = orc.u24(int(w))
        got = orc.ln32(u)
        ref = math.log(u)
        err = abs(got - ref) / _ulp32(ref)
        worst = max(worst, err)
    assert worst <= 2.0, worst


def test_sincos2pi32_accuracy(orc):
    rng = np.random.default_rng(2)
    Ks = [int(2 * k + 1) for k in rng.integers(0, 2 ** 23, 20000)] + [1, 2 ** 24 - 1, 2 ** 22 + 1,
                                                                       2 ** 23 - 1, 2 ** 23 + 1]
    worst = 0.0
    for K in Ks:
        s, c = orc.sincos2pi32(K)
        ang = 2 * math.pi * K / 2 ** 24
        worst = max(worst, abs(s - math.sin(ang)), abs(c - math.cos(ang)))
    # absolute error below 2 ulp of 1
    assert worst <= 2 * 2.0 ** -24, worst


def test_normal_pair_vs_fp64_box_muller(orc):
    """Normal32 against the FP64 textbook Box-Muller on the same uniforms:
    z = sqrt(-2 ln u1) (cos, sin)(2 pi u2), within 4 ulp of max(|z|, R/8)."""
    rng = np.random.default_rng(3)
    worst = 0.0
    for a, b in rng.integers(0, 2 ** 32, (20000, 2)):
        z = orc.normal_pair(int(a), int(b))
        u1 = (2 * (int(a) >> 9) + 1) / 2 ** 24
        u2 = (2 * (int(b) >> 9) + 1) / 2 ** 24
        R = math.sqrt(-2 * math.log(u1))
        ref = (R * math.cos(2 * math.pi * u2), R * math.sin(2 * math.pi * u2))
        for g, r in zip(z, ref):
            scale = _ulp32(max(abs(r), R / 8))
            worst = max(worst, abs(float(g) - r) / scale)
    assert worst <= 4.0, worst


def test_theta_counter_layout(orc):
    """theta_n[i] comes from block i//4 of Philox(ctr=(i//4, n, t, stream),
    key=(seed lo, seed hi)); words (0,1) feed entries 4q, 4q+1 and (2,3) feed
    4q+2, 4q+3; the radius comes from the first word of each pair."""
    seed, t, n = 0x0123456789ABCDEF, 17, 5
    th = orc.theta(seed, t, n, 11)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for q in range(3):
        w = orc.philox((q, n, t, 0), key)
        z01 = orc.normal_pair(w[0], w[1])
        z23 = orc.normal_pair(w[2], w[3])
        want = np.concatenate([z01, z23])[: min(4, 11 - 4 * q)]
        assert np.array_equal(th[4 * q: 4 * q + len(want)], want)
    # distinct (n, t, stream) give distinct streams
    a = orc.theta(seed, t, n, 64)
    assert not np.array_equal(a, orc.theta(seed, t, n + 1, 64))
    assert not np.array_equal(a, orc.theta(seed, t + 1, n, 64))
    assert not np.array_equal(a, orc.theta(seed, t, n, 64, stream=1))


def test_theta_moments_and_ks(orc):
    """Over 10^6 draws: mean 0, variance 1, fourth moment 3, and a KS test
    against N(0,1) (the distribution the parameters are sampled from)."""
    from scipy import stats
    draws = np.concatenate([orc.theta(0x5EED0000, 3, n, 4000) for n in range(250)]).astype(np.float64)
    n = draws.size
    assert abs(draws.mean()) < 5 / math.sqrt(n)
    assert abs(draws.var() - 1) < 5 * math.sqrt(2 / n)
    assert abs(np.mean(draws ** 4) - 3) < 5 * math.sqrt(96 / n)
    assert stats.kstest(draws, "norm").pvalue > 1e-4
    # the largest radius the 23-bit uniform admits: sqrt(-2 ln 2^-24)
    assert np.abs(draws).max() <= math.sqrt(-2 * math.log(2.0 ** -24)) * (1 + 1e-6)
