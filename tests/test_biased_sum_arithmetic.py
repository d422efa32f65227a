"""The arithmetic of the biased block sums (the hopping sums of the filter's compensated product),
emulated exactly on the CPU with rational numbers and correct rounding to FP32.

It backs the tolerance of the certifying-filter parity test: the operation sequence the kernel
runs -- a power-of-two bias from a bound of each block, the FMA into the biased sum, the exact
amount added, the FMA's rounding error into an error sum, the rebias between blocks -- is replayed
step by step, every step claimed exact is checked to be exact, and the error of the whole sum is
compared with the 2^-40.8 of the bound the parity test allows (and with the TwoSum (Dot2) form, which
must be the more accurate).  The error scales with the bound the bias is chosen for: here the bound
is sum |a| |bh| itself; the kernel bounds complex products by the products of their |re| + |im|
and shares one bound between the two halves' sums, which can make its bound, and so its error
relative to one sum, a few times larger.  The emulation is written from the description of the method
(Sterbenz's lemma for the differences in one binade, the FMA's single rounding), not from the
kernel source; it shares nothing with the CUDA library.
"""
import math
from fractions import Fraction as F

import numpy as np
import pytest

TWO = F(2)


def rn32(q: F) -> F:
    """q rounded to the nearest FP32 number, ties to even (normal and subnormal range)."""
    if q == 0:
        return F(0)
    sgn = -1 if q < 0 else 1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while TWO ** e > a:
        e -= 1
    while TWO ** (e + 1) <= a:
        e += 1
    e = max(e, -126)
    ulp = TWO ** (e - 23)
    m = a / ulp
    fl = m.numerator // m.denominator
    rem = m - fl
    if rem > F(1, 2) or (rem == F(1, 2) and fl % 2 == 1):
        fl += 1
    return sgn * fl * ulp


def f32(x: float) -> F:
    return F(float(np.float32(x)))


def fma(a, b, c):
    return rn32(a * b + c)


def add(a, b):
    return rn32(a + b)


def sub(a, b):
    return rn32(a - b)


def bias_of(bound: F) -> F:
    """1.5 sigma, sigma the smallest power of two >= fl(2.125 bound), at least 2^-100."""
    v = max(rn32(F(17, 8) * bound), TWO ** -100)
    k = -100
    while TWO ** k < v:
        k += 1
    return F(3, 2) * TWO ** k


def biased_sum(blocks):
    """blocks: lists of (a, bh, bl) FP32 triples.  Returns (hi, e) with hi + e ~ sum a (bh + bl)."""
    S = bias_of(F(0))
    bo, e, bound = S, F(0), F(0)
    for blk in blocks:
        for a, bh, _ in blk:
            bound = fma(abs(a), abs(bh), bound)          # the block's bound, accumulated with FMAs
        bn = bias_of(bound)
        d = sub(S, bo)
        assert d == S - bo                               # Sterbenz: exact
        t = add(d, bn)
        z = sub(t, bn)
        assert z == t - bn
        r = sub(d, z)
        assert r == d - z                                # what the rebias drops, exactly
        e = add(e, r)
        S, bo = t, bn
        for a, bh, bl in blk:
            assert bo * F(2, 3) <= S < bo * F(4, 3)      # S stays in [sigma, 2 sigma)
            t = fma(a, bh, S)
            z = sub(t, S)
            assert z == t - S                            # the exact amount added
            e = fma(a, bl, add(e, fma(a, bh, -z)))
            S = t
    hi = sub(S, bo)
    assert hi == S - bo
    return hi, e


def two_sum(a, b):
    s = add(a, b)
    bb = sub(s, a)
    return s, add(sub(a, sub(s, bb)), sub(b, bb))


def dot2_sum(blocks):
    s, e = F(0), F(0)
    for blk in blocks:
        for a, bh, bl in blk:
            p = rn32(a * bh)
            pe = fma(a, bh, -p)
            s, te = two_sum(s, p)
            e = fma(a, bl, add(e, add(te, pe)))
    return s, e


def random_blocks(rng, spread):
    """Four blocks of 12 products a (bh + bl): a FP32, bh + bl the (hi, lo) split of an FP64 value;
    each block's magnitudes scaled by 10^U(-spread, spread)."""
    out = []
    for _ in range(4):
        mag = 10.0 ** rng.uniform(-spread, spread)
        a = [f32(v) for v in rng.standard_normal(12)]
        xs = rng.standard_normal(12) * mag
        bh = [f32(v) for v in xs]
        bl = [f32(float(F(v) - h)) for v, h in zip(xs, bh)]
        out.append(list(zip(a, bh, bl)))
    return out


@pytest.mark.parametrize("spread", [0.0, 3.0])
def test_biased_block_sums_are_exact_where_claimed_and_within_the_tolerance(spread):
    rng = np.random.default_rng(17 + int(spread))
    worst_b, worst_d = 0.0, 0.0
    for _ in range(40):
        blocks = random_blocks(rng, spread)
        exact = sum(a * (bh + bl) for blk in blocks for a, bh, bl in blk)
        scale = sum(abs(a * bh) for blk in blocks for a, bh, _ in blk)
        hi, e = biased_sum(blocks)
        s, e2 = dot2_sum(blocks)
        worst_b = max(worst_b, float(abs(hi + e - exact) / scale))
        worst_d = max(worst_d, float(abs(s + e2 - exact) / scale))
    assert worst_b <= 2.0 ** -40.8                       # the parity test's per-product allowance
    assert worst_d <= worst_b                            # Dot2 is the more accurate form


def test_bias_is_a_power_of_two_and_a_half_above_the_bound():
    for bound in (F(0), F(1, 3), F(7), F(123456789, 1000), TWO ** -110):
        b = bias_of(bound)
        sigma = b * F(2, 3)
        k = math.log2(sigma)
        assert k == int(k)                               # a power of two
        assert sigma >= F(17, 8) * bound * (1 - TWO ** -23)
        assert sigma >= TWO ** -100
