"""Pins for the oracle's loop-body operations that the whole-chain pins do
not fix: the polynomial's coefficient order, the compare-and-select
operations on equal operands, signed zeros and NaN, the INC store, the MAX
reduction, and the FP32 heat operator.  Every expected value is computed
here from the IR's definition (include/opstile.h: POLY by Horner with one
rounding per step, MIN(a, b) = b < a ? b : a, MAX(a, b) = b > a ? b : a,
SGT(a, b, c, e) = a > b ? c : e, INC: dat = dat + r) with Python floats or
exact rationals, never by the oracle or the CUDA library."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from synth import rng as R
from synth.program import (Arg, BodyBuilder, Chain, DatSpec, Loop, DAT, REDARG, READ, WRITE, INC, RMAX, MIN,
                           MAX, SGT)


def fma_exact(a, b, c):
    """a*b + c rounded once to FP64."""
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def round_f32(q: Fraction) -> np.float32:
    """The exact rational q rounded once to binary32 (nearest, ties to even)."""
    if q == 0:
        return np.float32(0.0)
    neg = q < 0
    q = -q if neg else q
    e = q.numerator.bit_length() - q.denominator.bit_length()
    if Fraction(2) ** e > q:
        e -= 1
    e = max(e, -126)  # subnormals keep the smallest normal exponent
    scaled = q / Fraction(2) ** (e - 23)
    n = scaled.numerator // scaled.denominator
    rem = scaled - n
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and n % 2 == 1):
        n += 1
    v = float(Fraction(n) * Fraction(2) ** (e - 23))
    return np.float32(-v if neg else v)


def fmaf_exact(a, b, c):
    """a*b + c of floats, rounded once to binary32."""
    return round_f32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def _chain1d(vals, code, K, out_access=WRITE, init_out=None):
    """One 1D loop over len(vals[0]) points: arguments 0..k-1 read the given
    arrays, the last argument is the output dat."""
    n = len(vals[0])
    shp = (1, 1, n)
    dats = [DatSpec(f"in{i}", np.asarray(v, dtype=np.float64).reshape(shp)) for i, v in enumerate(vals)]
    out0 = np.zeros(shp) if init_out is None else np.asarray(init_out, dtype=np.float64).reshape(shp)
    dats.append(DatSpec("out", out0))
    args = [Arg(DAT, i, 0, READ) for i in range(len(vals))] + [Arg(DAT, len(vals), 0, out_access)]
    lp = Loop("pin", ((0, n), (0, 1), (0, 1)), args, code, K)
    return Chain("pin", 1, (n, 1, 1), (0, 0, 0), (0, 0, 0), dats, [[(0, 0, 0)]], [], [lp])


def _bits(x):
    return np.asarray(x, dtype=np.float64).view(np.uint64)


def test_poly_horner_order():
    """r = c0 + x (c1 + x (c2 + x c3)) with one rounding per fma, from the
    highest coefficient down; asymmetric coefficients, so a reversed order
    (or a multiply-then-add) gives other values."""
    rnd = np.random.default_rng(11)
    x = rnd.uniform(-2.0, 2.0, 64)
    coefs = [0.3, -1.7, 0.45, 2.25]
    code, K = BodyBuilder().ld(0, 0, 0).poly(1, 0, coefs).st(1, 1).build()
    got, _ = oracle.run_chain(_chain1d([x], code, K))
    want = []
    for v in x:
        t = coefs[3]
        for c in reversed(coefs[:3]):
            t = fma_exact(t, v, c)
        want.append(t)
    assert np.array_equal(_bits(got[1][0, 0]), _bits(want))
    rev = []
    for v in x:
        t = coefs[0]
        for c in coefs[1:]:
            t = fma_exact(t, v, c)
        rev.append(t)
    assert not np.array_equal(_bits(got[1][0, 0]), _bits(rev))


PAIRS = [(1.0, 2.0), (2.0, 1.0), (1.5, 1.5), (0.0, -0.0), (-0.0, 0.0), (math.nan, 1.0), (1.0, math.nan),
         (math.nan, math.nan), (-math.inf, 3.0), (3.0, math.inf), (-1e-310, 1e-310)]


@pytest.mark.parametrize("op,rule", [(MIN, lambda a, b: b if b < a else a), (MAX, lambda a, b: b if b > a else a)])
def test_min_max_rule_on_zeros_and_nan(op, rule):
    """MIN(a, b) = b < a ? b : a and MAX(a, b) = b > a ? b : a exactly as
    written: on +0/-0 and on NaN operands the first operand comes back (the
    bit pattern, sign and NaN included)."""
    a = np.array([p[0] for p in PAIRS])
    b = np.array([p[1] for p in PAIRS])
    code, K = BodyBuilder().ld(0, 0, 0).ld(1, 1, 0).emit(op, 2, 0, 1).st(2, 2).build()
    got, _ = oracle.run_chain(_chain1d([a, b], code, K))
    want = [rule(float(x), float(y)) for x, y in zip(a, b)]
    assert np.array_equal(_bits(got[2][0, 0]), _bits(want))
    # the rule is not symmetric: swapping the operands changes some results
    swapped = [rule(float(y), float(x)) for x, y in zip(a, b)]
    assert not np.array_equal(_bits(want), _bits(swapped))


def test_sgt_rule_on_zeros_and_nan():
    """SGT(a, b, c, e) = a > b ? c : e: a NaN or a signed-zero tie selects e."""
    a = np.array([p[0] for p in PAIRS])
    b = np.array([p[1] for p in PAIRS])
    c = np.arange(len(PAIRS)) + 10.0
    e = -np.arange(len(PAIRS)) - 10.0
    code, K = BodyBuilder().ld(0, 0, 0).ld(1, 1, 0).ld(2, 2, 0).ld(3, 3, 0).emit(SGT, 4, 0, 1, 2, 3).st(4, 4).build()
    got, _ = oracle.run_chain(_chain1d([a, b, c, e], code, K))
    want = [cc if x > y else ee for x, y, cc, ee in zip(a, b, c, e)]
    assert np.array_equal(got[4][0, 0], np.array(want))


def test_inc_store_adds_once():
    """An INC argument ends as old + value with one rounding; the value here
    is a weighted sum of the input, so the sum is checked in exact
    arithmetic (a WRITE would lose the old value, a double store double it)."""
    rnd = np.random.default_rng(12)
    x = rnd.uniform(-1.0, 1.0, 50)
    old = rnd.uniform(-1.0, 1.0, 50) * 1e3
    code, K = BodyBuilder().wsum(0, 0, [0.1]).st(1, 0).build()
    got, _ = oracle.run_chain(_chain1d([x], code, K, out_access=INC, init_out=old))
    want = [float(Fraction(float(o)) + Fraction(0.1 * float(v))) for o, v in zip(old, x)]
    assert np.array_equal(_bits(got[1][0, 0]), _bits(want))


def test_max_reduction_against_scalar_max():
    """A MAX reduction over U(0,1) data returns the largest per-point value."""
    n = 41
    shp = (1, n + 2, n + 2)
    a = R.uniform(R.subseed(9, "a"), shp)
    st = [[(0, 0, 0)], [(0, 0, 0), (0, 1, 0)]]
    code, K = BodyBuilder().wsum(0, 0, [0.5, -0.25]).red(1, 0).build()
    lp = Loop("redmax", ((0, n), (0, n)), [Arg(DAT, 0, 1, READ), Arg(REDARG, 0)], code, K)
    ch = Chain("redmax", 2, (n, n, 1), (1, 1, 0), (1, 1, 0), [DatSpec("a", a)], st, [RMAX], [lp])
    _, hist = oracle.run_chain(ch)
    vals = [fma_exact(-0.25, a[0, j + 2, i + 1], 0.5 * a[0, j + 1, i + 1]) for j in range(n) for i in range(n)]
    assert hist[0][0] == max(vals)
    assert hist[0][0] != min(vals)


def test_round_f32_helper():
    """The binary32 rounding used below: ties go to even, and values that a
    detour through FP64 would round twice are rounded once."""
    one = Fraction(1)
    ulp = Fraction(1, 2 ** 23)
    assert round_f32(one + ulp / 2) == np.float32(1.0)
    assert round_f32(one + 3 * ulp / 2) == np.float32(1.0 + 2.0 ** -22)
    q = one + ulp / 2 + Fraction(1, 2 ** 60)  # just above the tie: rounds up; via FP64 it would tie to 1.0
    assert round_f32(q) == np.float32(1.0 + 2.0 ** -23)
    assert np.float32(float(q)) == np.float32(1.0)


def test_matvec32_is_the_exactly_rounded_fp32_sequence():
    """The FP32 heat operator: w = d u, then four fused multiply-adds with the
    negated west, east, south and north face coefficients, each rounded once
    to binary32, zero outside the grid; faces and diagonal are the FP64 ones
    rounded to float.  Computed here cell by cell in exact arithmetic."""
    n = 7
    g = np.random.default_rng(13)
    kappa = np.exp(np.log(1e-2) + np.log(1e4) * g.random((n, n)))
    u = g.uniform(-1.0, 1.0, (n, n))
    got = oracle.matvec32(kappa, u)
    kx, ky, dg = oracle.faces(kappa)
    kxf, kyf, dgf, uf = (a.astype(np.float32) for a in (kx, ky, dg, u))
    for j in range(n):
        for i in range(n):
            uw = uf[j, i - 1] if i > 0 else np.float32(0)
            ue = uf[j, i + 1] if i < n - 1 else np.float32(0)
            us = uf[j - 1, i] if j > 0 else np.float32(0)
            un = uf[j + 1, i] if j < n - 1 else np.float32(0)
            t = round_f32(Fraction(float(dgf[j, i])) * Fraction(float(uf[j, i])))
            t = fmaf_exact(-kxf[j, i], uw, t)
            t = fmaf_exact(-kxf[j, i + 1], ue, t)
            t = fmaf_exact(-kyf[j, i], us, t)
            t = fmaf_exact(-kyf[j + 1, i], un, t)
            assert got[j, i] == float(t), (j, i, got[j, i], float(t))
