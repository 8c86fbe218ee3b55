"""The mixed form's device precision conversions (integer-pipe BF16/TF32 rounding of doubles
and exact widening of floats) against references built from arithmetic, not bits: the two
neighbours of |x| on the target grid and the exact distances to them (differences of
doubles in one binade are exact)."""
import numpy as np
import pytest

import paper_2311_08757_gb300 as dd

pytestmark = pytest.mark.gpu


def _nearest(x, keep, ties_even):
    """Round doubles to `keep` explicit mantissa bits: nearest, ties to even or away."""
    a = np.abs(x)
    _, e = np.frexp(a)                        # a = m 2^e, m in [1/2, 1)
    ulp = np.ldexp(1.0, e - 1 - keep)         # grid spacing in [2^(e-1), 2^e)
    q = np.floor(a / ulp)                     # exact: scaling by a power of two
    lo = q * ulp
    hi = lo + ulp
    dlo, dhi = a - lo, hi - a                 # exact
    up = (dhi < dlo) | ((dhi == dlo) & ((q % 2 == 1) if ties_even else True))
    return np.copysign(np.where(up, hi, lo), x)


def _inputs(seed, n=200_000, emin=-120, emax=120):
    rng = np.random.default_rng(seed)
    x = np.ldexp(rng.uniform(0.5, 1.0, n), rng.integers(emin, emax, n)) * rng.choice([-1.0, 1.0], n)
    # ties and near-ties on the BF16 grid (7 bits) and the TF32 grid (10 bits)
    base = np.ldexp(rng.integers(128, 256, 4000).astype(np.float64), rng.integers(-100, 100, 4000))
    ties = []
    for keep in (7, 10):
        b = np.ldexp(rng.integers(2 ** keep, 2 ** (keep + 1), 4000).astype(np.float64),
                     rng.integers(-100, 100, 4000))
        half = np.ldexp(1.0, np.frexp(b)[1] - 2 - keep)
        ties += [b + half, b + half * (1 + 2.0 ** -40), b + half * (1 - 2.0 ** -40), -(b + half)]
    # the top of the range: rounds to the largest finite value or overflows to infinity
    top = [np.ldexp(1.0, 128) * (1 - 2.0 ** -9), np.ldexp(1.0, 128) * (1 - 2.0 ** -10),
           np.ldexp(1.0, 128) * (1 - 2.0 ** -12), np.ldexp(1.0, -126), -np.ldexp(1.0, -126)]
    return np.concatenate([x, base, *ties, top])


def test_f64_to_bf16_bits():
    x = _inputs(1)
    got = dd.dd_convert_test(0, x)
    ref = (_nearest(x, 7, True).astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)
    bad = np.flatnonzero(got != ref)
    assert bad.size == 0, (x[bad[:5]], got[bad[:5]], ref[bad[:5]])


def test_f64_to_tf32():
    x = _inputs(2)
    got = dd.dd_convert_test(1, x)
    ref = _nearest(x, 10, False).astype(np.float32)
    bad = np.flatnonzero(got.view(np.uint32) != ref.view(np.uint32))
    assert bad.size == 0, (x[bad[:5]], got[bad[:5]], ref[bad[:5]])


def test_specials_round_like_the_hardware_path():
    x = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-300, -1e-300, 5e-324])
    b = dd.dd_convert_test(0, x)
    assert list(b[:4]) == [0x0000, 0x8000, 0x7F80, 0xFF80]
    assert (b[4] & 0x7F80) == 0x7F80 and (b[4] & 0x7F) != 0          # NaN stays NaN
    assert list(b[5:]) == [0x0000, 0x8000, 0x0000]
    t = dd.dd_convert_test(1, x)
    assert list(t[:4].view(np.uint32)) == [0, 0x80000000, 0x7F800000, 0xFF800000]
    assert np.isnan(t[4]) and list(t[5:].view(np.uint32)) == [0, 0x80000000, 0]


def test_f32_to_f64_exact():
    rng = np.random.default_rng(3)
    bits = rng.integers(0, 2 ** 32, 300_000, dtype=np.uint64).astype(np.uint32)
    f = bits.view(np.float32)
    f = np.concatenate([f, np.array([0.0, -0.0, np.inf, -np.inf, 1e-45, -1e-45, 3.4e38], np.float32)])
    got = dd.dd_convert_test(2, f)
    ref = f.astype(np.float64)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan].view(np.uint64), ref[~nan].view(np.uint64))
