"""CPU model of the FP64-by-digit-slices product scheme of the emulated Gram / V C
kernels, written with exact Python integers, checked against the properties the
kernels rely on:

* every per-scale partial sum of digit products over a window of 128 entries is an
  integer below 2^24, so the FP32 tensor-core accumulators hold it exactly (worst case:
  all digits 127, seven pairs on the middle scale);
* the combined window sum T = sum_{s<=4} I_s 2^(28-7s) + round((I_5 2^7 + I_6) / 2^14)
  stays below 2^50 (exact in int64, one rounding when converted to FP64);
* the emulated dot product of two vectors lies within the scheme's worst case
  (2^(Ex+Ey-46) per term, window exponents) and within the error model of the GPU
  tests (2^-45 * 128 * sum over windows of max|x| max|y|) of the exactly rounded result
  (math.fsum of error-free products), for data spanning many binades, zeros and sign
  mixes, and for the all-127-digit worst case;
* integer data of up to 15 bits is reproduced exactly.

Slicing rule (one exponent per row and 128-entry window): E with max|x| < 2^E (E = the
biased exponent of the maximum minus 1022), F = round(|x| 2^(49 - E)) clamped below
2^49, digits d_p = floor(F / 2^(42 - 7p)) mod 128 for p = 0..6 with the sign of x.
The 28 pairs with i + j <= 6 are kept.  No GPU and no library code.
"""
import math
import struct

import numpy as np
import pytest

WIN = 128


def _bits(x):
    return struct.unpack("<Q", struct.pack("<d", float(x)))[0]


def _window_exponent(xs):
    """E with max|x| < 2^E from the largest exponent field (None: all zero/subnormal)."""
    ex = max(((_bits(x) >> 52) & 0x7FF) for x in xs)
    return None if ex == 0 else ex - 1022


def _digits(x, E):
    """Seven signed 7-bit digits of x / 2^E rounded to 49 fraction bits."""
    u = _bits(x)
    ex = (u >> 52) & 0x7FF
    if E is None or ex == 0:
        return [0] * 7
    sh = 1026 + E - ex
    assert sh >= 4
    mant = (u & ((1 << 52) - 1)) | (1 << 52)
    f = (mant + (1 << (sh - 1))) >> sh if sh < 64 else 0
    f = min(f, (1 << 49) - 1)
    sign = -1 if (u >> 63) else 1
    return [sign * ((f >> (42 - 7 * p)) & 127) for p in range(7)]


def _window_sum(xw, yw):
    """(T, Ex, Ey): the window's combined integer sum in units of 2^(Ex + Ey - 42)."""
    Ex, Ey = _window_exponent(xw), _window_exponent(yw)
    if Ex is None or Ey is None:
        return 0, 0, 0
    dx = [_digits(x, Ex) for x in xw]
    dy = [_digits(y, Ey) for y in yw]
    I = [0] * 7
    for a, b in zip(dx, dy):
        for s in range(7):
            for i in range(s + 1):
                I[s] += a[i] * b[s - i]
    for s in range(7):
        assert abs(I[s]) < 2 ** 24            # exact in an FP32 accumulator
    T = sum(I[s] << (28 - 7 * s) for s in range(5))
    T += ((I[5] << 7) + I[6] + (1 << 13)) >> 14    # rounded (floor of +1/2)
    assert abs(T) < 2 ** 50
    return T, Ex, Ey


def emulated_dot(x, y):
    acc = 0.0
    for w0 in range(0, len(x), WIN):
        T, Ex, Ey = _window_sum(x[w0:w0 + WIN], y[w0:w0 + WIN])
        if T:
            acc += float(T) * 2.0 ** (Ex + Ey - 42)
    return acc


def exact_dot(x, y):
    """Correctly rounded sum of x_i y_i: each product split without error into p + e
    (Dekker), all parts summed exactly by math.fsum."""
    terms = []
    for a, b in zip(x, y):
        p = a * b
        # error-free product: a*b = p + e exactly (Dekker split)
        c = 134217729.0
        ah = c * a - (c * a - a)
        al = a - ah
        bh = c * b - (c * b - b)
        bl = b - bh
        e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
        terms += [p, e]
    return math.fsum(terms)


def model_bound(x, y):
    """The error model the GPU tests use: 2^-45 * 128 * sum over windows of
    max|x| max|y| (random data sits well inside it)."""
    b = 0.0
    for w0 in range(0, len(x), WIN):
        b += WIN * np.abs(x[w0:w0 + WIN]).max() * np.abs(y[w0:w0 + WIN]).max()
    return 2.0 ** -45 * b


def rigorous_bound(x, y):
    """Worst case from the scheme: per term, the digit rounding of both operands
    (2 * 2^(Ex+Ey-49)) plus the dropped pairs i + j >= 7 (6 pairs of at most 127^2 at
    2^(Ex+Ey-63), and less below) is under 2^(Ex+Ey-46); per window the combine
    rounds once (2^(Ex+Ey-43)); the FP64 accumulation of the windows adds its own."""
    b = 0.0
    for w0 in range(0, len(x), WIN):
        Ex, Ey = _window_exponent(x[w0:w0 + WIN]), _window_exponent(y[w0:w0 + WIN])
        if Ex is None or Ey is None:
            continue
        b += WIN * 2.0 ** (Ex + Ey - 46) + 2.0 ** (Ex + Ey - 43)
    return b + 4e-16 * float(np.abs(x) @ np.abs(y))


def test_worst_case_digits_fit_fp32_accumulators():
    # every digit 127 on both sides: the middle scale (s = 6) collects 7 pairs per row
    worst = WIN * 7 * 127 * 127
    assert worst < 2 ** 24
    x = np.full(WIN, np.nextafter(1.0, 0.0))      # F just below 2^49: all digits 127
    T, Ex, Ey = _window_sum(x, x)                   # asserts inside
    assert T > 0


@pytest.mark.parametrize("seed,spread", [(0, 0), (1, 10), (2, 40), (3, 300)])
def test_emulated_dot_within_error_model(seed, spread):
    rng = np.random.default_rng(seed)
    n = 3 * WIN + 57                                 # several windows and a ragged tail
    x = rng.standard_normal(n) * np.exp2(rng.integers(-spread, spread + 1, n))
    y = rng.standard_normal(n) * np.exp2(rng.integers(-spread, spread + 1, n))
    x[5] = 0.0
    y[WIN + 3] = -0.0
    got = emulated_dot(x, y)
    ref = exact_dot(x, y)
    assert abs(got - ref) <= rigorous_bound(x, y)
    assert abs(got - ref) <= model_bound(x, y)


def test_integer_data_is_exact():
    rng = np.random.default_rng(7)
    x = rng.integers(-2 ** 15, 2 ** 15, 2 * WIN + 9).astype(np.float64)
    y = rng.integers(-2 ** 15, 2 ** 15, 2 * WIN + 9).astype(np.float64)
    assert emulated_dot(x, y) == float(sum(int(a) * int(b) for a, b in zip(x, y)))


def test_zero_and_subnormal_windows_contribute_nothing():
    x = np.zeros(WIN)
    x[3] = 5e-324                                    # subnormal: flushed by the slicing
    y = np.ones(WIN)
    assert emulated_dot(x, y) == 0.0


def test_worst_case_digits_stay_inside_the_rigorous_bound():
    """All digits 127 (x just below 2^E) maximise the dropped pairs."""
    x = np.full(WIN, np.nextafter(1.0, 0.0))
    y = np.full(WIN, -np.nextafter(2.0, 0.0))
    assert abs(emulated_dot(x, y) - exact_dot(x, y)) <= rigorous_bound(x, y)


def test_a_missing_scale_is_seen():
    """A plausible mistake -- dropping the pairs of one scale -- moves the result by
    far more than the model allows, so the tests above would catch it."""
    rng = np.random.default_rng(11)
    x = rng.standard_normal(WIN)
    y = rng.standard_normal(WIN)
    Ex, Ey = _window_exponent(x), _window_exponent(y)
    dx = [_digits(a, Ex) for a in x]
    dy = [_digits(b, Ey) for b in y]
    for s in (4, 5):
        Is = sum(a[i] * b[s - i] for a, b in zip(dx, dy) for i in range(s + 1))
        missing = Is * 2.0 ** (Ex + Ey - 14 - 7 * s)   # that scale's contribution
        assert abs(missing) > 4 * model_bound(x, y)
