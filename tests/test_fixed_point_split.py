"""The fixed-point split of the particle kernel's deposit, replayed in numpy
FP32 with the constants read from the kernel header (FX_SHIFT, FX_SCALE,
GPD_PPT_MAX in csrc/qpic_internal.h).

A contribution x becomes t = x * (qscale 2^-FX_SHIFT) in FP32; the kernel
takes hi = round(t) from the bit pattern of t + 1.5 2^23, r = t - hi (exact),
and lo = round(r 2^FX_SHIFT) from the bit pattern of r 2^FX_SHIFT + 1.5 2^23;
before the parts reach the shared planes lo is carried into hi so that it lies
in [0, 2^FX_SHIFT).  Checked here, on random, extreme and tie-heavy inputs:
  - hi 2^FX_SHIFT + lo is the round-to-nearest-even integer of t 2^FX_SHIFT
    (the same integer the int64 global path adds);
  - the carry keeps the value and puts lo in [0, 2^FX_SHIFT);
  - a chunk of GPD_PPT_MAX x 256 contributions of the largest size (2 qref,
    plus FP32 rounding) keeps the signed hi sum and the unsigned lo sum
    inside 32 bits.
"""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2303_12874_gb300", "csrc", "qpic_internal.h")
M = np.float32(12582912.0)            # 1.5 * 2^23
MBITS = 0x4B400000


def _constants():
    src = open(HDR).read()
    shift = int(re.search(r"constexpr int FX_SHIFT = (\d+);", src).group(1))
    expr = re.search(r"constexpr double FX_SCALE = ([0-9.eE+\-*/() ]+);", src).group(1)
    assert re.fullmatch(r"[0-9.eE+\-*/() ]+", expr)
    scale = float(eval(expr, {"__builtins__": {}}))
    ppt = int(re.search(r"constexpr int GPD_PPT_MAX = (\d+);", src).group(1))
    return shift, scale, ppt


def _bits(a):
    return a.astype(np.float32).view(np.int32).astype(np.int64)


def _split(x, q_down, shift):
    """the kernel's FP32 operations, lane by lane"""
    t = (x.astype(np.float32) * np.float32(q_down)).astype(np.float32)
    tm = (t + M).astype(np.float32)
    hi = _bits(tm) - MBITS
    hf = (tm - M).astype(np.float32)
    r = (t - hf).astype(np.float32)                       # exact
    lm = (r * np.float32(2.0 ** shift) + M).astype(np.float32)   # r 2^shift is exact
    lo = _bits(lm) - MBITS
    return t, hi, lo


def _carry(hi, lo, shift):
    return hi + (lo >> shift), lo & ((1 << shift) - 1)


def _inputs(qref, rng):
    n = 200000
    x = np.concatenate([
        rng.uniform(-2, 2, n) * qref,                               # the full range
        rng.uniform(-1e-3, 1e-3, n) * qref,                         # small contributions
        np.array([2.0, -2.0, 2.0 * (1 + 2 ** -22), -2.0 * (1 + 2 ** -22), 0.0, 1e-30]) * qref,
    ])
    return x


def test_split_is_the_rounded_integer_and_the_carry_keeps_it():
    shift, scale, _ = _constants()
    rng = np.random.default_rng(11)
    for qref in (1.0, 3.7e-5, 0.125):
        q_down = np.float32(np.float32(scale / qref) * np.float32(2.0 ** -shift))
        x = _inputs(qref, rng)
        t, hi, lo = _split(x, q_down, shift)
        exact = np.rint(t.astype(np.float64) * 2.0 ** shift).astype(np.int64)   # ties to even
        assert np.array_equal(hi * (1 << shift) + lo, exact)
        assert np.all(np.abs(lo) <= 1 << (shift - 1))
        h2, l2 = _carry(hi, lo, shift)
        assert np.array_equal(h2 * (1 << shift) + l2, exact)
        assert np.all((l2 >= 0) & (l2 < 1 << shift))


def test_ties_round_to_even():
    shift, _, _ = _constants()
    # t with a fractional part of exactly one half at the scale 2^-shift
    k = np.arange(-2000, 2000, dtype=np.float64)
    t = ((k + 0.5) * 2.0 ** -shift).astype(np.float32)
    _, hi, lo = _split(t, np.float32(1.0), shift)
    v = hi * (1 << shift) + lo
    assert np.array_equal(v, np.rint(t.astype(np.float64) * 2.0 ** shift).astype(np.int64))
    assert np.all(v % 2 == 0)


def test_a_full_chunk_of_the_largest_contributions_fits_32_bits():
    shift, scale, ppt = _constants()
    chunk = 256 * ppt
    qref = 1.0
    q_down = np.float32(np.float32(scale / qref) * np.float32(2.0 ** -shift))
    # the largest contribution, with a generous FP32 excess
    x = np.array([2.0 * (1 + 2 ** -20), -2.0 * (1 + 2 ** -20)]) * qref
    _, hi, lo = _split(x, q_down, shift)
    h2, l2 = _carry(hi, lo, shift)
    assert np.abs(hi).max() <= (1 << 19) - 511
    # each contribution adds at most once per node and chunk: worst case all alike
    assert chunk * (int(np.abs(h2).max()) + 1) < 2 ** 31
    assert chunk * ((1 << shift) - 1) < 2 ** 32
    # the same bound a 2^40 scale would break (the split the chunks outgrew)
    _, hi40, _ = _split(x, np.float32(2.0 ** 40 * 2.0 ** -shift), shift)
    assert chunk * int(np.abs(hi40).max()) >= 2 ** 31
