"""The exact FP64 <-> FP32 conversions of the sparse setup pass, built from IEEE
bit patterns with integer instructions (ipt_check_conversions), against numpy's
IEEE conversions, bit for bit: the two-float split hi = fl32(x), lo = fl32(x - hi),
the round-to-nearest-even x -> FP32 (ties to even, carries into the exponent) and
the exact FP32 -> FP64 conversion.  Inside the range the integer forms handle
(normal FP32 results, remainders with a normal FP32 scale) every flag is set;
outside it (subnormal, infinite, NaN, out of FP32 range) the flags are clear so
the solver falls back to the hardware conversion."""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def bits(a):
    return np.asarray(a).view(np.uint64 if np.asarray(a).dtype == np.float64 else np.uint32)


def make_inputs(seed):
    g = np.random.default_rng(seed)
    # random signs, exponents in [-70, 120], full random 52-bit mantissas
    e = g.integers(-70, 121, 20000)
    m = g.integers(0, 1 << 52, 20000, dtype=np.uint64)
    s = g.integers(0, 2, 20000, dtype=np.uint64)
    b = (s << np.uint64(63)) | ((e + 1023).astype(np.uint64) << np.uint64(52)) | m
    x = b.view(np.float64)
    # ties: the 29 bits below FP32 exactly half, with even and odd last FP32 bits,
    # and the carry case (all 23 FP32 mantissa bits set, rounding up)
    base = (np.uint64(1023 + 5) << np.uint64(52))
    ties = [base | (np.uint64(m23) << np.uint64(29)) | np.uint64(1 << 28)
            for m23 in (0, 1, 2, 3, 0x7ffffe, 0x7fffff)]
    near = [base | (np.uint64(0x7fffff) << np.uint64(29)) | np.uint64((1 << 28) + 1),
            base | (np.uint64(5) << np.uint64(29)) | np.uint64((1 << 28) - 1)]
    extra = np.array(ties + near, dtype=np.uint64).view(np.float64)
    plain = np.array([0.0, -0.0, 1.0, -1.0, 0.1, 1e-3, 123.456, 8192.125, 2.0 ** 100,
                      -2.0 ** -60])
    return np.concatenate([x, extra, -extra, plain])


def test_conversions_match_ieee(ipt):
    x = make_inputs(5)
    hi, lo, f, back, ok = ipt.check_conversions(torch.as_tensor(x, device="cuda"))
    hi, lo, f, back, ok = (t.cpu().numpy() for t in (hi, lo, f, back, ok))
    assert np.all(ok == 7)
    ref_f = x.astype(np.float32)
    np.testing.assert_array_equal(bits(f), bits(ref_f))
    np.testing.assert_array_equal(bits(hi), bits(ref_f))
    ref_lo = (x - ref_f.astype(np.float64)).astype(np.float32)
    np.testing.assert_array_equal(bits(lo), bits(ref_lo))
    np.testing.assert_array_equal(bits(back), bits(ref_f.astype(np.float64)))
    # the split keeps ~48 bits
    big = np.abs(x) > 0
    rel = np.abs(hi.astype(np.float64) + lo.astype(np.float64) - x)[big] / np.abs(x[big])
    assert np.max(rel) <= 2.0 ** -47


def test_conversions_flag_what_they_do_not_handle(ipt):
    x = np.array([np.inf, -np.inf, np.nan, 1e300, -1e300, 1e-310, 2.0 ** -130, 2.0 ** 128,
                  2.0 ** -80])
    _, _, _, _, ok = ipt.check_conversions(torch.as_tensor(x, device="cuda"))
    ok = ok.cpu().numpy()
    # infinite, NaN and out-of-range inputs: no rounding, no split
    assert np.all(ok[:8] & 3 == 0)
    # 2^-80 rounds to a normal FP32 value, but its remainder's scale is not normal
    assert ok[8] & 2 and not ok[8] & 1
