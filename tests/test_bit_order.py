"""The largest change of a sweep (the ||u^n - u^(n-1)||_inf stop of Sec. 4.2.2)
is reduced on the device as an integer max over the binary64 bit patterns of
|u' - u| (sign bit cleared), not with FP64 compares.  This pins the IEEE-754
property that makes that exact: for non-negative doubles the patterns, read as
signed 64-bit integers, order like the values, and every NaN pattern lies
above +inf, so the integer max equals the largest |d| with a NaN kept."""
import numpy as np

MASK = np.int64(0x7FFFFFFFFFFFFFFF)


def bits_max(d):
    b = np.asarray(d, dtype=np.float64).view(np.int64) & MASK
    return np.int64(b.max()).view(np.float64)


def nan_keeping_max(d):
    a = np.abs(np.asarray(d, dtype=np.float64))
    return np.nan if np.isnan(a).any() else a.max()


SPECIAL = [0.0, -0.0, 5e-324, -5e-324, 2.2250738585072014e-308, 1e-10, -1e-10, 1.0, -3.5,
           1.7976931348623157e308, -1.7976931348623157e308, np.inf, -np.inf]


def test_patterns_order_like_values():
    rng = np.random.default_rng(0)
    v = np.concatenate([np.abs(SPECIAL),
                        np.exp(rng.uniform(-740, 709, 4000)),  # subnormal .. huge
                        rng.uniform(0, 1, 1000)])
    v = np.unique(v)  # sorted, -0.0 merged with 0.0
    b = v.view(np.int64) & MASK
    assert np.all(np.diff(b) > 0)


def test_integer_max_equals_largest_change():
    rng = np.random.default_rng(1)
    for trial in range(200):
        d = rng.standard_normal(rng.integers(1, 64)) * 10.0 ** rng.integers(-12, 3)
        if trial % 7 == 0:
            d[rng.integers(0, d.size)] = SPECIAL[trial % len(SPECIAL)]
        assert bits_max(d) == nan_keeping_max(d)


def test_nan_is_kept_whatever_its_sign_or_payload():
    payloads = [0x7FF8000000000000, 0xFFF8000000000000, 0x7FF0000000000001,
                0xFFFFFFFFFFFFFFFF]
    for p in payloads:
        nan = np.array([p], dtype=np.uint64).view(np.float64)[0]
        assert np.isnan(nan)
        got = bits_max([1.0, np.inf, nan, -2.0])
        assert np.isnan(got)
    # +inf beats every finite change; the empty reduction's 0 is the identity
    assert bits_max([np.inf, 1e308]) == np.inf
    assert bits_max([0.0]) == 0.0 and bits_max([-0.0]) == 0.0
