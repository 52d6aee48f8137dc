"""Pins of the oracle's aggregate (R19: analytics on compressed data, Sec. 7): count, NaN count,
min / max in IEEE 754 totalOrder over the non-NaN values, and their exact sum rounded once.
The sum is checked against Python's math.fsum (an independent correctly rounded summation),
min / max against numpy, and hand-worked cases pin the zeros, infinities and cancellation."""
import math
import struct

import numpy as np
import pytest


def _bits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def test_hand_worked(oracle):
    vals = np.array([1.5, -0.0, np.nan, 2.25, -3.0])
    a = oracle.aggregate(oracle.compress(vals, 1024))
    assert (a["count"], a["nan_count"], a["min"], a["max"], a["sum"]) == (5, 1, -3.0, 2.25, 0.75)


def test_zeros_in_total_order(oracle):
    a = oracle.aggregate(oracle.compress(np.array([0.0, -0.0, 0.0]), 2))
    assert _bits(a["min"]) == _bits(-0.0) and _bits(a["max"]) == _bits(0.0) and _bits(a["sum"]) == _bits(0.0)
    a = oracle.aggregate(oracle.compress(np.array([-0.0, -0.0]), 2))
    assert _bits(a["sum"]) == _bits(-0.0)


def test_exact_sum_cancels(oracle):
    a = oracle.aggregate(oracle.compress(np.array([1e16, 1.0, -1e16]), 1024))
    assert a["sum"] == 1.0                                  # a left-to-right FP64 sum gives 0.0
    a = oracle.aggregate(oracle.compress(np.full(10, 0.1), 1024))
    assert a["sum"] == 1.0 == math.fsum([0.1] * 10)


def test_infinities_and_nan_only(oracle):
    assert oracle.aggregate(oracle.compress(np.array([np.inf, 1.0]), 2))["sum"] == np.inf
    assert math.isnan(oracle.aggregate(oracle.compress(np.array([np.inf, -np.inf, 1.0]), 2))["sum"])
    a = oracle.aggregate(oracle.compress(np.array([np.nan, np.nan]), 2))
    assert a["nan_count"] == 2 and math.isnan(a["min"]) and math.isnan(a["max"]) and a["sum"] == 0.0
    a = oracle.aggregate(oracle.compress(np.zeros(0), 1024))
    assert a["count"] == 0 and math.isnan(a["min"])


@pytest.mark.parametrize("dtype", [np.float64, np.float32, np.float16])
def test_random_against_fsum_and_numpy(oracle, dtype):
    rng = np.random.default_rng(3)
    for n in (1, 1023, 5000, 70001):
        x = (rng.standard_normal(n) * 10.0 ** rng.integers(-3, 4, n)).astype(dtype)
        x[rng.random(n) < 0.01] = np.nan
        a = oracle.aggregate(oracle.compress(x, 1024))
        ok = x[~np.isnan(x)].astype(np.float64)
        assert a["count"] == n and a["nan_count"] == n - len(ok)
        assert a["sum"] == math.fsum(ok.tolist())
        if len(ok):
            assert a["min"] == ok.min() and a["max"] == ok.max()
