"""FP32 early stops of Alg. 2 (R14): a value stops early when eps <= mu passes at a decimal place
below its own and the round trip fails there (Alg. 2 then reports an exception).  With d / 10^k
the value's shortest decimal, v 10^a (a < k) lies at least 10^-(k-a) - |v| 10^a 2^-24 from every
integer, which exceeds mu = |v 10^a| 2^-23 unless |v| 10^k >= 2^23 / 1.5.  The GPU's FP32
analysis runs Alg. 2 value by value only for values with 3 |v| 10^alpha >= 2^23 (half that
bound), so the bound must hold for every value the oracle stops early.

Exhaustive over the values it matters for: every decimal d / 10^k with 3 d < 2^23 + 3 and
k = 0..10, rounded to FP32, with both FP32 neighbours (which covers every float whose shortest
decimal lies below the bound whatever the rounding of the conversion).  The oracle's Alg. 2
decides each value alone (a two-value chunk of the value twice); a value's decimal place k is
the first a with a round trip within Alg. 2's limits (a <= 10, a + floor(log10 |v|) + 1 <= 7)."""
import numpy as np
import pytest

pytestmark = pytest.mark.slow


def _oracle_alpha(oracle, v):
    """The alpha byte of each value's record: 11 means Alg. 2 reported an exception."""
    s = np.frombuffer(oracle.compress(np.repeat(v, 2), 2, threads=8), dtype=np.uint8)
    nc = len(v)
    sizes = s[32:32 + 4 * nc].view(np.uint32).astype(np.int64)
    off = 32 + 4 * nc + np.cumsum(sizes) - sizes
    return s[off]


def _decimal_place(v):
    """First a in 0..10 with fl32(round(v 10^a)) / fl32(10^a) == v (IEEE FP32 division) and
    a + floor(log10 v) + 1 <= 7; -1 if none (v > 0)."""
    v64 = v.astype(np.float64)
    e = np.floor(np.log10(v64)).astype(np.int64)
    k = np.full(len(v), -1, dtype=np.int64)
    for a in range(11):
        x = v64 * 10.0 ** a                        # exact: 24-bit significand times 10^a <= 10^10
        r = np.floor(x + 0.5)
        ok = (k < 0) & (r < 2 ** 24) & (a + e + 1 <= 7)
        back = r.astype(np.float32) / np.float32(10.0 ** a)
        k[ok & (back == v)] = a
    return k


def test_early_stops_need_the_bound(oracle):
    limit = (2 ** 23) // 3 + 2                     # every d with 3 d < 2^23 + 3
    early_total = 0
    smallest = np.inf
    for kk in range(11):
        d = np.arange(1, limit, dtype=np.float64)
        v = (d / 10.0 ** kk).astype(np.float32)
        v = np.unique(np.concatenate([v, np.nextafter(v, np.float32(0)), np.nextafter(v, np.float32(np.inf))]))
        v = v[v > 0]
        alpha = _oracle_alpha(oracle, v)
        k = _decimal_place(v)
        early = (alpha == 11) & (k >= 0)           # exception although a decimal place exists
        scaled = v[early].astype(np.float64) * 10.0 ** k[early]     # |v| 10^k, exact
        early_total += int(early.sum())
        if early.any():
            smallest = min(smallest, float(scaled.min()))
        # the bound itself (|v| 10^k >= 2^23 / 1.5), and so the kernel's half of it
        assert not np.any(1.5 * scaled < 2 ** 23), kk
    # early stops exist (the pinned example of Alg. 2 has one), all of them above the bound
    assert early_total > 0 and smallest >= 2 ** 23 / 1.5
