"""Pins of the oracle's binary16 reading (R18: the method of Alg. 2, Eq. 4-5 and Sec. 3.3 with
FP16's constants: alpha <= 4, beta <= 3, mu = |x| 2^-10, fl16 round trip, sentinels (5, 4)).

The paper prints no FP16 example, so the pins come from the format and the mathematics:
numpy's exact float16 -> float64 conversion, nearest-value searches over exact rationals
(Fraction) for every rounded quotient and power of ten, every one of the 65,536 patterns for
the classification, the round trip and the minimality of Alg. 2's decimal place, Thm 4's
margin for short decimals, the early-stop bound, and a hand-worked chunk."""
from fractions import Fraction

import numpy as np
import pytest

ALL = np.arange(1 << 16, dtype=np.uint32).astype(np.uint16)
HALF = ALL.view(np.float16)


def _finite_sorted():
    """All finite non-negative binary16 values (patterns 0..0x7BFF) as exact Fractions."""
    pats = np.arange(0, 0x7C00, dtype=np.uint16)
    return pats, [Fraction(float(v)) for v in pats.view(np.float16)]


PATS, VALS = _finite_sorted()


def nearest_half(q: Fraction) -> int:
    """binary16 pattern nearest to q, ties to even, overflow to infinity: binary search over
    the sorted finite values (independent of the oracle's arithmetic)."""
    neg = q < 0
    a = -q if neg else q
    if a >= Fraction(65520):                       # halfway between 65504 and 2^16 rounds to inf
        return (0x8000 if neg else 0) | 0x7C00
    lo, hi = 0, len(VALS) - 1
    while lo < hi:                                 # first value >= a
        mid = (lo + hi) // 2
        if VALS[mid] < a:
            lo = mid + 1
        else:
            hi = mid
    i = lo
    if VALS[i] == a or i == 0:
        best = i
    else:
        d_lo, d_hi = a - VALS[i - 1], VALS[i] - a
        if d_lo < d_hi:
            best = i - 1
        elif d_hi < d_lo:
            best = i
        else:
            best = i if int(PATS[i]) % 2 == 0 else i - 1
    return (0x8000 if neg else 0) | int(PATS[best])


def test_half_to_double_is_exact(oracle):
    for u in range(0, 1 << 16, 7):
        want = float(np.uint16(u).view(np.float16))
        got = oracle.half_to_double(u)
        assert (np.isnan(want) and np.isnan(got)) or got == want, hex(u)


def test_pow10_f16_correctly_rounded(oracle):
    for k in range(-8, 5):
        q = Fraction(10) ** k
        assert int(np.float16(oracle.pow10(k, np.float16)).view(np.uint16)) == nearest_half(q), k
    assert np.isinf(oracle.pow10(5, np.float16))
    # 10^0..10^4 are exact in binary16
    assert [float(oracle.pow10(k, np.float16)) for k in range(5)] == [1.0, 10.0, 100.0, 1000.0, 10000.0]


def test_f16_div_pow10_correctly_rounded(oracle):
    for a in range(5):
        for g in list(range(-1100, 1101)) + [32767, -32768, 2049, 4097]:
            assert oracle.f16_div_pow10(g, a) == nearest_half(Fraction(g, 10 ** a)), (g, a)


def test_fp32_then_fp16_quotient_is_correctly_rounded(oracle):
    """The GPU decodes FP16 Case 1 as fl16(fl32(g / 10^a)): for every 16-bit g and a <= 4 that
    double rounding equals the correctly rounded fl16(g / 10^a) (numpy's FP32 division and
    FP32 -> FP16 conversion are IEEE round-to-nearest-even)."""
    g = np.arange(-32768, 32768, dtype=np.int64)
    for a in range(5):
        two_step = (g.astype(np.float32) / np.float32(10.0 ** a)).astype(np.float16).view(np.uint16)
        exact = np.array([oracle.f16_div_pow10(int(x), a) for x in g], dtype=np.uint16)
        assert np.array_equal(two_step, exact), a


def test_special_f16_every_pattern(oracle):
    f = HALF.astype(np.float64)
    sub = (ALL & 0x7C00 == 0) & (ALL & 0x3FF != 0)
    want = np.isnan(f) | np.isinf(f) | sub | (ALL == 0x8000)
    got = np.array([oracle.is_special(int(u), np.float16) for u in ALL])
    assert np.array_equal(got, want)


def test_floor_log10_f16_sweep(oracle):
    """R3 at every power of ten and its neighbours: the largest k with |v| >= fl16(10^k)."""
    for k in range(-4, 5):
        p = np.float16(oracle.pow10(k, np.float16))
        for v in (p, np.nextafter(p, np.float16(0)), np.nextafter(p, np.float16(np.inf))):
            if not np.isfinite(v) or v < np.float16(6.104e-05):
                continue
            want = max(j for j in range(-5, 5) if float(v) >= float(oracle.pow10(j, np.float16)))
            assert oracle.floor_log10(v, np.float16) == want, (k, float(v))


def test_zigzag16_closed_form(oracle):
    for x in list(range(-300, 300)) + [32767, -32768, -1, 0]:
        want = 2 * x if x >= 0 else -2 * x - 1
        assert oracle.zigzag16(x & 0xFFFF) == want
        assert oracle.unzigzag16(want) == x & 0xFFFF


def _dp_all(oracle):
    return np.array([oracle.dp_ds(int(u), np.float16) for u in ALL])


def test_alg2_f16_every_pattern(oracle):
    """For every pattern: specials are exceptions (5, 4); a reported decimal place round-trips
    (exact nearest search) and no smaller place does; beta = alpha + floor(log10|v|) + 1."""
    dp = _dp_all(oracle)
    for u, (a, b) in zip(ALL.tolist(), dp.tolist()):
        if oracle.is_special(u, np.float16):
            assert (a, b) == (5, 4)
            continue
        if u == 0:
            assert (a, b) == (0, 0)
            continue
        v = Fraction(float(np.uint16(u).view(np.float16)))
        if a <= 4 and b <= 3:
            assert nearest_half(Fraction(round(v * 10 ** a), 10 ** a)) == u, hex(u)
            for a2 in range(a):
                assert nearest_half(Fraction(round(v * 10 ** a2), 10 ** a2)) != u, hex(u)
            assert b == a + oracle.floor_log10(u, np.float16) + 1


def test_short_decimals_keep_their_place(oracle):
    """Thm 4's margin holds for beta <= 2 (10^2 * 1.5 * 2^-10 < 1): every decimal d / 10^k
    with at most two significant digits, rounded to binary16, gets alpha = k."""
    for k in range(0, 5):
        for d in range(1, 100):
            if d % 10 == 0 and k > 0:
                continue
            u = nearest_half(Fraction(d, 10 ** k))
            if (u & 0x7C00) == 0:                  # subnormal: an exception by R1
                continue
            assert oracle.dp_ds(u, np.float16)[0] == k, (d, k)
            assert oracle.dp_ds(u | 0x8000, np.float16)[0] == k, (-d, k)


def test_early_stops_need_the_bound(oracle):
    """An early stop (eps <= mu passes below the decimal place and the round trip fails) needs
    |v| 10^k >= 2^10 / 1.5, k the smallest round-tripping place; early stops exist."""
    dp = _dp_all(oracle)
    early = 0
    for u, (a, b) in zip(ALL.tolist(), dp.tolist()):
        if (a, b) != (5, 4) or oracle.is_special(u, np.float16) or u == 0:
            continue
        v = Fraction(float(np.uint16(u).view(np.float16)))
        e = oracle.floor_log10(u, np.float16)
        ks = [k for k in range(5) if k + e + 1 <= 3 and nearest_half(Fraction(round(v * 10 ** k), 10 ** k)) == u]
        if ks:
            early += 1
            assert abs(v) * 10 ** ks[0] * Fraction(3, 2) >= 2 ** 10, hex(u)
    assert early > 0


def test_hand_worked_f16_chunk(oracle):
    """[1.5, 2.25, -0.5]: places 1, 2, 1 -> alpha_max = 2; v_max = 2.25 -> beta_hat = 2 + 0 + 1
    = 3 <= 3: Case 1, G = (150, 225, -50), Z = (150, zz(75), zz(-275)) = (150, 150, 549)."""
    v = np.array([1.5, 2.25, -0.5], dtype=np.float16)
    a, b, case1, g = oracle.chunk_transform(v)
    assert (a, b, case1) == (2, 3, True)
    assert [int(x) for x in g] == [150, 225, (-50) & 0xFFFF]
    z = oracle.delta_zigzag(g, oracle.F16)
    assert [int(x) for x in z] == [150, 150, 549]
    # w = 10 (549 < 2^10); one 64-column row per plane (8 bytes, bitmap 1 byte), z_2 at
    # column 0 (bit 7 of row byte 0), z_3 at column 1 (bit 6); every row has 7 or 8 zero bytes,
    # more than cols/64 = 1, so every row is sparse (flags 0); planes 9 .. 0:
    #   150 = 0b0010010110, 549 = 0b1000100101
    rows = [0x40, 0x00, 0x80, 0x00, 0x40, 0x80, 0x00, 0xC0, 0x80, 0x40]
    body = b"".join(bytes([0x80, r]) if r else bytes([0x00]) for r in rows)
    want = bytes([2, 3, 150, 0, 10, 0x00, 0x00]) + body
    rec = oracle.encode_z(z, oracle.F16, a, b)
    assert rec == want
    assert oracle.decode_chunk(rec, 3, np.float16).view(np.uint16).tolist() == v.view(np.uint16).tolist()
    # 10.25 has beta = 2 + 1 + 1 = 4 > 3: an exception, Case 2 with G = zigzag16(bits)
    a, b, case1, g = oracle.chunk_transform(np.array([10.25, 1.0], dtype=np.float16))
    assert (a, b, case1) == (5, 4, False)
    assert int(g[0]) == oracle.zigzag16(int(np.float16(10.25).view(np.uint16)))


@pytest.mark.parametrize("block", [2, 1024, 1025])
def test_f16_codec_round_trip_every_pattern(oracle, block):
    s = oracle.compress(HALF, block)
    assert oracle.stream_info(s)[1] == oracle.F16
    back = oracle.decompress(s)
    assert back.dtype == np.float16 and np.array_equal(back.view(np.uint16), ALL)
    assert s == oracle.compress(HALF, block, threads=4)
