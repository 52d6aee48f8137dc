"""Properties the paper's theorems fix, checked on the CPU oracle.

Thm 2-4: for a decimal with DS <= 15 and DP <= 22, Alg. 2 returns exactly
(DP, DS) of that decimal; Thm 5: a Case-1 chunk decodes bit-exactly; the
codec as a whole is lossless on every bit pattern (specials included)."""
from decimal import Decimal

import numpy as np
import pytest

from paper_2511_04140_gb300 import synth


def shortest_dp_ds(v, f32=False):
    if v == 0:
        return 0, 0
    s = np.format_float_scientific(np.float32(v), unique=True) if f32 else repr(float(v))
    d = Decimal(s).normalize()
    dp = max(0, -d.as_tuple().exponent)
    return dp, dp + d.adjusted() + 1


def random_decimals(rng, count, max_ds, max_dp):
    """Random decimals with DS <= max_ds and DP <= max_dp, as (Decimal string)."""
    out = []
    while len(out) < count:
        ds = int(rng.integers(1, max_ds + 1))
        digits = int(rng.integers(10 ** (ds - 1), 10 ** ds))
        dp = int(rng.integers(0, max_dp + 1))
        sign = "-" if rng.random() < 0.5 else ""
        out.append(f"{sign}{digits}e-{dp}")
    return out


def test_alg2_returns_decimal_place_and_significand(oracle):
    """Thm 4 + Thm 3: for DS <= 15, DP <= 22 the enumeration stops exactly at DP and the
    round trip succeeds, so Alg. 2 yields (DP, DS) of the shortest decimal."""
    rng = np.random.default_rng(11)
    for s in random_decimals(rng, 20000, 15, 22):
        v = float(s)
        dp, ds = shortest_dp_ds(v)
        if ds > 15 or dp > 22:
            continue
        assert oracle.dp_ds(v) == (dp, ds), s


def test_alg2_flags_long_decimals(oracle):
    """Values with 16-17 significant digits (or DP > 22) are exceptions (alpha > 22 or
    beta > 15), so they can never reach Case 1."""
    rng = np.random.default_rng(12)
    vals = rng.standard_normal(5000) * 10.0 ** rng.uniform(-5, 8, size=5000)
    for v in vals:
        dp, ds = shortest_dp_ds(v)
        a, b = oracle.dp_ds(v)
        if ds > 15 or dp > 22:
            assert a > 22 or b > 15, v
        else:
            assert (a, b) == (dp, ds), v


def test_alg2_f32_small_significands(oracle):
    """FP32 analogue: for DS <= 6 (where the error-bound argument of Thm 4 carries over
    to 24-bit significands) Alg. 2 yields the shortest float decimal's (DP, DS)."""
    rng = np.random.default_rng(13)
    for s in random_decimals(rng, 20000, 6, 10):
        v = np.float32(float(Decimal(s)))
        dp, ds = shortest_dp_ds(v, f32=True)
        if ds > 6 or dp > 10:
            continue
        assert oracle.dp_ds(v, np.float32) == (dp, ds), s


def test_floor_log10_at_powers_of_ten(oracle):
    """R3: floor(log10|v|) is the largest k with |v| >= fl(10^k)."""
    from fractions import Fraction
    for k in range(-300, 300):
        p = float(Fraction(10) ** k)
        assert oracle.floor_log10(p) == k
        assert oracle.floor_log10(np.nextafter(p, np.inf)) == k
        assert oracle.floor_log10(np.nextafter(p, -np.inf)) == k - 1
    for k in range(-37, 38):
        p = np.float32(float(Fraction(10) ** k))
        if not np.isfinite(p) or p < np.finfo(np.float32).tiny:
            continue
        assert oracle.floor_log10(p, np.float32) == k
        assert oracle.floor_log10(np.nextafter(p, np.float32(np.inf)), np.float32) == k
        assert oracle.floor_log10(np.nextafter(p, np.float32(-np.inf)), np.float32) == k - 1


def test_thm2_case1_integers_are_the_decimal_digits(oracle):
    """Thm 2 / Thm 5: in Case 1, g_i = v_i * 10^alpha_max exactly (the decimal digits)."""
    rng = np.random.default_rng(14)
    for trial in range(300):
        m = int(rng.integers(1, 80))
        places = int(rng.integers(0, 8))
        digits = rng.integers(-10 ** 7, 10 ** 7, size=m)
        vals = np.array([float(Decimal(int(d)).scaleb(-places)) for d in digits])
        a, b, case1, g = oracle.chunk_transform(vals)
        assert case1
        expect_alpha = max(shortest_dp_ds(v)[0] for v in vals)
        assert a == expect_alpha
        scale = 10 ** (a - places) if a >= places else None
        for d, gi in zip(digits, g.view(np.int64)):
            if scale is not None:
                assert int(gi) == int(d) * scale
        assert np.array_equal(oracle.decompress(oracle.compress(vals, 64)).view(np.uint64),
                              vals.view(np.uint64))


def test_case_boundary_beta_hat_15(oracle):
    """Eq. 4: Case 1 iff alpha_max <= 22 and beta_hat_max <= 15."""
    a, b, case1, _ = oracle.chunk_transform(np.array([0.5, 12345678901234.0]))
    assert (a, b, case1) == (1, 15, True)
    a, b, case1, _ = oracle.chunk_transform(np.array([0.05, 12345678901234.0]))
    assert case1 is False and (a, b) == (23, 16)
    a, b, case1, _ = oracle.chunk_transform(np.array([1e-22, 0.0]))
    assert (a, b, case1) == (22, 1, True)
    a, b, case1, _ = oracle.chunk_transform(np.array([1e-23]))
    assert case1 is False
    a, b, case1, g = oracle.chunk_transform(np.zeros(5))
    assert (a, b, case1) == (0, 0, True) and not g.any()
    a, b, case1, _ = oracle.chunk_transform(np.array([0.0, -0.0]))
    assert case1 is False                                   # -0.0 is an exception (R1)


def test_f32_case_boundary(oracle):
    a, b, case1, _ = oracle.chunk_transform(np.array([0.5, 123456.0], dtype=np.float32))
    assert (a, b, case1) == (1, 7, True)
    a, b, case1, _ = oracle.chunk_transform(np.array([0.05, 123456.0], dtype=np.float32))
    assert case1 is False and (a, b) == (11, 8)


@pytest.mark.parametrize("block", [2, 3, 64, 65, 100, 1024, 1025])
def test_roundtrip_adversarial(oracle, block):
    for arr in (synth.adversarial_f64(), synth.adversarial_f32()):
        s = oracle.compress(arr, block)
        d = oracle.decompress(s)
        u = np.uint64 if arr.dtype == np.float64 else np.uint32
        assert np.array_equal(d.view(u), arr.view(u))


def test_roundtrip_random_bit_patterns(oracle):
    """Lossless on arbitrary bit patterns (NaN payloads, subnormals, any sign)."""
    rng = np.random.default_rng(21)
    a64 = rng.integers(0, 2 ** 64 - 1, size=50000, dtype=np.uint64).view(np.float64)
    a32 = rng.integers(0, 2 ** 32 - 1, size=50000, dtype=np.uint64).astype(np.uint32).view(np.float32)
    for arr, u in ((a64, np.uint64), (a32, np.uint32)):
        for block in (1024, 1025, 77):
            d = oracle.decompress(oracle.compress(arr, block))
            assert np.array_equal(d.view(u), arr.view(u))


def test_f32_exhaustive_sample(oracle):
    """A dense sweep of FP32 bit patterns (every 4099th pattern) as 1024-value blocks."""
    pats = np.arange(0, 2 ** 32, 4099, dtype=np.uint64).astype(np.uint32)
    arr = pats.view(np.float32)
    d = oracle.decompress(oracle.compress(arr, 1024))
    assert np.array_equal(d.view(np.uint32), pats)


def test_roundtrip_workloads(oracle):
    for arr in (synth.random_walk(20000, seed=0), synth.segments(40000, seed=1),
                synth.segments(40000, seed=1, dtype=np.float32),
                synth.random_walk(5000, places=3, outlier_rate=0.005)):
        u = np.uint64 if arr.dtype == np.float64 else np.uint32
        for block in (1024, 1025):
            d = oracle.decompress(oracle.compress(arr, block))
            assert np.array_equal(d.view(u), arr.view(u))


def test_random_walk_is_case1_and_compresses(oracle):
    arr = synth.random_walk(1 << 16, seed=0)
    s = oracle.compress(arr, 1024)
    recs = oracle.chunk_records(s)
    assert all(r[0] == 2 for r in recs)                     # alpha_max = 2 everywhere
    assert len(s) / arr.nbytes < 0.2


def test_empty_and_tiny(oracle):
    for n in (0, 1, 2, 3, 65, 66):
        arr = np.arange(n, dtype=np.float64) * 0.25
        s = oracle.compress(arr, 1024)
        assert np.array_equal(oracle.decompress(s), arr)
    assert len(oracle.compress(np.zeros(0), 1024)) == 32
    s = oracle.compress(np.array([3.5]), 1024)
    assert len(s) == 32 + 4 + 11                            # m = 1: w = 0, no flags, no rows


def test_eq5_worked_by_hand(oracle):
    """Eq. 5 by hand: g = (100, 103, 101, 101) -> z = (100, Zigzag(3), Zigzag(-2), Zigzag(0))
    = (100, 6, 3, 0); w = 3 bits, row 1 = plane 2 holds only z_2's bit (column 0)."""
    g = np.array([100, 103, 101, 101], dtype=np.uint64)
    z = oracle.delta_zigzag(g, oracle.F64)
    assert [int(x) for x in z] == [100, 6, 3, 0]
    rec = oracle.encode_z(z, oracle.F64, 0, 3)
    assert rec[10] == 3
    # 3 columns + 61 pads = 8 row bytes per plane, 7 of them zero: lambda = 7 > 64/64,
    # so every row is sparse: bitmap 0b10000000 followed by the single non-zero byte
    assert rec[11] == 0b00000000
    assert list(rec[12:]) == [0b10000000, 0b10000000,     # plane 2: bits of 6, 3, 0
                              0b10000000, 0b11000000,     # plane 1
                              0b10000000, 0b01000000]     # plane 0


def test_corruption_is_detected(oracle):
    arr = synth.random_walk(5000, seed=4)
    s = bytearray(oracle.compress(arr, 1024))
    assert oracle.decompress_status(bytes(s[:-1]))[0] == oracle.ERR_CORRUPT
    bad = bytearray(s); bad[0] = ord("X")
    assert oracle.decompress_status(bytes(bad))[0] == oracle.ERR_CORRUPT
    bad = bytearray(s); bad[32] ^= 0xFF                       # first size entry
    assert oracle.decompress_status(bytes(bad))[0] == oracle.ERR_CORRUPT
    data_start = 32 + 4 * 5
    bad = bytearray(s); bad[data_start + 10] = 200            # w > 64
    assert oracle.decompress_status(bytes(bad))[0] == oracle.ERR_CORRUPT
