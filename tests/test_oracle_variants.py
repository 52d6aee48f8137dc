"""The oracle's ablation variants of Sec. 5.4.2 (Fal._Sparse, Fal._Dense, Fal._Elf) and its
multi-threaded drivers, pinned to what the paper and the definitions fix:
  - Fal._Dense stores every row as its cols/8 bytes, so a record's size has a closed form;
  - Sec. 3.3 picks the cheaper storage per row, so an adaptive record is never larger than
    the all-sparse or the all-dense one, and equals one of them when every row prefers it;
  - Fal._Elf's decimal place is never below Alg. 2's for values with DS <= 15 (the margin
    of Thm 4 rules out an integral product before the true decimal place), is 0 for integers,
    and its chunk alpha_max is never below Falcon's;
  - every variant decodes with the one decoder, bit for bit;
  - the multi-threaded drivers give the single-threaded bytes and values."""
import random
from decimal import Decimal

import numpy as np
import pytest

from paper_2511_04140_gb300 import synth


def records(oracle, stream):
    n, dt, blk, nc = oracle.stream_info(stream)
    recs = oracle.chunk_records(stream)
    ms = [min(blk, n - c * blk) for c in range(nc)]
    return dt, ms, recs


def flags_of(rec, z1b):
    w = rec[2 + z1b]
    fb = (w + 7) // 8
    bits = int.from_bytes(rec[3 + z1b:3 + z1b + fb], "big") if fb else 0
    return w, [(bits >> (w - 1 - r)) & 1 for r in range(w)]     # rows 1..w, 1 = dense


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_dense_variant_closed_form_and_sparse_variant_flags(oracle, dtype):
    vals = synth.segments(40_000, seed=5, dtype=dtype)
    z1b = 8 if dtype == np.float64 else 4
    for blk in (1024, 1025, 64, 100):
        _, ms, dense = records(oracle, oracle.compress(vals, blk, variant=oracle.DENSE))
        _, _, sparse = records(oracle, oracle.compress(vals, blk, variant=oracle.SPARSE))
        for m, rec in zip(ms, dense):
            cols = 0 if m <= 1 else (m - 1 + 63) // 64 * 64
            w, fl = flags_of(rec, z1b)
            assert all(fl)
            assert len(rec) == 3 + z1b + (w + 7) // 8 + w * cols // 8
        for rec in sparse:
            w, fl = flags_of(rec, z1b)
            assert not any(fl)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_adaptive_is_the_cheaper_storage_per_row(oracle, dtype):
    vals = synth.segments(60_000, seed=6, dtype=dtype)
    for blk in (1024, 1025):
        _, _, ad = records(oracle, oracle.compress(vals, blk))
        _, _, sp = records(oracle, oracle.compress(vals, blk, variant=oracle.SPARSE))
        _, _, de = records(oracle, oracle.compress(vals, blk, variant=oracle.DENSE))
        assert all(len(a) <= min(len(s), len(d)) for a, s, d in zip(ad, sp, de))
        assert sum(len(a) < min(len(s), len(d)) for a, s, d in zip(ad, sp, de)) > 0


def test_adaptive_equals_a_static_scheme_when_every_row_prefers_it(oracle):
    rng = np.random.default_rng(7)
    # random 52-bit deltas: no zero bytes below the top planes of the significand...
    noisy = np.frombuffer(rng.integers(1, 2**62, 4096, dtype=np.int64).tobytes(), dtype=np.float64)
    noisy = np.where(np.isfinite(noisy) & (np.abs(noisy) > 1e-300), noisy, 1.5)
    # ...and a chunk whose only non-zero delta bytes sit in a single column: every row sparse
    flat = np.full(1025, 3.25)
    flat[500] = 3.5
    assert oracle.compress(flat, 1025) == oracle.compress(flat, 1025, variant=oracle.SPARSE)
    s_ad = oracle.compress(noisy, 1024)
    assert len(s_ad) <= len(oracle.compress(noisy, 1024, variant=oracle.DENSE))


def test_sparse_variant_bound_is_reached_by_rows_without_zero_bytes(oracle):
    # Case 2 (a subnormal is an exception, R1) with G = Zigzag(BinLong(v)) alternating between
    # 2 and 2 + 2^63: every delta is 2^63, Zigzag(2^63) has all 64 bits set, so every row of
    # M^T is 128 non-zero bytes and each sparse row takes its 16-byte bitmap on top
    bits = np.zeros(1025, dtype=np.uint64)
    bits[::2] = np.uint64(1)                              # BinLong = 1 (5e-324), Zigzag -> 2
    bits[1::2] = np.uint64(0x4000000000000001)            # Zigzag -> 2 + 2^63
    vals = bits.view(np.float64)
    s = oracle.compress(vals, 1025, variant=oracle.SPARSE)
    assert len(s) == oracle.bound(1025, oracle.F64, 1025, oracle.SPARSE)
    assert len(oracle.compress(vals, 1025)) == oracle.bound(1025, oracle.F64, 1025)
    assert np.array_equal(oracle.decompress(s).view(np.uint64), bits)


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_every_variant_decodes_bit_exact(oracle, variant, dtype):
    u = np.uint64 if dtype == np.float64 else np.uint32
    for vals in (synth.segments(30_011, seed=8, dtype=dtype),
                 synth.random_walk(20_000, seed=9, places=3, dtype=dtype, outlier_rate=0.002),
                 np.tile(synth.adversarial_f64() if dtype == np.float64 else synth.adversarial_f32(), 20)):
        s = oracle.compress(vals, 1024, variant=variant)
        assert np.array_equal(oracle.decompress(s).view(u), vals.view(u))


def test_elf_decimal_place_is_never_below_alg2(oracle):
    rnd = random.Random(11)
    for _ in range(5000):
        ds = rnd.randint(1, 15)
        dp = rnd.randint(0, min(ds + 6, 22))
        digits = rnd.randint(10 ** (ds - 1), 10 ** ds - 1)
        v = float(Decimal(digits).scaleb(-dp) * (1 if rnd.random() < 0.5 else -1))
        a_alg2, _ = oracle.dp_ds(v)
        a_elf, _ = oracle.dp_elf(v)
        if a_alg2 <= 22:
            assert a_elf >= a_alg2, v
    for k in (0, 1, 7, 123456, -99999, 10**14):
        assert oracle.dp_elf(float(k))[0] == 0


def test_elf_chunk_alpha_is_never_below_falcon(oracle):
    vals = synth.random_walk(50_000, seed=12, places=2)
    more = 0
    for c in range(0, len(vals), 1024):
        a0, _, c0, _ = oracle.chunk_transform(vals[c:c + 1024])
        a1, _, c1, _ = oracle.chunk_transform(vals[c:c + 1024], elf=True)
        if c0 and c1:
            assert a1 >= a0
            more += a1 > a0
    assert more > 0                       # the imprecise decimal place does show up


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_multithreaded_drivers_match(oracle, dtype):
    for n in (0, 1, 1023, 1024, 1025, 5000, (1 << 17) + 3):
        vals = synth.segments(max(n, 1), seed=13, dtype=dtype)[:n]
        for blk in (1024, 1025, 2):
            if n > 20_000 and blk == 2:
                continue
            ref = oracle.compress(vals, blk)
            for t in (2, 3, 8, 64):
                assert oracle.compress(vals, blk, threads=t) == ref, (n, blk, t)
            back = oracle.decompress(ref, threads=5)
            assert back.tobytes() == vals.tobytes()
    vals = synth.random_walk(9000, seed=14, places=2, dtype=dtype)
    for variant in (1, 2, 3):
        assert oracle.compress(vals, 1024, variant=variant, threads=4) == oracle.compress(vals, 1024, variant=variant)
