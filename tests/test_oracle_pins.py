"""Pins the CPU oracle to what the paper itself prints (tests/golden/paper_examples.txt)
and to the definitions it states, independently of the oracle's own code."""
import os
from decimal import Decimal

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_examples.txt")


def def_dp_ds(v: float):
    """Def. 1-2 read on the shortest round-trip decimal of v (Python's repr):
    DP = number of fractional digits, DS = DP + floor(log10|v|) + 1 (Eq. 2)."""
    if v == 0:
        return 0, 0
    d = Decimal(repr(float(v))).normalize()
    exp = d.as_tuple().exponent
    dp = max(0, -exp)
    return dp, dp + d.adjusted() + 1


def golden_lines():
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        body, cite = line.split("|", 1)
        lhs, rhs = body.split("->")
        kind, *args = lhs.split()
        yield kind, args, rhs.split(), cite.strip()


@pytest.mark.parametrize("kind,args,expected,cite", list(golden_lines()))
def test_paper_example(oracle, kind, args, expected, cite):
    if kind == "mul":
        v, i = float(args[0]), int(args[1])
        assert repr(v * oracle.pow10(i)) == repr(float(expected[0])), cite
    elif kind == "def":
        assert def_dp_ds(float(args[0])) == (int(expected[0]), int(expected[1])), cite
    elif kind == "alg2":
        assert oracle.dp_ds(float(args[0])) == (int(expected[0]), int(expected[1])), cite
    elif kind == "round":
        v, i = float(args[0]), int(args[1])
        assert round(v * oracle.pow10(i)) == int(expected[0]), cite
    elif kind == "roundtrip":
        v, i = float(args[0]), int(args[1])
        p = oracle.pow10(i)
        assert round(v * p) / p == float(expected[0]), cite
    elif kind == "chunk_g":
        vals = np.array([float(x) for x in args[0].split(",")])
        a, b, case1, g = oracle.chunk_transform(vals)
        assert case1, cite
        assert a == int(expected[0]), cite
        assert [int(np.int64(x)) for x in g.view(np.int64)] == \
            [int(x) for x in expected[1].split(",")], cite
    elif kind == "bits":
        assert int(args[0]).bit_length() == int(expected[0]), cite
    elif kind == "elf":
        assert oracle.dp_elf(float(args[0]))[0] == int(expected[0]), cite
    elif kind == "chunk_g_elf":
        vals = np.array([float(x) for x in args[0].split(",")])
        a, b, case1, g = oracle.chunk_transform(vals, elf=True)
        assert case1 and a == int(expected[0]), cite
        assert [int(np.int64(x)) for x in g.view(np.int64)] == \
            [int(x) for x in expected[1].split(",")], cite
    else:
        raise AssertionError(kind)


def test_alg2_exceptions_on_paper_counterexamples(oracle):
    # beta > 15: 111.00000000000001 (DS 17) and 9.110900773177071 (DS 16, Thm 2
    # counterexample) are exceptions; alpha = 23 (Thm 3 counterexample) as well.
    for v in (111.00000000000001, 9.110900773177071, 1.23456789876543e-9):
        a, b = oracle.dp_ds(v)
        assert a > 22 or b > 15, v


def test_fig8_bitmap_msb_first_and_row1_is_top_plane(oracle):
    """Fig. 8 (Sec. 3.3): n = 65 values, w = 10, and the bitmap of the first row of M^T
    is "10000000": only the first byte of the top bit plane is non-zero, so that row is
    stored sparse with bitmap byte 0b10000000."""
    rng = np.random.default_rng(7)
    z = rng.integers(0, 1 << 9, size=65).astype(np.uint64)   # planes 0..8
    z[0] = 12345                                              # z_1 is stored raw
    z[3] = (1 << 9) | 5                                       # the single value using plane 9
    rec = oracle.encode_z(z, oracle.F64, 2, 5)
    assert rec[0] == 2 and rec[1] == 5
    assert int.from_bytes(rec[2:10], "little") == 12345
    w = rec[10]
    assert w == 10
    flags = rec[11:13]                                        # ceil(10/8) = 2 flag bytes
    # row 1 (top plane) is sparse: its flag (first of the last 10 bits) is 0
    assert (flags[0] >> (7 - 6)) & 1 == 0
    row1 = rec[13:]
    assert row1[0] == 0b10000000                              # bitmap of (n-1)/64 = 1 byte
    # the non-zero byte: z_4 is column 2 -> bit 7-2 of byte 0
    assert row1[1] == 0b00100000


def test_storage_choice_is_minimum_cost(oracle):
    """Sec. 3.3: sparse cost (n-1)/64 + (n-1)/8 - lambda, dense cost (n-1)/8; the record
    length must equal the header plus the minimum per row (tie -> either; lengths equal)."""
    rng = np.random.default_rng(3)
    for trial in range(200):
        m = int(rng.integers(2, 300))
        nbits = int(rng.integers(1, 64))
        z = rng.integers(0, 1 << nbits, size=m, dtype=np.uint64)
        # make some planes sparse by zeroing most values' high bits
        mask = rng.random(m) < rng.random()
        z[mask] &= np.uint64((1 << max(nbits // 2, 1)) - 1)
        rec = oracle.encode_z(z, oracle.F64, 23, 16)
        cols = ((m - 1 + 63) // 64) * 64
        zz = np.zeros(cols, dtype=np.uint64)
        zz[:m - 1] = z[1:]
        w = int(max(int(x) for x in zz).bit_length()) if cols else 0
        expect = 2 + 8 + 1 + (w + 7) // 8
        for p in range(w):
            bits = ((zz >> np.uint64(p)) & np.uint64(1)).astype(np.uint8).reshape(-1, 8)
            nz_bytes = int(np.count_nonzero(bits.any(axis=1)))
            dense = cols // 8
            sparse = cols // 64 + nz_bytes
            expect += min(dense, sparse)
        assert len(rec) == expect, (m, nbits)
        assert rec[10] == w


def test_tie_goes_dense(oracle):
    """Sec. 3.3 selects sparse iff lambda > (n-1)/64; at equality the row is dense."""
    m = 65                                                    # 64 columns, 8 row bytes
    z = np.zeros(m, dtype=np.uint64)
    # plane 0: 7 non-zero bytes, lambda = 1 = (n-1)/64 -> dense
    for j in range(7):
        z[1 + 8 * j] = 1
    rec = oracle.encode_z(z, oracle.F64, 0, 0)
    assert rec[10] == 1
    assert rec[11] & 1 == 1                                  # dense flag
    assert len(rec) == 12 + 8
    # 6 non-zero bytes, lambda = 2 > 1 -> sparse: 1 bitmap byte + 6 bytes
    z[1 + 8 * 6] = 0
    rec = oracle.encode_z(z, oracle.F64, 0, 0)
    assert rec[11] & 1 == 0
    assert len(rec) == 12 + 1 + 6


def test_zigzag_closed_form(oracle):
    """Eq. 5: Zigzag maps x >= 0 to 2x and x < 0 to -2x-1 (as an unsigned word)."""
    rng = np.random.default_rng(0)
    vals = [0, 1, -1, 2, -2, 2 ** 63 - 1, -2 ** 63, 12345, -98765]
    vals += [int(x) for x in rng.integers(-2 ** 63, 2 ** 63 - 1, size=2000, dtype=np.int64)]
    for x in vals:
        expect = 2 * x if x >= 0 else -2 * x - 1
        assert oracle.zigzag64(x) == expect
        assert oracle.unzigzag64(expect) == x & 0xFFFFFFFFFFFFFFFF
    for x in [0, 1, -1, 2 ** 31 - 1, -2 ** 31] + [int(v) for v in rng.integers(-2 ** 31, 2 ** 31 - 1, size=500)]:
        expect = 2 * x if x >= 0 else -2 * x - 1
        assert oracle.zigzag32(x) == expect
        assert oracle.unzigzag32(expect) == x & 0xFFFFFFFF


def test_delta_is_modular(oracle):
    """Eq. 5 on Case-2 integers: differences wrap modulo 2^64 (R7) and invert exactly."""
    g = np.array([0, 2 ** 64 - 1, 1, 2 ** 63, 2 ** 63 - 1, 5], dtype=np.uint64)
    z = oracle.delta_zigzag(g, oracle.F64)
    assert z[0] == g[0]
    back = [int(g[0])]
    for i in range(1, len(g)):
        back.append((back[-1] + oracle.unzigzag64(int(z[i]))) % 2 ** 64)
    assert back == [int(x) for x in g]


def test_alg2_f32_spurious_early_pass(oracle):
    """With 24-bit significands the error bound of Thm 4 has no margin at beta = 7:
    fl32(0.001) - 1 ulp = 0.00099999993 passes eps <= mu already at alpha = 3 (x rounds
    to 1), the round trip 1/10^3 then fails, so Alg. 2 reports an exception."""
    v = np.nextafter(np.float32(0.001), np.float32(-1))
    assert oracle.dp_ds(v, np.float32) == (11, 8)
    a, b, case1, _ = oracle.chunk_transform(np.array([v], dtype=np.float32))
    assert not case1
