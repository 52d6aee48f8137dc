"""Writes falcon_tables.h: the constants the CUDA kernels need, computed from exact
rational arithmetic (Python's Fraction -> float conversion rounds exactly once).

  FALCON_POW5[a]          5^a for a = 0..22 (exact integers)
  FALCON_RECIP5[a]        floor(2^(64 + d) / 5^a) with d = floor(log2 5^a), a = 1..22 (a 64-bit
                          reciprocal in [2^63, 2^64); entry 0 unused)
  FALCON_LOG2_POW5[a]     d = floor(log2 5^a)
  FALCON_POW5_NORM[a]     5^a << (63 - d): 5^a with its top bit at bit 63
  FALCON_P10_F64[k - LO]  bits of fl64(10^k), k in [-30, 22]
  FALCON_P10_F32[k - LO]  bits of fl32(10^k), k in [-15, 10]
  FALCON_P10_F16[k - LO]  bits of fl16(10^k) (binary16), k in [-8, 4]

Run: python gen_tables.py > falcon_tables.h
"""
import struct
from fractions import Fraction

F64_LO, F64_HI = -30, 22
F32_LO, F32_HI = -15, 10
F16_LO, F16_HI = -8, 4


def f64_bits(q: Fraction) -> int:
    return struct.unpack("<Q", struct.pack("<d", float(q)))[0]


def f32_nearest_bits(q: Fraction) -> int:
    """Bits of the FP32 value nearest to q (ties to even), found without double rounding."""
    d = float(q)
    b = struct.unpack("<I", struct.pack("<f", d))[0]
    best = None
    for cand in (b - 1, b, b + 1):
        val = Fraction(struct.unpack("<f", struct.pack("<I", cand))[0])
        err = abs(val - q)
        key = (err, cand & 1)
        if best is None or key < best[0]:
            best = (key, cand)
    return best[1]


def f16_nearest_bits(q: Fraction) -> int:
    """Bits of the binary16 value nearest to q (ties to even), without double rounding."""
    b = struct.unpack("<H", struct.pack("<e", float(q)))[0]
    best = None
    for cand in (b - 1, b, b + 1):
        if not 0 <= cand <= 0x7BFF:                    # finite non-negative patterns only
            continue
        val = Fraction(struct.unpack("<e", struct.pack("<H", cand))[0])
        key = (abs(val - q), cand & 1)
        if best is None or key < best[0]:
            best = (key, cand)
    return best[1]


def main():
    out = ["/* Generated by gen_tables.py -- exact constants for the Falcon kernels. */",
           "#pragma once", "#include <stdint.h>", "",
           "#ifndef FALCON_TABLE_QUAL", "#define FALCON_TABLE_QUAL static const", "#endif", "",
           f"#define FALCON_P10_F64_LO ({F64_LO})", f"#define FALCON_P10_F64_HI ({F64_HI})",
           f"#define FALCON_P10_F32_LO ({F32_LO})", f"#define FALCON_P10_F32_HI ({F32_HI})",
           f"#define FALCON_P10_F16_LO ({F16_LO})", f"#define FALCON_P10_F16_HI ({F16_HI})", "",
           "FALCON_TABLE_QUAL uint64_t FALCON_POW5[23] = {"]
    out += [f"    0x{5 ** a:016x}ull, /* 5^{a} */" for a in range(23)]
    out += ["};", "", "FALCON_TABLE_QUAL uint64_t FALCON_RECIP5[23] = {"]
    out += [f"    0x{(0 if a == 0 else (1 << (64 + (5 ** a).bit_length() - 1)) // 5 ** a):016x}ull, /* 5^{a} */"
            for a in range(23)]
    out += ["};", "", "FALCON_TABLE_QUAL uint64_t FALCON_POW5_NORM[23] = {"]
    out += [f"    0x{(5 ** a) << (64 - (5 ** a).bit_length()):016x}ull, /* 5^{a} */" for a in range(23)]
    out += ["};", "", "FALCON_TABLE_QUAL uint8_t FALCON_LOG2_POW5[23] = {"]
    out += ["    " + ", ".join(str((5 ** a).bit_length() - 1) for a in range(23))]
    out += ["};", "", f"FALCON_TABLE_QUAL uint64_t FALCON_P10_F64[{F64_HI - F64_LO + 1}] = {{"]
    out += [f"    0x{f64_bits(Fraction(10) ** k):016x}ull, /* fl64(1e{k}) */"
            for k in range(F64_LO, F64_HI + 1)]
    out += ["};", "", f"FALCON_TABLE_QUAL uint32_t FALCON_P10_F32[{F32_HI - F32_LO + 1}] = {{"]
    out += [f"    0x{f32_nearest_bits(Fraction(10) ** k):08x}u, /* fl32(1e{k}) */"
            for k in range(F32_LO, F32_HI + 1)]
    out += ["};", "", f"FALCON_TABLE_QUAL uint16_t FALCON_P10_F16[{F16_HI - F16_LO + 1}] = {{"]
    out += [f"    0x{f16_nearest_bits(Fraction(10) ** k):04x}u, /* fl16(1e{k}) */"
            for k in range(F16_LO, F16_HI + 1)]
    out += ["};", ""]
    print("\n".join(out))


if __name__ == "__main__":
    main()
