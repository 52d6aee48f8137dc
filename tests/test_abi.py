"""CPU-side checks of the C-ABI library: it loads, exports every entry point the header
declares, and its host-only functions agree with the oracle (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def falcon_lib():
    from paper_2511_04140_gb300 import build
    build.build()
    from paper_2511_04140_gb300 import falcon
    return falcon


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "falcon.h")).read()
    return sorted(set(re.findall(r"\b(falcon_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(falcon_lib):
    L = falcon_lib.lib()
    names = declared_symbols()
    assert "falcon_compress" in names and "falcon_decompress" in names and "falcon_bound" in names
    for name in names:
        assert hasattr(L, name), name
    assert L.falcon_abi_version() == 1


def test_bound_matches_oracle(falcon_lib, oracle):
    for n in (0, 1, 2, 63, 64, 65, 1023, 1024, 1025, 1 << 20, 67108864):
        for dt in (0, 1, 2):
            for blk in (2, 64, 1000, 1024, 1025):
                assert falcon_lib.bound(n, dt, blk) == oracle.bound(n, dt, blk), (n, dt, blk)
    assert falcon_lib.bound(10, 3, 1024) == 0 and oracle.bound(10, 3, 1024) == 0
    assert falcon_lib.bound(10, 0, 1) == 0
    for blk in (1026, 4096, 65537):                    # the format stops at n = 1025 (Sec. 3.3)
        assert falcon_lib.bound(10, 0, blk) == 0 and oracle.bound(10, 0, blk) == 0


def test_stream_info_parses_oracle_streams(falcon_lib, oracle):
    vals = np.linspace(0, 1, 3000)
    s = oracle.compress(vals, 1000)
    assert falcon_lib.stream_info(s[:32]) == (3000, 0, 1000, 3)
    s32 = oracle.compress(vals.astype(np.float32), 64)
    assert falcon_lib.stream_info(s32[:32]) == (3000, 1, 64, 47)
    bad = bytearray(s[:32]); bad[0] = 0
    with pytest.raises(falcon_lib.FalconError) as e:
        falcon_lib.stream_info(bytes(bad))
    assert e.value.status == falcon_lib.ERR_CORRUPT
    bad = bytearray(s[:32]); bad[24] ^= 1                    # num_chunks inconsistent with n
    with pytest.raises(falcon_lib.FalconError):
        falcon_lib.stream_info(bytes(bad))
    bad = bytearray(s[:32])                                  # block 4096, 1 chunk: outside the format
    bad[8:12] = (4096).to_bytes(4, "little"); bad[24:32] = (1).to_bytes(8, "little")
    with pytest.raises(falcon_lib.FalconError) as e:
        falcon_lib.stream_info(bytes(bad))
    assert e.value.status == falcon_lib.ERR_CORRUPT
    with pytest.raises(ValueError):
        oracle.decompress(bytes(bad) + bytes(4 + 20))


def test_workspace_bytes(falcon_lib):
    assert falcon_lib.workspace_bytes(0) == 256
    assert falcon_lib.workspace_bytes(1) == 512
    # two words per chunk, one per 64-chunk tile and one per 4096-chunk group, 256-byte granules
    words = 2 * 65536 + 1024 + 16
    assert falcon_lib.workspace_bytes(65536) == 256 + (8 * words + 255) // 256 * 256
