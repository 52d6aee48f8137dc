"""Analytics on compressed data (R19): the GPU aggregate of a stream, computed from its records
without writing the values, against the oracle's (decompress, then the definition): count and
NaN count exact, min / max bit-exact (totalOrder over non-NaN values), and the sum within the
bound of its summation tree, depth * 2^-53 * sum(|x|), depth = 38 + ceil(chunks / 1024) + 10
(each lane's 32 values + the value past 1024, 5 butterfly levels, each finishing thread's
chunks, 10 tree levels), equal to the oracle's where that is infinite or NaN."""
import math
import struct

import numpy as np
import pytest
import torch

from paper_2511_04140_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2511_04140_gb300 import build
    build.build()
    from paper_2511_04140_gb300 import falcon
    return falcon


def _bits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _same(a: float, b: float) -> bool:
    return (math.isnan(a) and math.isnan(b)) or _bits(a) == _bits(b)


def check(F, oracle, vals, block):
    s = oracle.compress(vals, block)
    got = F.aggregate(torch.frombuffer(bytearray(s), dtype=torch.uint8).cuda())
    want = oracle.aggregate(s)
    assert got["count"] == want["count"] == len(vals)
    assert got["nan_count"] == want["nan_count"]
    assert _same(got["min"], want["min"]) and _same(got["max"], want["max"])
    if math.isfinite(want["sum"]):
        with np.errstate(invalid="ignore"):         # NaN payloads widen with a warning
            ok = np.asarray(vals).astype(np.float64)
        ok = ok[~np.isnan(ok)]
        nc = (len(vals) + block - 1) // block
        depth = 38 + (nc + 1023) // 1024 + 10
        bound = depth * 2.0 ** -53 * math.fsum(np.abs(ok).tolist())
        assert abs(got["sum"] - want["sum"]) <= bound, (got["sum"], want["sum"], bound)
        if want["sum"] == 0.0 and bound == 0.0:
            assert _same(got["sum"], want["sum"])
    else:
        assert _same(got["sum"], want["sum"])
    return got


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("n,block", [(0, 1024), (1, 1024), (1023, 1024), (1025, 1025), (150_001, 1024),
                                     (20_011, 2), (70_000, 1000)])
def test_segments(F, oracle, dtype, n, block):
    check(F, oracle, synth.segments(n, seed=40 + n % 7, dtype=dtype), block)


@pytest.mark.parametrize("places", [0, 2, 5])
def test_case1_walks(F, oracle, places):
    check(F, oracle, synth.random_walk(200_003, seed=places, places=places), 1024)
    check(F, oracle, synth.random_walk(200_003, seed=places, places=places, dtype=np.float32), 1024)


def test_f16(F, oracle):
    check(F, oracle, synth.segments_f16(300_001, seed=3), 1024)
    every = np.arange(1 << 16, dtype=np.uint32).astype(np.uint16).view(np.float16)
    check(F, oracle, every, 1024)
    check(F, oracle, every, 3)


def test_edge_values(F, oracle):
    check(F, oracle, np.array([0.0, -0.0, 0.0]), 2)
    check(F, oracle, np.array([-0.0, -0.0, -0.0]), 1024)
    check(F, oracle, np.array([np.nan] * 5), 2)
    check(F, oracle, np.array([np.inf, 1.0, 2.0]), 1024)
    check(F, oracle, np.array([np.inf, -np.inf, 1.0]), 1024)
    check(F, oracle, np.array([1e16, 1.0, -1e16, 3.5]), 2)
    check(F, oracle, synth.adversarial_f64(), 1025)
    check(F, oracle, synth.adversarial_f32(), 65)


def test_matches_decompress_then_reduce(F):
    """On the GPU alone: the aggregate equals torch's reductions of the decompressed values
    (count, NaN count and min / max exactly; the sum within the same bound)."""
    vals = synth.segments(1 << 22, seed=9)
    x = torch.from_numpy(vals).cuda()
    s = F.compress(x, 1024)
    a = F.aggregate(s)
    y = F.decompress(s)
    ok = y[~torch.isnan(y)]
    assert a["count"] == y.numel() and a["nan_count"] == int(torch.isnan(y).sum())
    assert a["min"] == float(ok.min()) and a["max"] == float(ok.max())


def test_corrupt_stream_status(F, oracle):
    vals = synth.segments(10_000, seed=2)
    s = bytearray(oracle.compress(vals, 1024))
    nc = (len(vals) + 1023) // 1024
    rec0 = 32 + 4 * nc
    s[rec0 + 10] ^= 0xFF                          # inside the first record
    s[32:36] = (5).to_bytes(4, "little")           # and a size that cannot be right
    with pytest.raises(F.FalconError) as e:
        F.aggregate(torch.frombuffer(s, dtype=torch.uint8).cuda())
    assert e.value.status == F.ERR_CORRUPT


def test_async_form_and_graph(F, oracle):
    vals = synth.segments(100_000, seed=8)
    s = torch.frombuffer(bytearray(oracle.compress(vals, 1024)), dtype=torch.uint8).cuda()
    hdr = s[:32].cpu().numpy().tobytes()
    ws = torch.empty(F.workspace_bytes((len(vals) + 1023) // 1024), dtype=torch.uint8, device="cuda")
    st = torch.empty(F.STATS_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    F.aggregate_async(s, s.numel(), hdr, ws, st, stream)
    torch.cuda.synchronize()
    first = F.stats_of(st)
    assert first["status"] == 0 and first["count"] == len(vals)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        F.aggregate_async(s, s.numel(), hdr, ws, st, stream)
    st.zero_()
    g.replay()
    torch.cuda.synchronize()
    again = F.stats_of(st)
    assert all(_same(float(first[k]), float(again[k])) for k in ("min", "max", "sum"))
