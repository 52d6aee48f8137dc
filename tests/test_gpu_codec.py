"""GPU parity: libfalcon's streams must equal the CPU oracle's byte for byte, and
decompression must give back every input bit (tolerance: 0 bits, the codec is lossless).
All calls go through the C ABI (ctypes binding)."""
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


def _u(arr):
    return arr.view(np.uint64 if arr.dtype == np.float64 else np.uint32)


def check_parity(F, oracle, vals, block):
    x = torch.from_numpy(np.ascontiguousarray(vals)).cuda()
    s = F.compress(x, block)
    got = s.cpu().numpy().tobytes()
    expect = oracle.compress(vals, block)
    if got != expect:
        # locate the first differing chunk for a readable failure
        n, dt, blk, nc = oracle.stream_info(expect)
        sz_e = np.frombuffer(expect, "<u4", nc, 32)
        sz_g = np.frombuffer(got, "<u4", nc, 32) if len(got) >= 32 + 4 * nc else None
        first_bad = None if sz_g is None else int(np.argmax(sz_e != sz_g)) if (sz_e != sz_g).any() else None
        raise AssertionError(f"stream mismatch: len {len(got)} vs {len(expect)}, first size mismatch at "
                             f"chunk {first_bad}, header ok={got[:32] == expect[:32]}")
    y = F.decompress(s)
    assert np.array_equal(_u(y.cpu().numpy()), _u(vals)), "round trip not bit-exact"
    # the GPU decoder also reads oracle-written streams
    s2 = torch.frombuffer(bytearray(expect), dtype=torch.uint8).cuda()
    y2 = F.decompress(s2)
    assert np.array_equal(_u(y2.cpu().numpy()), _u(vals))


@pytest.mark.parametrize("block", [1024, 1025, 64, 1000, 2, 77])
def test_random_walk(F, oracle, block):
    check_parity(F, oracle, synth.random_walk(200_003, seed=0), block)


def test_random_walk_full_size(F, oracle):
    """The 1,048,576-value, 2-place random walk in 1024-value blocks."""
    check_parity(F, oracle, synth.random_walk(1 << 20, seed=0), 1024)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("block", [1024, 1025, 333])
def test_segments(F, oracle, dtype, block):
    check_parity(F, oracle, synth.segments(300_001, seed=1, dtype=dtype), block)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_adversarial(F, oracle, dtype):
    arr = synth.adversarial_f64() if dtype == np.float64 else synth.adversarial_f32()
    for block in (2, 3, 64, 65, 1024, 1025):
        check_parity(F, oracle, arr, block)
    # each adversarial value alone, and next to ordinary decimals
    for v in arr:
        check_parity(F, oracle, np.array([v], dtype=dtype), 1024)
        mix = np.array([0.5, 1.25, v, 3.75], dtype=dtype)
        check_parity(F, oracle, mix, 1024)


@pytest.mark.parametrize("n", [0, 1, 2, 31, 32, 33, 63, 64, 65, 1023, 1024, 1025, 1026, 2049])
def test_sizes_and_tails(F, oracle, n):
    for dtype in (np.float64, np.float32):
        vals = synth.random_walk(n, seed=n, places=3, dtype=dtype)
        for block in (1024, 1025):
            check_parity(F, oracle, vals, block)


def test_random_bit_patterns(F, oracle):
    rng = np.random.default_rng(5)
    a64 = rng.integers(0, 2 ** 64 - 1, size=100_000, dtype=np.uint64).view(np.float64)
    a32 = rng.integers(0, 2 ** 32 - 1, size=100_000, dtype=np.uint64).astype(np.uint32).view(np.float32)
    for arr in (a64, a32):
        for block in (1024, 1025):
            check_parity(F, oracle, arr, block)


def _decimal_chunks(rng, nchunks, block, dtype):
    """Chunks of decimals with per-chunk decimal places and magnitudes spread over the
    whole Case-1 range (alpha 0..22, beta_hat up to 15 and just beyond)."""
    out = []
    amax, smax = (22, 15) if dtype == np.float64 else (10, 7)
    for c in range(nchunks):
        places = int(rng.integers(0, amax + 2))
        sig = int(rng.integers(1, smax + 2))
        hi = 10 ** sig
        k = rng.integers(-hi + 1, hi, size=block)
        if rng.random() < 0.3:
            k[rng.integers(0, block)] = 0
        pl = np.minimum(places, 22)
        vals = synth.decimal_to_f64(k, pl) if dtype == np.float64 else synth.decimal_to_f32(k, min(pl, 10))
        if rng.random() < 0.2:                        # one value nudged off its decimal
            i = int(rng.integers(0, block))
            vals[i] = np.nextafter(vals[i], dtype(np.inf))
        if rng.random() < 0.1:                        # one value with a different place count
            i = int(rng.integers(0, block))
            vals[i] = vals[i] * dtype(10.0) if rng.random() < 0.5 else vals[i] / dtype(10.0)
        out.append(vals.astype(dtype))
    return np.concatenate(out)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_case1_decisions_across_alpha(F, oracle, dtype):
    """Alg. 2 / Eq. 4 decisions at every alpha and at the beta_hat boundary."""
    rng = np.random.default_rng(17)
    vals = _decimal_chunks(rng, 600, 1024, dtype)
    check_parity(F, oracle, vals, 1024)
    recs = oracle.chunk_records(oracle.compress(vals, 1024))
    alphas = {r[0] for r in recs}
    assert len(alphas) > 10                           # many decimal places exercised


def test_unaligned_input(F, oracle):
    vals = synth.random_walk(10_001, seed=3, places=1)
    x = torch.from_numpy(vals).cuda()[1:]              # 8-byte aligned, not 16
    s = F.compress(x, 1024)
    assert s.cpu().numpy().tobytes() == oracle.compress(vals[1:], 1024)
    f = synth.segments(10_001, seed=3, dtype=np.float32)
    xf = torch.from_numpy(f).cuda()[3:]
    assert F.compress(xf, 1025).cpu().numpy().tobytes() == oracle.compress(f[3:], 1025)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_config2_full_size(F, oracle, dtype):
    """67,108,864 values of the segment workload: full stream equality and round trip."""
    vals = synth.segments(1 << 26, seed=1, dtype=dtype)
    check_parity(F, oracle, vals, 1024)


def test_capacity_error(F):
    vals = synth.segments(100_000, seed=2)
    x = torch.from_numpy(vals).cuda()
    out = torch.empty(50_000, dtype=torch.uint8, device="cuda")
    with pytest.raises(F.FalconError) as e:
        F.compress(x, 1024, out=out)
    assert e.value.status == F.ERR_CAPACITY
    out = torch.empty(100, dtype=torch.uint8, device="cuda")
    with pytest.raises(F.FalconError) as e:
        F.compress(x, 1024, out=out)
    assert e.value.status == F.ERR_CAPACITY


def test_block_size_outside_format_is_invalid(F):
    x = torch.zeros(10, dtype=torch.float64, device="cuda")
    for blk in (1026, 4096, 65537):
        with pytest.raises(F.FalconError) as e:
            F.compress(x, blk)
        assert e.value.status == F.ERR_INVALID
    with pytest.raises(F.FalconError) as e:
        F.compress(x, 1)
    assert e.value.status == F.ERR_INVALID


def test_corrupt_streams(F, oracle):
    vals = synth.random_walk(50_000, seed=4)
    good = bytearray(oracle.compress(vals, 1024))
    nc = (len(vals) + 1023) // 1024
    data_start = 32 + 4 * nc
    cases = {
        "truncated": bytes(good[:-1]),
        "magic": bytes(b"XLCN" + good[4:]),
        "size_entry": bytes(good[:32] + (int.from_bytes(good[32:36], "little") + 5).to_bytes(4, "little") + good[36:]),
        "w_too_large": bytes(good[:data_start + 10] + bytes([200]) + good[data_start + 11:]),
        "huge_size": bytes(good[:36] + (0xFFFFFFF0).to_bytes(4, "little") + good[40:]),
    }
    for name, blob in cases.items():
        st_o, _ = oracle.decompress_status(blob)
        assert st_o == oracle.ERR_CORRUPT, name
        s = torch.frombuffer(bytearray(blob), dtype=torch.uint8).cuda()
        with pytest.raises(F.FalconError) as e:
            F.decompress(s)
        assert e.value.status == F.ERR_CORRUPT, name
    # the context is still healthy
    check_parity(F, oracle, vals[:5000], 1024)


def test_async_and_graph_capture(F, oracle):
    vals = synth.segments(200_000, seed=6)
    x = torch.from_numpy(vals).cuda()
    nc = (len(vals) + 1023) // 1024
    cap = F.bound(len(vals), F.F64, 1024)
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    ws = torch.zeros(F.workspace_bytes(nc), dtype=torch.uint8, device="cuda")
    res = torch.zeros(2, dtype=torch.int64, device="cuda")
    expect = oracle.compress(vals, 1024)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        F.compress_async(x, 1024, out, ws, res, stream)
    stream.synchronize()
    nbytes, status = (int(v) for v in res.cpu())
    assert status == 0 and nbytes == len(expect)
    assert out[:nbytes].cpu().numpy().tobytes() == expect
    # capture compress + decompress in one graph and replay it twice
    y = torch.empty_like(x)
    ws2 = torch.zeros_like(ws)
    res2 = torch.zeros(2, dtype=torch.int64, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        F.compress_async(x, 1024, out, ws, res, stream)
        F.decompress_async(out, nbytes, expect[:32], y, ws2, res2, stream)
    for _ in range(2):
        out.zero_()
        y.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert out[:nbytes].cpu().numpy().tobytes() == expect
        assert int(res2[1]) == 0 and int(res2[0]) == len(vals)
        assert np.array_equal(y.cpu().numpy().view(np.uint64), vals.view(np.uint64))


def test_corrupt_size_in_a_long_stream(F, oracle):
    """A stream long enough for whole 32-tile groups in the offsets scan (4096 chunks): a huge
    size entry (only a malformed stream has one) must still be reported as corrupt."""
    vals = synth.random_walk(1 << 22, seed=8)
    good = bytearray(oracle.compress(vals, 1024))
    for chunk in (5, 2100, 4095):
        blob = bytearray(good)
        blob[32 + 4 * chunk:36 + 4 * chunk] = (0xFFFFFFF0).to_bytes(4, "little")
        st_o, _ = oracle.decompress_status(bytes(blob))
        assert st_o == oracle.ERR_CORRUPT, chunk
        s = torch.frombuffer(blob, dtype=torch.uint8).cuda()
        with pytest.raises(F.FalconError) as e:
            F.decompress(s)
        assert e.value.status == F.ERR_CORRUPT, chunk
    s = torch.frombuffer(good, dtype=torch.uint8).cuda()
    y = F.decompress(s)
    assert np.array_equal(_u(y.cpu().numpy()), _u(vals))


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_degenerate_series(F, oracle, dtype):
    """Series whose chunks sit at the method's corners: all zeros and a constant (w = 0),
    alternating signs (every row dense), consecutive integers (Case 1 at alpha = 0) and NaN
    only (every chunk Case 2), each with a ragged tail."""
    n = 5 * 1024 + 17
    cases = {
        "zeros": np.zeros(n, dtype=dtype),
        "constant": np.full(n, 3.14, dtype=dtype),
        "alternating": np.where(np.arange(n) % 2 == 0, 1.5, -1.5).astype(dtype),
        "integers": np.arange(n).astype(dtype),
        "nan": np.full(n, np.nan, dtype=dtype),
    }
    for name, vals in cases.items():
        for block in (1024, 1025, 64):
            check_parity(F, oracle, vals, block)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_more_than_32_chunk_groups(F, oracle, dtype):
    """More than 32 groups of 4096 chunks (2-value blocks, 163,842 chunks): record offsets past
    the first 32 groups are added in 64 bits, and every offset still equals the oracle's."""
    vals = synth.segments(2 * 40 * 4096 + 3, seed=12, dtype=dtype)
    check_parity(F, oracle, vals, 2)
