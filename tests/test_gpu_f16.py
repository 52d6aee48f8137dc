"""GPU parity for binary16 (R18, FALCON_F16): every stream equals the oracle's byte for byte and
decodes to the input bits (tolerance 0 bits), through the single-stream entry points, the
ablation variants, the batched launch (FP16 mixed with FP64 and FP32), the host pipeline and
the server.  Every one of the 65,536 patterns goes through as values, in 1024-, 1025-, 3- and
2-value chunks; every Case-1 quotient g / 10^alpha (|g| < 1000, alpha <= 4) is decoded."""
from fractions import Fraction

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

ALL = np.arange(1 << 16, dtype=np.uint32).astype(np.uint16)


@pytest.fixture(scope="module")
def F():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2511_04140_gb300 import build
    build.build()
    from paper_2511_04140_gb300 import falcon
    return falcon


def _half(bits: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(bits.astype(np.uint16)).view(np.float16)


def decimals_f16(n: int, seed: int, places: int, amp: float = 30.0, outliers: float = 0.0) -> np.ndarray:
    """Random-walk values with `places` decimals, rounded to binary16 (a few full-precision
    outliers and specials when asked)."""
    rng = np.random.default_rng(seed)
    x = np.cumsum(rng.normal(0, amp / 20, n)) % (2 * amp) - amp
    v = np.round(x, places).astype(np.float16)
    if outliers:
        k = rng.random(n) < outliers
        v[k] = rng.integers(0, 1 << 16, int(k.sum()), dtype=np.uint32).astype(np.uint16).view(np.float16)
    return v


def check(F, oracle, vals, block, variant=0):
    x = torch.from_numpy(np.ascontiguousarray(vals)).cuda()
    s = F.compress_variant(x, block, variant) if variant else F.compress(x, block)
    got = s.cpu().numpy().tobytes()
    assert got == oracle.compress(vals, block, variant=variant), (block, variant)
    y = F.decompress(s)
    assert y.dtype == torch.float16
    assert np.array_equal(y.cpu().numpy().view(np.uint16), np.asarray(vals).view(np.uint16))
    return got


@pytest.mark.parametrize("block", [1024, 1025, 3, 2])
def test_every_pattern(F, oracle, block):
    vals = _half(ALL)
    check(F, oracle, vals, block)
    rng = np.random.default_rng(block)
    check(F, oracle, _half(rng.permutation(ALL)), block)


def test_every_case1_quotient(F, oracle):
    """Chunks of one decimal place each: fl16(g / 10^a) for every |g| < 1000 and a = 0..4."""
    parts = []
    for a in range(5):
        g = np.arange(-999, 1000)
        parts.append(np.array([float(Fraction(int(k), 10 ** a)) for k in g]).astype(np.float16))
    vals = np.concatenate([np.pad(p, (0, (-len(p)) % 1024), constant_values=np.float16(0)) for p in parts])
    check(F, oracle, vals, 1024)
    check(F, oracle, vals, 1000)


@pytest.mark.parametrize("places", [0, 1, 2, 3])
@pytest.mark.parametrize("block", [1024, 1025, 100])
def test_decimal_walks(F, oracle, places, block):
    check(F, oracle, decimals_f16(150_001, seed=places, places=places, outliers=0.001), block)


def test_unaligned_and_tails(F, oracle):
    vals = decimals_f16(70_003, seed=7, places=2)
    base = torch.from_numpy(np.concatenate([np.zeros(1, np.float16), vals])).cuda()
    x = base[1:]                                        # 2-byte aligned, not 16
    s = F.compress(x, 1024)
    assert s.cpu().numpy().tobytes() == oracle.compress(vals, 1024)
    out = torch.empty(len(vals) + 1, dtype=torch.float16, device="cuda")
    y = F.decompress(s, out=out[1:])
    assert np.array_equal(y.cpu().numpy().view(np.uint16), vals.view(np.uint16))
    for n in (0, 1, 2, 1023, 1025, 1026):
        check(F, oracle, vals[:n], 1024)


@pytest.mark.parametrize("variant", [1, 2, 3])
def test_variants(F, oracle, variant):
    check(F, oracle, decimals_f16(80_001, seed=11, places=2, outliers=0.002), 1024, variant)
    check(F, oracle, _half(ALL[::3]), 1025, variant)


def test_batch_mixed_dtypes(F, oracle):
    rng = np.random.default_rng(5)
    series = []
    for i in range(30):
        n = int(rng.integers(0, 50_000))
        kind = i % 3
        if kind == 0:
            series.append(decimals_f16(n, seed=100 + i, places=i % 4, outliers=0.001))
        elif kind == 1:
            series.append(np.round(rng.normal(0, 100, n), 2).astype(np.float32))
        else:
            series.append(np.round(rng.normal(0, 100, n), 3))
    xs = [torch.from_numpy(np.ascontiguousarray(s)).cuda() for s in series]
    b = F.Batch(F.COMPRESS, xs, block=1024)
    b.launch()
    torch.cuda.synchronize()
    streams = b.streams()
    for s, (nb, st), out in zip(series, b.results(), streams):
        assert st == 0 and out.cpu().numpy().tobytes() == oracle.compress(s, 1024)
    dec = F.Batch(F.DECOMPRESS, [(o, o.numel(), o[:32].cpu().numpy().tobytes()) for o in streams])
    dec.launch()
    torch.cuda.synchronize()
    for s, (nv, st), y in zip(series, dec.results(), dec.outputs):
        assert st == 0 and nv == len(s)
        w = {2: np.uint16, 4: np.uint32, 8: np.uint64}[s.dtype.itemsize]
        assert np.array_equal(y[:len(s)].cpu().numpy().view(w), s.view(w))
    b.close()
    dec.close()


def test_pipeline(F, oracle):
    vals = decimals_f16(300_007, seed=21, places=2, outliers=0.001)
    frame = 65_536
    s, fb = F.pipeline_compress(torch.from_numpy(vals).pin_memory(), block=1024, frame_values=frame, nstreams=4)
    blob = s.numpy().tobytes()
    off = 0
    for i, nb in enumerate(fb):
        assert blob[off:off + nb] == oracle.compress(vals[i * frame:(i + 1) * frame], 1024), i
        off += nb
    y = F.pipeline_decompress(s, fb, nstreams=4)
    assert y.dtype == torch.float16 and np.array_equal(y.numpy().view(np.uint16), vals.view(np.uint16))


def test_server(F, oracle):
    from paper_2511_04140_gb300.serve import Server
    vals = decimals_f16(123_457, seed=31, places=1)
    with Server(budget_bytes=1 << 30) as srv:
        s = srv.submit("compress", torch.from_numpy(vals)).result()
        assert s.numpy().tobytes() == oracle.compress(vals, 1024)
        y = srv.submit("decompress", s.clone()).result()
        assert y.dtype == torch.float16 and np.array_equal(y.numpy().view(np.uint16), vals.view(np.uint16))
