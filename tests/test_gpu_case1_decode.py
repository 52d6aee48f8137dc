"""Case-1 decoding (inverse of Eq. 4: v = fl(g / 10^alpha_max)) on the GPU against the oracle,
bit for bit, on streams built record by record from chosen integers g: every alpha 0..22
(FP32: 0..10), g spread over the whole Case-1 range, exact multiples of 5^alpha and their
neighbours, and |g| beyond 2^53, where the decoder's conversion of g to a double itself
rounds.  The records come from the oracle's own Eq. 5 and Sec. 3.3 functions; the stream
header and size array follow the documented stream format."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2511_04140_gb300 import build
    build.build()
    from paper_2511_04140_gb300 import falcon
    return falcon


def stream_of(oracle, gs, alpha, beta_hat, dtype_code, block):
    n = len(gs)
    nc = (n + block - 1) // block
    recs = []
    for c in range(nc):
        g = np.ascontiguousarray(gs[c * block:(c + 1) * block])
        z = oracle.delta_zigzag(g.astype(np.int64).view(np.uint64) if dtype_code == 0
                                else g.astype(np.int32).view(np.uint32).astype(np.uint64), dtype_code)
        recs.append(oracle.encode_z(z, dtype_code, alpha, beta_hat))
    hdr = (b"FLCN" + bytes([1, dtype_code, 0, 0]) + block.to_bytes(4, "little") + bytes(4)
           + n.to_bytes(8, "little") + nc.to_bytes(8, "little"))
    return hdr + b"".join(len(r).to_bytes(4, "little") for r in recs) + b"".join(recs)


def decode_both(F, oracle, s):
    want = oracle.decompress(s)
    t = torch.frombuffer(bytearray(s), dtype=torch.uint8).cuda()
    got = F.decompress(t).cpu().numpy()
    return got, want


@pytest.mark.parametrize("alpha", range(23))
def test_f64_every_alpha(F, oracle, alpha):
    rng = np.random.default_rng(100 + alpha)
    p5 = 5 ** alpha
    g = [0, 1, -1, 2, 3, 7, 10 ** 15 - 1, -(10 ** 15 - 1), (1 << 53) - 1, 1 << 53, -(1 << 53), (1 << 52) + 1]
    g += [k * p5 + d for k in (1, 2, 3, 99, 12345) for d in (-1, 0, 1) if abs(k * p5 + d) <= 1 << 53]
    g += list(rng.integers(-10 ** 15, 10 ** 15, 3000))
    g += list(rng.integers(-(1 << 53), 1 << 53, 3000))
    g += list(rng.integers(-10 ** 6, 10 ** 6, 2000))
    gs = np.array(g, dtype=np.int64)
    got, want = decode_both(F, oracle, stream_of(oracle, gs, alpha, 15, 0, 1024))
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
    # the oracle's values are fl(g / 10^alpha) (10^alpha is exact in FP64 for alpha <= 22)
    assert np.array_equal(want.view(np.uint64), (gs.astype(np.float64) / 10.0 ** alpha).view(np.uint64))


@pytest.mark.parametrize("alpha", [0, 1, 5, 17, 22])
def test_f64_beyond_2_53_takes_the_rounded_conversion(F, oracle, alpha):
    rng = np.random.default_rng(200 + alpha)
    big = rng.integers(1 << 53, 1 << 62, 600, dtype=np.int64)
    gs = np.concatenate([big, -big, rng.integers(-1000, 1000, 400), [np.iinfo(np.int64).max, np.iinfo(np.int64).min + 1]])
    got, want = decode_both(F, oracle, stream_of(oracle, gs.astype(np.int64), alpha, 15, 0, 1024))
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


@pytest.mark.parametrize("alpha", range(11))
def test_f32_every_alpha(F, oracle, alpha):
    rng = np.random.default_rng(300 + alpha)
    gs = np.concatenate([rng.integers(-10 ** 7, 10 ** 7, 3000), rng.integers(-(1 << 24), 1 << 24, 1000),
                         [0, 1, -1, 5 ** alpha, 2 * 5 ** alpha + 1]]).astype(np.int64)
    got, want = decode_both(F, oracle, stream_of(oracle, gs, alpha, 7, 1, 1025))
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
