"""Every FP32 bit pattern through the GPU codec against the oracle (R14's FP32 reading of
Alg. 2 and Eq. 4, and R1's specials): all 2^32 patterns in order, in 1024-value chunks, as
16 slices of 2^28 values; each slice's stream equals the oracle's byte for byte and decodes
to the same bits.  Chunks of two values take each value's decimal place almost alone: a
stratified sample (every exponent and sign, random and decimal-like significands) as B = 2
chunks.  Slow: about a minute of host-core oracle work."""
import os

import numpy as np
import pytest
import torch

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def F():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2511_04140_gb300 import build
    build.build()
    from paper_2511_04140_gb300 import falcon
    return falcon


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def test_all_fp32_patterns_in_1024_chunks(F, oracle):
    step = 1 << 28
    for k in range((1 << 32) // step):
        p64 = torch.arange(k * step, (k + 1) * step, dtype=torch.int64, device="cuda")
        pat = torch.where(p64 >= 1 << 31, p64 - (1 << 32), p64).to(torch.int32)    # the 32-bit patterns
        del p64
        x = pat.view(torch.float32)
        s = F.compress(x, 1024)
        got = s.cpu().numpy().tobytes()
        host = x.cpu().numpy()
        assert got == oracle.compress(host, 1024, threads=_cores()), f"slice {k}"
        y = F.decompress(s)
        assert torch.equal(y.view(torch.int32), pat), f"slice {k}"
        del pat, x, s, y


def test_fp32_stratified_pairs(F, oracle):
    rng = np.random.default_rng(41)
    parts = []
    for sign in (0, 1):
        for e in range(256):
            mant = rng.integers(0, 1 << 23, 4096, dtype=np.uint32)
            parts.append((sign << 31) | (e << 23) | mant)
    bits = np.concatenate(parts).astype(np.uint32)
    # decimal-like values at every magnitude: k / 10^p rounded to FP32
    k = rng.integers(1, 10 ** 7, 1 << 18)
    p = rng.integers(0, 12, 1 << 18)
    dec = (k / 10.0 ** p).astype(np.float32).view(np.uint32)
    bits = np.concatenate([bits, dec, (dec ^ np.uint32(1 << 31))])
    vals = bits.view(np.float32)
    for block in (2, 3):
        x = torch.from_numpy(vals).cuda()
        s = F.compress(x, block)
        assert s.cpu().numpy().tobytes() == oracle.compress(vals, block, threads=_cores()), block
        y = F.decompress(s)
        assert torch.equal(y.view(torch.int32), x.view(torch.int32)), block
