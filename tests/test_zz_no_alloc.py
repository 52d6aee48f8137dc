"""falcon_compress_noalloc (the static-scratch variant of asynchronous compression) against
falcon_compress on the same inputs, through the C ABI, two calls in a row on one stream.
The file sorts last so that it also runs after every other test has used the device."""
import numpy as np
import pytest
import torch

from paper_2511_04140_gb300 import synth

pytestmark = pytest.mark.gpu

MAX_CHUNKS = 65536


@pytest.fixture(scope="module")
def F():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2511_04140_gb300 import build
    build.build()
    from paper_2511_04140_gb300 import falcon
    return falcon


def _enqueue(F, x, block, stream):
    code = F._dtype_code(x)
    out = torch.empty(F.bound(x.numel(), code, block), dtype=torch.uint8, device=x.device)
    res = torch.full((2,), -1, dtype=torch.int64, device=x.device)      # the call must clear it
    torch.cuda.synchronize()
    st = F.lib().falcon_compress_noalloc(x.data_ptr(), x.numel(), code, block, out.data_ptr(), out.numel(),
                                         res.data_ptr(), stream.cuda_stream)
    assert st == F.OK, st
    return out, res


def _check(out, res, ref):
    nbytes, status = (int(v) for v in res.cpu())
    assert status == 0
    assert nbytes == ref.numel()
    assert torch.equal(out[:nbytes], ref)


def test_two_calls_in_a_row_match_compress(F):
    a = torch.from_numpy(synth.segments(1_000_003, seed=21)).cuda()
    b = torch.from_numpy(synth.random_walk(700_001, seed=22, places=4, dtype=np.float32, outlier_rate=0.01)).cuda()
    ref_a, ref_b = F.compress(a, 1024).clone(), F.compress(b, 1024).clone()
    stream = torch.cuda.Stream()
    out_a, res_a = _enqueue(F, a, 1024, stream)
    out_b, res_b = _enqueue(F, b, 1024, stream)          # same scratch, reused right away
    stream.synchronize()
    _check(out_a, res_a, ref_a)
    _check(out_b, res_b, ref_b)


def test_same_input_twice_and_ragged_block(F):
    x = torch.from_numpy(synth.random_walk(123_457, seed=23, places=2, outlier_rate=0.003)).cuda()
    ref = F.compress(x, 1000).clone()
    stream = torch.cuda.Stream()
    first = _enqueue(F, x, 1000, stream)
    second = _enqueue(F, x, 1000, stream)
    stream.synchronize()
    _check(*first, ref)
    _check(*second, ref)


def test_maximum_size_and_rejection_above_it(F):
    n = MAX_CHUNKS * 1024                                  # exactly the static scratch's capacity
    g = torch.Generator(device="cuda").manual_seed(24)
    x = torch.round(torch.cumsum(torch.randn(n, generator=g, device="cuda") * 0.5, 0) * 100) / 100
    ref = F.compress(x, 1024).clone()
    stream = torch.cuda.Stream()
    out, res = _enqueue(F, x, 1024, stream)
    stream.synchronize()
    _check(out, res, ref)
    del out
    y = torch.empty(n + 1, dtype=torch.float32, device="cuda")
    big = torch.empty(F.bound(n + 1, F.F32, 1024), dtype=torch.uint8, device="cuda")
    r = torch.zeros(2, dtype=torch.int64, device="cuda")
    st = F.lib().falcon_compress_noalloc(y.data_ptr(), n + 1, F.F32, 1024, big.data_ptr(), big.numel(),
                                         r.data_ptr(), stream.cuda_stream)
    assert st == F.ERR_UNSUPPORTED
    # argument errors are reported before the size limit, as falcon_compress_async reports them
    bad_dtype = F.lib().falcon_compress_noalloc(y.data_ptr(), n + 1, 7, 1024, big.data_ptr(), big.numel(),
                                                r.data_ptr(), stream.cuda_stream)
    null_out = F.lib().falcon_compress_noalloc(y.data_ptr(), n + 1, F.F32, 1024, None, big.numel(),
                                               r.data_ptr(), stream.cuda_stream)
    bad_block = F.lib().falcon_compress_noalloc(y.data_ptr(), n + 1, F.F32, 4096, big.data_ptr(), big.numel(),
                                                r.data_ptr(), stream.cuda_stream)
    assert (bad_dtype, null_out, bad_block) == (F.ERR_INVALID, F.ERR_INVALID, F.ERR_INVALID)


def test_calls_allocate_no_device_memory(F):
    """The point of the entry point: after one call has loaded the module, further calls of
    several sizes leave the device's free memory and torch's pool exactly as they were."""
    xs = [torch.from_numpy(synth.segments(k, seed=25 + k % 7)).cuda() for k in (5_000, 300_000, 2_000_001)]
    outs = [torch.empty(F.bound(x.numel(), F.F64, 1024), dtype=torch.uint8, device="cuda") for x in xs]
    res = torch.zeros(2, dtype=torch.int64, device="cuda")
    stream = torch.cuda.Stream()

    def call(i):
        st = F.lib().falcon_compress_noalloc(xs[i].data_ptr(), xs[i].numel(), F.F64, 1024, outs[i].data_ptr(),
                                             outs[i].numel(), res.data_ptr(), stream.cuda_stream)
        assert st == F.OK, st

    call(0)
    stream.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(2):
        for i in range(len(xs)):
            call(i)
    stream.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_reserved() == reserved0
    assert free1 == free0
    assert int(res[1].item()) == 0
