"""GPU parity of the codec variants (Falcon and the Sec. 5.4.2 ablations Fal._Sparse,
Fal._Dense, Fal._Elf): falcon_compress_variant_async's streams equal the oracle's variant
streams byte for byte, and the one GPU decoder gives back every input bit (tolerance 0 bits)."""
import numpy as np
import pytest
import torch

from paper_2511_04140_gb300 import synth

pytestmark = pytest.mark.gpu

VARIANTS = [0, 1, 2, 3]


@pytest.fixture(scope="module")
def F():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2511_04140_gb300 import build
    build.build()
    from paper_2511_04140_gb300 import falcon
    return falcon


def _u(arr):
    return arr.view(np.uint64 if arr.dtype == np.float64 else np.uint32)


def check_variant(F, oracle, vals, block, variant):
    x = torch.from_numpy(np.ascontiguousarray(vals)).cuda()
    s = F.compress_variant(x, block, variant)
    got = s.cpu().numpy().tobytes()
    expect = oracle.compress(vals, block, variant=variant)
    assert len(got) == len(expect) and got == expect, (variant, block, len(got), len(expect))
    assert len(got) <= F.variant_bound(len(vals), F._dtype_code(x), block, variant)
    y = F.decompress(s)
    assert np.array_equal(_u(y.cpu().numpy()), _u(vals)), "round trip not bit-exact"


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("block", [1024, 1025, 100, 2])
def test_segments(F, oracle, variant, dtype, block):
    n = 20_011 if block == 2 else 150_001
    check_variant(F, oracle, synth.segments(n, seed=31, dtype=dtype), block, variant)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("places", [0, 2, 5])
def test_random_walk(F, oracle, variant, dtype, places):
    vals = synth.random_walk(100_003, seed=32 + places, places=places, dtype=dtype, outlier_rate=0.0005)
    check_variant(F, oracle, vals, 1024, variant)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_adversarial(F, oracle, variant, dtype):
    arr = synth.adversarial_f64() if dtype == np.float64 else synth.adversarial_f32()
    for block in (2, 3, 65, 1024, 1025):
        check_variant(F, oracle, arr, block, variant)
    for v in arr[::3]:
        check_variant(F, oracle, np.array([0.5, 1.25, v, 3.75, 1.11, 7.15], dtype=dtype), 1024, variant)


@pytest.mark.parametrize("variant", VARIANTS)
def test_elf_differs_from_falcon_on_decimals(F, oracle, variant):
    """Decimal series where Elf's trial-and-error places exceed Alg. 2's in some chunks: the
    GPU follows the oracle in each variant, and Elf's stream is the longer one."""
    vals = synth.random_walk(300_000, seed=33, places=2)
    check_variant(F, oracle, vals, 1024, variant)
    if variant == 3:
        assert len(oracle.compress(vals, 1024, variant=3)) > len(oracle.compress(vals, 1024))


def test_sparse_variant_worst_case_record(F, oracle):
    """Rows without a zero byte stored sparse: the largest record the format allows (bitmap +
    128 bytes per row), which needs the wide emit buffer and the decoder's full record buffer."""
    bits = np.zeros(5 * 1025, dtype=np.uint64)
    bits[::2] = np.uint64(1)
    bits[1::2] = np.uint64(0x4000000000000001)
    vals = bits.view(np.float64)
    for block in (1025, 1024):
        check_variant(F, oracle, vals, block, 1)
        check_variant(F, oracle, vals, block, 0)
    s = F.compress_variant(torch.from_numpy(vals).cuda(), 1025, 1)
    assert s.numel() == F.variant_bound(len(vals), F.F64, 1025, 1)


def test_unknown_variant_is_invalid(F):
    x = torch.zeros(10, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FalconError) as e:
        F.compress_variant(x, 1024, 4)
    assert e.value.status == F.ERR_INVALID
