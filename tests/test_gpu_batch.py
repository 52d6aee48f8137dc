"""Batched form (the launches of one direction over many series at once): every series' stream must be the
oracle's stream for that series, byte for byte, and decode bit-exactly; results are the
same alone, in the batch, and replayed from a CUDA graph."""
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


def _u(a):
    return a.view(np.uint64 if a.dtype == np.float64 else np.uint32)


def _mixed_series():
    series = synth.series_batch(count=48, seed=9, min_len=1, max_len=1 << 17, max_outlier_rate=0.05)
    series += [np.zeros(0, dtype=np.float64), np.array([2.5], dtype=np.float32),
               synth.segments(70_001, seed=3), synth.segments(50_000, seed=4, dtype=np.float32),
               synth.adversarial_f64(), synth.adversarial_f32()]
    return series


@pytest.mark.parametrize("block", [1024, 1025])
def test_batch_matches_oracle(F, oracle, block):
    series = _mixed_series()
    xs = [torch.from_numpy(np.ascontiguousarray(s)).cuda() for s in series]
    b = F.Batch(F.COMPRESS, xs, block=block)
    b.launch()
    torch.cuda.synchronize()
    res = b.results()
    streams = b.streams()
    for s, (nb, st), out in zip(series, res, streams):
        assert st == 0
        assert out.cpu().numpy().tobytes() == oracle.compress(s, block)
    dec = F.Batch(F.DECOMPRESS, [(o, o.numel(), o[:32].cpu().numpy().tobytes()) for o in streams])
    dec.launch()
    torch.cuda.synchronize()
    for s, (nv, st), y in zip(series, dec.results(), dec.outputs):
        assert st == 0 and nv == len(s)
        assert np.array_equal(_u(y[:len(s)].cpu().numpy()), _u(s))
    b.close()
    dec.close()


def test_batch_same_alone_and_in_mix(F):
    series = _mixed_series()
    xs = [torch.from_numpy(np.ascontiguousarray(s)).cuda() for s in series]
    b = F.Batch(F.COMPRESS, xs, block=1024)
    b.launch()
    torch.cuda.synchronize()
    for x, s in zip(xs, b.streams()):
        alone = F.compress(x, 1024)
        assert torch.equal(alone, s)


def test_batch_graph_replay(F):
    series = _mixed_series()[:20]
    xs = [torch.from_numpy(np.ascontiguousarray(s)).cuda() for s in series]
    b = F.Batch(F.COMPRESS, xs, block=1024)
    b.launch()
    torch.cuda.synchronize()
    first = [s.clone() for s in b.streams()]
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        b.launch(stream)
    for _ in range(2):
        for o in b.outputs:
            o.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert all(torch.equal(a, s) for a, s in zip(first, b.streams()))


def test_batch_capacity_and_invalid(F):
    x = torch.from_numpy(synth.segments(20_000, seed=5)).cuda()
    small = torch.empty(1000, dtype=torch.uint8, device="cuda")
    with pytest.raises(F.FalconError):
        F.Batch(F.COMPRESS, [x], block=1024, outputs=[torch.empty(16, dtype=torch.uint8, device="cuda")])
    b = F.Batch(F.COMPRESS, [x], block=1024, outputs=[small])
    b.launch()
    torch.cuda.synchronize()
    assert b.results()[0][1] == F.ERR_CAPACITY
    with pytest.raises(F.FalconError):
        F.Batch(F.COMPRESS, [x], block=4096)


def test_autotune_keeps_bytes(F, oracle):
    from paper_2511_04140_gb300 import tune
    series = synth.series_batch(count=12, seed=11, min_len=1024, max_len=1 << 16)
    xs = [torch.from_numpy(s).cuda() for s in series]
    out = tune.autotune(xs, blocks=(512, 1024), compress_ctas=(0, 1), decompress_ctas=(0, 1), reps=1)
    choice = out["choice"]
    # 2 blocks x 3 x 3 CTA shapes at the occupancy limit, then 3 resident-CTA caps
    assert choice["block"] in (512, 1024) and len(out["table"]) == 2 * 3 * 3 + 3
    blk = tune.apply(choice)
    try:
        b = F.Batch(F.COMPRESS, xs, block=blk)
        b.launch()
        torch.cuda.synchronize()
        for s, st in zip(series, b.streams()):
            assert st.cpu().numpy().tobytes() == oracle.compress(s, blk)
    finally:
        F.set_launch_config(0, 0)
        F.set_cta_warps(4, 4)


def test_cta_shape_changes_no_byte(F, oracle):
    """Warps per CTA and resident CTAs per SM are launch shape only: every shape the autotuner
    may pick gives the oracle's bytes, in both directions."""
    vals = synth.segments(300_001, seed=51)
    x = torch.from_numpy(vals).cuda()
    ref = oracle.compress(vals, 1024)
    try:
        for cw, dw, cc, dc in ((1, 1, 0, 0), (2, 12, 0, 0), (8, 3, 2, 1), (16, 8, 0, 2)):
            F.set_cta_warps(cw, dw)
            F.set_launch_config(cc, dc)
            s = F.compress(x, 1024)
            assert s.cpu().numpy().tobytes() == ref, (cw, dw, cc, dc)
            y = F.decompress(s)
            assert torch.equal(y.view(torch.int64), x.view(torch.int64)), (cw, dw, cc, dc)
        for bad in ((0, 4), (17, 4), (4, 13)):
            with pytest.raises(F.FalconError):
                F.set_cta_warps(*bad)
    finally:
        F.set_cta_warps(4, 4)
        F.set_launch_config(0, 0)
