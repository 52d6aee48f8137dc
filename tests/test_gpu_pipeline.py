"""Host <-> device streaming pipeline (Sec. 3.1, Alg. 1): every frame of the output is the
oracle's stream for that frame's values, frames are placed in launch order, and the
inverse pipeline restores every bit."""
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


@pytest.mark.parametrize("nstreams", [1, 3, 16])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_pipeline_frames_match_oracle(F, oracle, nstreams, dtype):
    vals = synth.segments(700_001, seed=12, dtype=dtype)
    frame = 65_536
    x = torch.from_numpy(vals).pin_memory()
    s, fb = F.pipeline_compress(x, block=1024, frame_values=frame, nstreams=nstreams)
    assert len(fb) == (len(vals) + frame - 1) // frame
    blob = s.numpy().tobytes()
    off = 0
    for i, nb in enumerate(fb):
        part = vals[i * frame:(i + 1) * frame]
        assert blob[off:off + nb] == oracle.compress(part, 1024), i
        off += nb
    assert off == len(blob)
    y = F.pipeline_decompress(s, fb, nstreams=nstreams)
    assert np.array_equal(_u(y.numpy()), _u(vals))


def test_pipeline_pageable_and_tail(F, oracle):
    vals = synth.random_walk(100_003, seed=7, places=3, outlier_rate=0.005)
    x = torch.from_numpy(vals)                     # pageable: copies serialise, bytes identical
    s, fb = F.pipeline_compress(x, block=1025, frame_values=30_000, nstreams=2)
    blob = s.numpy().tobytes()
    off = 0
    for i, nb in enumerate(fb):
        assert blob[off:off + nb] == oracle.compress(vals[i * 30_000:(i + 1) * 30_000], 1025)
        off += nb
    y = F.pipeline_decompress(s, fb, nstreams=2)
    assert np.array_equal(_u(y.numpy()), _u(vals))


def test_pipeline_capacity(F):
    vals = synth.segments(200_000, seed=3)
    x = torch.from_numpy(vals).pin_memory()
    out = torch.empty(100_000, dtype=torch.uint8).pin_memory()
    with pytest.raises(F.FalconError) as e:
        F.pipeline_compress(x, block=1024, frame_values=50_000, nstreams=4, out=out)
    assert e.value.status == F.ERR_CAPACITY


@pytest.mark.parametrize("scheduler", [1, 2])
@pytest.mark.parametrize("nstreams", [1, 2, 5, 16])
def test_schedulers_write_the_event_driven_bytes(F, oracle, scheduler, nstreams):
    """Sec. 3.1's sync-based and pre-allocation schedulers (the ablation of Sec. 5.4.1) give
    the same frames as the event-driven one, each equal to the oracle's stream."""
    vals = synth.segments(520_003, seed=14)
    frame = 65_536
    x = torch.from_numpy(vals).pin_memory()
    ref, fb_ref = F.pipeline_compress(x, block=1024, frame_values=frame, nstreams=nstreams)
    s, fb = F.pipeline_compress(x, block=1024, frame_values=frame, nstreams=nstreams, scheduler=scheduler)
    assert fb == fb_ref
    assert torch.equal(s, ref)
    blob = s.numpy().tobytes()
    off = 0
    for i, nb in enumerate(fb):
        assert blob[off:off + nb] == oracle.compress(vals[i * frame:(i + 1) * frame], 1024), i
        off += nb


def test_scheduler_capacity_and_unknown(F):
    vals = synth.segments(200_000, seed=3)
    x = torch.from_numpy(vals).pin_memory()
    out = torch.empty(100_000, dtype=torch.uint8).pin_memory()
    for sch in (1, 2):
        with pytest.raises(F.FalconError) as e:
            F.pipeline_compress(x, block=1024, frame_values=50_000, nstreams=4, out=out, scheduler=sch)
        assert e.value.status == F.ERR_CAPACITY
    with pytest.raises(F.FalconError) as e:
        F.pipeline_compress(x, block=1024, frame_values=50_000, nstreams=4, scheduler=3)
    assert e.value.status == F.ERR_INVALID
