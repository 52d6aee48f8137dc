"""Continuous-batching server: requests that arrive while others are on the GPU join later
batches; every result equals the same request processed alone (0-bit tolerance: the codec is
lossless and deterministic); a malformed request fails alone."""
import concurrent.futures as cf
import threading

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


def _requests(F, count=40, seed=3):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(10), np.log(400_000))))
        dtype = np.float64 if rng.random() < 0.5 else np.float32
        vals = synth.random_walk(n, seed=int(rng.integers(1 << 30)), places=int(rng.integers(0, 5)), dtype=dtype,
                                 outlier_rate=float(rng.uniform(0, 0.02)))
        if i % 2 == 0:
            reqs.append(("compress", torch.from_numpy(vals).pin_memory(), vals))
        else:
            s = F.compress(torch.from_numpy(vals).cuda(), 1024).cpu()
            reqs.append(("decompress", s, vals))
    return reqs


def _check(oracle, op, out, vals):
    if op == "compress":
        assert out.numpy().tobytes() == oracle.compress(vals, 1024)
    else:
        u = np.uint64 if vals.dtype == np.float64 else np.uint32
        assert np.array_equal(out.numpy().view(u), vals.view(u))


def test_mixed_concurrent_requests_match_solo(F, oracle):
    from paper_2511_04140_gb300.serve import Server
    reqs = _requests(F)
    with Server(budget_bytes=1 << 30, host_budget_bytes=256 << 20) as srv:
        futs = [None] * len(reqs)

        def client(idx):
            for i in idx:
                op, payload, _ = reqs[i]
                futs[i] = srv.submit(op, payload)

        threads = [threading.Thread(target=client, args=(range(k, len(reqs), 4),)) for k in range(4)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        for f, (op, _, vals) in zip(futs, reqs):
            _check(oracle, op, f.result(timeout=120), vals)
            assert f.latency > 0
        stats = dict(srv.stats)
    assert stats["requests"] == len(reqs) == stats["completed"]
    assert stats["multi_request_batches"] >= 1          # requests really were batched together


def test_device_budget_bounds_memory_in_flight(F, oracle):
    from paper_2511_04140_gb300.serve import Server
    reqs = _requests(F, count=24, seed=8)
    budget = 16 << 20                                    # about two of the largest requests
    with Server(budget_bytes=budget, host_budget_bytes=64 << 20) as srv:
        futs = [srv.submit(op, p) for op, p, _ in reqs]
        for f, (op, _, vals) in zip(futs, reqs):
            _check(oracle, op, f.result(timeout=120), vals)
        st = srv.stats
    assert st["device_peak"] <= st["device_capacity"] == budget
    assert st["completed"] == len(reqs) and st["failed"] == 0


def test_request_larger_than_budget_is_rejected(F):
    from paper_2511_04140_gb300.serve import Server
    x = torch.from_numpy(synth.random_walk(1 << 20, seed=2)).pin_memory()     # 8 MiB of values
    with Server(budget_bytes=4 << 20, host_budget_bytes=64 << 20) as srv:
        f = srv.submit("compress", x)
        with pytest.raises(F.FalconError) as e:
            f.result(timeout=5)
        assert e.value.status == F.ERR_CAPACITY
        small = srv.submit("compress", x[:1000]).result(timeout=60)           # the server keeps serving
        assert small.numel() > 32


def test_host_arena_backpressure(F, oracle):
    import gc
    from paper_2511_04140_gb300.serve import Server
    a = synth.random_walk(300_000, seed=4, places=3)                         # 2.4 MB of values
    b = synth.random_walk(200_000, seed=5, places=3)
    s_a = F.compress(torch.from_numpy(a).cuda(), 1024).cpu()
    s_b = F.compress(torch.from_numpy(b).cuda(), 1024).cpu()
    with Server(budget_bytes=256 << 20, host_budget_bytes=3 << 20) as srv:
        held = srv.submit("decompress", s_a).result(timeout=60)               # occupies 2.4 of 3 MB
        f = srv.submit("decompress", s_b)                                    # needs 1.6 MB: must wait
        with pytest.raises(cf.TimeoutError):
            f.result(timeout=0.5)
        assert np.array_equal(held.numpy().view(np.uint64), a.view(np.uint64))
        del held
        gc.collect()                                                         # output back to the arena
        assert np.array_equal(f.result(timeout=60).numpy().view(np.uint64), b.view(np.uint64))


def test_injected_bad_request_fails_alone(F, oracle):
    from paper_2511_04140_gb300.serve import Server
    reqs = _requests(F, count=8, seed=9)
    good = reqs[1][1].clone()
    bad = good.clone()
    bad[0] = ord("X")                                    # corrupt magic: rejected at admission
    bad2 = good.clone()
    bad2[32] ^= 0x55                                     # corrupt first size entry: the kernel flags it
    with Server(budget_bytes=1 << 30, host_budget_bytes=256 << 20) as srv:
        futs = [srv.submit(op, p) for op, p, _ in reqs]
        f_bad = srv.submit("decompress", bad)
        f_bad2 = srv.submit("decompress", bad2)
        for f, (op, _, vals) in zip(futs, reqs):
            _check(oracle, op, f.result(timeout=120), vals)
        with pytest.raises(F.FalconError) as e:                 # rejected at submission
            f_bad.result(timeout=1)
        assert e.value.status == F.ERR_CORRUPT
        with pytest.raises(F.FalconError) as e:                 # found by the kernel
            f_bad2.result(timeout=120)
        assert e.value.status == F.ERR_CORRUPT
        st = srv.stats
    assert st["failed"] == 1 and st["completed"] == len(reqs) + 1


def test_load_run(F):
    from paper_2511_04140_gb300 import serve
    pool = serve.make_pool(count=8, min_bytes=4 << 10, max_bytes=4 << 20)
    with serve.Server(budget_bytes=1 << 30, host_budget_bytes=256 << 20) as srv:
        res = serve.run_load(srv, pool, rate=300, duration=0.5)
    assert res["requests"] > 50 and res["p99_ms"] is not None and res["gbs"] > 0
    base = serve.run_one_at_a_time(pool, rate=300, duration=0.5)
    assert base["requests"] > 50
