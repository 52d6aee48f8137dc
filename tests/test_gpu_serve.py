"""Continuous-batching server: requests that arrive while others are on the GPU join later
batches; every result equals the same request processed alone (0-bit tolerance: the codec is
lossless and deterministic); a malformed request fails alone."""
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
    with Server(budget_bytes=1 << 30) as srv:
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
        stats = dict(srv.stats)
    assert stats["requests"] == len(reqs)
    assert stats["multi_request_batches"] >= 1          # requests really were batched together


def test_budget_limits_admission(F, oracle):
    from paper_2511_04140_gb300.serve import Server
    reqs = _requests(F, count=16, seed=8)
    budget = 12 << 20
    with Server(budget_bytes=budget) as srv:
        futs = [srv.submit(op, p) for op, p, _ in reqs]
        peak = 0
        while not all(f.done() for f in futs):
            peak = max(peak, srv.in_use)
        for f, (op, _, vals) in zip(futs, reqs):
            _check(oracle, op, f.result(timeout=120), vals)
    biggest = max(srv._need(type("R", (), {"op": op, "payload": p, "block": 1024})()) for op, p, _ in reqs)
    assert peak <= max(budget, biggest)


def test_injected_bad_request_fails_alone(F, oracle):
    from paper_2511_04140_gb300.serve import Server
    reqs = _requests(F, count=8, seed=9)
    good = reqs[1][1].clone()
    bad = good.clone()
    bad[0] = ord("X")                                    # corrupt magic: rejected at admission
    bad2 = good.clone()
    bad2[32] ^= 0x55                                     # corrupt first size entry: the kernel flags it
    with Server(budget_bytes=1 << 30) as srv:
        futs = [srv.submit(op, p) for op, p, _ in reqs]
        f_bad = srv.submit("decompress", bad)
        f_bad2 = srv.submit("decompress", bad2)
        for f, (op, _, vals) in zip(futs, reqs):
            _check(oracle, op, f.result(timeout=120), vals)
        with pytest.raises(F.FalconError):
            f_bad.result(timeout=120)
        with pytest.raises(F.FalconError):
            f_bad2.result(timeout=120)


def test_load_run(F):
    from paper_2511_04140_gb300 import serve
    pool = serve.make_pool(count=8, min_bytes=4 << 10, max_bytes=4 << 20)
    with serve.Server(budget_bytes=1 << 30) as srv:
        res = serve.run_load(srv, pool, rate=300, duration=0.5)
    assert res["requests"] > 50 and res["p99_ms"] is not None and res["gbs"] > 0
    base = serve.run_one_at_a_time(pool, rate=300, duration=0.5)
    assert base["requests"] > 50
