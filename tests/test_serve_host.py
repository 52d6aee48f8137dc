"""Host logic of the serving load generator (no GPU): Poisson arrivals and the latency
summary that the serving measurement reports."""
import numpy as np
import pytest

from paper_2511_04140_gb300 import serve


def test_poisson_arrivals():
    rate, duration, npool = 5000.0, 4.0, 64
    arr = serve._arrivals(rate, duration, npool, seed=3)
    t = np.array([a for a, _ in arr])
    idx = np.array([i for _, i in arr])
    # count ~ Poisson(rate * duration): within 5 standard deviations
    assert abs(len(arr) - rate * duration) < 5 * np.sqrt(rate * duration)
    assert np.all(np.diff(t) > 0) and t[0] > 0 and t[-1] < duration
    gaps = np.diff(t)
    assert gaps.mean() == pytest.approx(1.0 / rate, rel=0.05)
    assert np.std(gaps) == pytest.approx(1.0 / rate, rel=0.1)       # exponential: sd = mean
    assert idx.min() >= 0 and idx.max() < npool and len(np.unique(idx)) == npool
    assert arr == serve._arrivals(rate, duration, npool, seed=3)      # seeded


def test_latency_summary():
    lat = [i / 1000.0 for i in range(1, 101)]                         # 1 .. 100 ms
    out = serve._summary(lat[::-1], nbytes=4e9, wall=2.0, n=100)
    assert out["p50_ms"] == pytest.approx(51.0) and out["p99_ms"] == pytest.approx(100.0)
    assert out["gbs"] == pytest.approx(2.0) and out["requests"] == 100
    assert serve._summary([], 0, 1.0, 0)["p99_ms"] is None
