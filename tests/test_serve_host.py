"""Host-side serving logic (no GPU): the seeded Poisson arrival process and the latency summary."""
import numpy as np

from paper_2603_02887_gb300.serve import _latency_summary, poisson_arrivals


def test_poisson_arrivals_rate_and_seed():
    a = poisson_arrivals(20000, rate=200.0, seed=3)
    assert np.all(np.diff(a) > 0)
    gaps = np.diff(np.concatenate([[0.0], a]))
    assert abs(gaps.mean() - 1 / 200.0) < 0.03 / 200.0  # mean inter-arrival 1/rate
    assert abs(gaps.std() - 1 / 200.0) < 0.05 / 200.0   # exponential: std = mean
    assert np.array_equal(a, poisson_arrivals(20000, rate=200.0, seed=3))


def test_latency_summary_percentiles():
    lat = np.arange(1, 101, dtype=float)  # 1 .. 100 ms
    s = _latency_summary(lat, elapsed_s=2.0, n=100)
    assert s["p50_ms"] == 50.5 and s["p99_ms"] == 99.01
    assert s["frames_per_s"] == 50.0 and s["max_ms"] == 100.0
