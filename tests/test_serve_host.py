"""Host-side logic of the serving loop (no GPU): the seeded arrival
schedules and the latency summary."""
import numpy as np
import pytest

from paper_1711_00231_gb300 import serve as sv


def _cand():
    return [np.arange(1, 50, dtype=np.int32), np.array([3, 4], dtype=np.int32), np.arange(0, 1000, 7, dtype=np.int32)]


def test_poisson_schedule_is_seeded_and_well_formed():
    cand = _cand()
    a = sv.poisson_schedule(500, 200.0, [50, 5, 1000], cand, seed=3)
    b = sv.poisson_schedule(500, 200.0, [50, 5, 1000], cand, seed=3)
    assert [(r.arrival_s, r.graph, r.src, r.kind) for r in a] == [(r.arrival_s, r.graph, r.src, r.kind) for r in b]
    t = np.array([r.arrival_s for r in a])
    assert np.all(np.diff(t) > 0)
    # exponential gaps at rate 200/s: mean gap 5 ms (500 draws: within 20%)
    assert np.mean(np.diff(t)) == pytest.approx(1 / 200.0, rel=0.2)
    for r in a:
        assert r.src in set(cand[r.graph].tolist())
        assert r.kind in ("bfs", "sssp")
    kinds = [r.kind for r in a]
    assert 0.35 < kinds.count("sssp") / len(kinds) < 0.65
    assert len({r.graph for r in a}) == 3


def test_burst_schedule_and_unweighted_graphs():
    cand = _cand()
    burst = sv.poisson_schedule(100, float("inf"), [50, 5, 1000], cand, seed=1, sssp_ok=[True, False, True])
    assert all(r.arrival_s == 0.0 for r in burst)
    assert all(r.kind == "bfs" for r in burst if r.graph == 1)


def test_latency_percentiles():
    p = sv._percentiles([0.001] * 98 + [0.5, 1.0])
    assert p["p50_ms"] == pytest.approx(1.0)
    assert p["max_ms"] == pytest.approx(1000.0)
    assert p["p99_ms"] > 100.0
