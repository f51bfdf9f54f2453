"""Seeded input generators: the serving request stream and its problems (host only)."""
import numpy as np

import synth


def test_serving_stream_shape_and_determinism():
    a = synth.serving_requests(count=200, seed=5)
    b = synth.serving_requests(count=200, seed=5)
    assert a == b
    t = np.array([r["arrival"] for r in a])
    assert np.all(np.diff(t) > 0)
    # Poisson arrivals at 100 Hz: mean gap 10 ms within sampling error
    assert 0.008 < np.diff(t).mean() < 0.012
    for r in a:
        assert 16 <= r["s"] <= 128
        assert r["N"] in (32, 64, 128) and r["L"] in (8, 16, 32) and r["M"] == 8
        assert r["family"] in ("delay", "drude")
        assert -0.5 <= r["shift"] <= 0.5
    assert {r["family"] for r in a} == {"delay", "drude"}


def test_serving_problem_matches_request():
    for r in synth.serving_requests(count=6, seed=1, s_min=8, s_max=20):
        p = synth.serving_problem(r)
        assert p.n == r["s"] ** 2
        assert (p.N, p.L, p.M) == (r["N"], min(r["L"], p.n), r["M"])
        centre = (-2.0 if r["family"] == "delay" else 2.0) + r["shift"]
        assert abs(p.region["center"] - centre) < 1e-15
        assert len(p.mats) == len(p.fns) == 3
