"""The seeded input generators of the serving stream (host only).

- The default stream draws one problem per request: 2D / 3D sides from the
  listed sets, ppw in [8, 12], medium seed 1000 + request id, Poisson arrivals
  (mean gap 1/rate) in increasing order; the same seed gives the same stream.
- problems = K: every request takes one of K problems (dimension, side,
  medium, frequency, seed 1000 + problem index) and its own source, so
  requests of one problem differ only in the source.
"""
import numpy as np

import workloads


def test_default_stream_is_one_problem_per_request():
    a = workloads.config5(n_requests=400)
    b = workloads.config5(n_requests=400)
    assert a == b
    t = np.array([r.arrival_s for r in a])
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean(np.diff(t)) - 1 / 40.0) < 0.2 / 40.0          # 400 exponential gaps
    assert [r.seed for r in a] == [1000 + r.rid for r in a]
    for r in a:
        assert (r.dim, r.n) in {(2, 257), (2, 513), (2, 1025), (2, 2049), (3, 65), (3, 129), (3, 193)}
        assert 8.0 <= r.ppw <= 12.0 and r.generator in ("homogeneous", "layered")
        assert len(r.src_u) == r.dim and all(0.0 <= u < 1.0 for u in r.src_u)


def test_shared_problem_stream():
    reqs = workloads.config5(n_requests=300, problems=6)
    probs = {(r.dim, r.n, r.generator, r.ppw, r.seed) for r in reqs}
    assert len(probs) <= 6 and len(probs) >= 4
    assert {r.seed for r in reqs} <= set(range(1000, 1006))
    # requests of one problem differ in their sources
    by = {}
    for r in reqs:
        by.setdefault((r.dim, r.n, r.generator, r.ppw, r.seed), []).append(r)
    for members in by.values():
        if len(members) > 1:
            assert len({r.src_u for r in members}) > 1
    # the medium and frequency follow from the problem alone (smallest problem
    # with two requests: its generated inputs agree except for the source)
    key = min((k for k, v in by.items() if len(v) > 1), key=lambda k: k[1] ** k[0])
    a, b = by[key][0].workload(), by[key][1].workload()
    assert np.array_equal(a.kappa, b.kappa) and np.array_equal(a.gamma, b.gamma) and a.omega == b.omega
