"""CPU checks of the serving loop's host logic: the work estimate of a request,
its priority class and the CUDA stream priority it maps to, and nearest-rank
percentiles of run latencies."""
import math

import pytest

import galpic_inputs as gi


@pytest.fixture(scope="module")
def serve():
    from paper_1608_00215_gb300 import build
    build.build()
    from paper_1608_00215_gb300 import serve
    return serve


def test_pushes_counts_every_species(serve):
    wl = gi.drifting_plasma(32, 32, 64, 10.0, galilean=True, shape_order=1, precision=32,
                            ppc=(2, 1, 3), seed=1)
    assert serve.pushes(wl, 7) == 32 * 32 * 64 * (6 + 6) * 7
    wl1 = gi.drifting_plasma(32, 32, 64, 10.0, galilean=True, shape_order=1, precision=32,
                             ppc=(2, 2, 2), seed=1, electron_only=True)
    assert serve.pushes(wl1, 1) == 32 * 32 * 64 * 8


def test_priority_levels_are_monotone_in_work(serve):
    b = serve.PRIORITY_BOUNDS
    assert serve.priority_level(1) == 3
    assert serve.priority_level(b[0] - 1) == 3 and serve.priority_level(b[0]) == 2
    assert serve.priority_level(b[1]) == 1 and serve.priority_level(b[2]) == 0
    works = [2 ** k for k in range(10, 40)]
    levels = [serve.priority_level(w) for w in works]
    assert levels == sorted(levels, reverse=True)


def test_stream_priority_clamps_to_the_device_range(serve):
    # CUDA reports (least, greatest) with lower numbers meaning higher priority
    assert [serve.stream_priority(k, (0, -5)) for k in range(4)] == [0, -1, -2, -3]
    assert [serve.stream_priority(k, (0, -1)) for k in range(4)] == [0, -1, -1, -1]
    assert [serve.stream_priority(k, (0, 0)) for k in range(4)] == [0, 0, 0, 0]


def test_serving_trace_spans_the_priority_classes(serve):
    wls = gi.serving_requests(32, seed=4, steps=50)
    levels = {serve.priority_level(serve.pushes(wl, 50)) for wl in wls}
    assert len(levels) >= 3


def test_nearest_rank_percentiles(serve):
    recs = []
    for i, lat in enumerate([5.0, 1.0, 3.0, 2.0, 4.0]):
        r = serve.RunRecord(i, 0.0)
        r.finish = lat
        recs.append(r)
    bad = serve.RunRecord(9, 0.0)
    bad.error = "rejected"
    res = serve.ServeResult(recs + [bad], makespan=5.0, max_concurrent=5, chunk=1)
    assert res.percentile(50) == 3.0 and res.percentile(99) == 5.0 and res.percentile(1) == 1.0
    assert res.runs_per_s == 1.0
    assert math.isnan(serve.ServeResult([bad], 1.0, 1, 1).percentile(50))


def test_run_strategy_and_share_key(serve):
    """FP32 linear runs take the one-thread-per-cell pass; cubic, FP64 and deterministic
    runs the default grouped deposit; the strategy is part of the shared-launch key, so
    runs of different strategies never share launches."""
    lin = gi.drifting_plasma(32, 32, 32, 10.0, shape_order=1, precision=32)
    cub = gi.drifting_plasma(32, 32, 32, 10.0, shape_order=3, precision=32)
    assert serve.run_strategy(lin, 32) == (1, 4)
    assert serve.run_strategy(lin, 64) == (1, 0)
    assert serve.run_strategy(cub, 32) == (1, 0)
    det = gi.drifting_plasma(32, 32, 32, 10.0, shape_order=1, precision=32)
    det.deterministic = 1
    assert serve.run_strategy(det, 32) == (1, 0)
    assert serve.share_key(lin, 32, 1, 4) != serve.share_key(lin, 32, 1, 0)
    assert serve.share_key(lin, 32, 1, 4) == serve.share_key(
        gi.drifting_plasma(32, 32, 32, 30.0, shape_order=1, precision=32, seed=9), 32, 1, 4)
