"""Host-side checks of the serving workload's trace (no GPU)."""
import numpy as np

import linview_inputs as li


def test_trace_is_seeded_and_packed():
    sizes = li.serving_views(6, sizes=(64, 128), seed=2)
    assert sizes == li.serving_views(6, sizes=(64, 128), seed=2)
    assert set(sizes) <= {64, 128}
    t, v, r, f, o = li.serving_trace(sizes, 500, rate=1e3, seed=4)
    t2, v2, r2, f2, o2 = li.serving_trace(sizes, 500, rate=1e3, seed=4)
    for x, y in ((t, t2), (v, v2), (r, r2), (f, f2), (o, o2)):
        assert np.array_equal(x, y)
    assert t[0] == 0 and np.all(np.diff(t) >= 0)
    assert v.min() >= 0 and v.max() < len(sizes)
    assert r.min() >= 1 and r.max() <= 8
    # factors of consecutive requests tile the array without gaps
    ends = o + np.array([2 * sizes[a] * b for a, b in zip(v, r)])
    assert np.array_equal(o[1:], ends[:-1]) and ends[-1] == f.size
    u, w = li.trace_factors(sizes, v, r, f, o, 7)
    assert u.shape == (sizes[v[7]], r[7]) and w.shape == u.shape
    assert np.shares_memory(u, f)


def test_trace_rate_and_spread():
    sizes = [64] * 4
    t, v, r, f, o = li.serving_trace(sizes, 20000, rate=5e3, seed=1)
    # Poisson arrivals: mean gap 1/rate, coefficient of variation 1
    gaps = np.diff(t)
    assert abs(gaps.mean() * 5e3 - 1) < 0.03
    assert abs(gaps.std() / gaps.mean() - 1) < 0.05
    # uniform targets and ranks
    assert np.all(np.abs(np.bincount(v, minlength=4) / len(v) - 0.25) < 0.02)
    assert np.all(np.abs(np.bincount(r, minlength=9)[1:] / len(r) - 1 / 8) < 0.02)
    assert abs(f.std() - 0.01) < 1e-3
