"""The seeded synthetic inputs (the workloads of Section 6 at the sizes the
tests and the bench use): seeding, shapes, distributions and structure, as
the input recipe states them.  CPU only; no method arithmetic is involved."""
import numpy as np
import pytest

import linview_inputs as li


def test_power_matrix_seeded_scaled_and_rounded_once():
    n = 512
    a = li.power_matrix(n, seed=3)
    assert a.shape == (n, n) and a.dtype == np.float64
    assert np.array_equal(a, li.power_matrix(n, seed=3))
    assert not np.array_equal(a, li.power_matrix(n, seed=4))
    # N(0,1)/(2 sqrt n): sample std within 1% of 1/(2 sqrt n) over n^2 draws
    assert abs(a.std() * 2 * np.sqrt(n) - 1) < 0.01
    assert abs(a.mean()) * 2 * np.sqrt(n) < 0.01
    # the FP32 input is the FP64 draw rounded once (round to nearest)
    assert np.array_equal(li.power_matrix(n, seed=3, dtype=np.float32), a.astype(np.float32))
    # spectral radius ~ 0.5 (circular law): the "preconditioned" scale of the workload
    rho = np.abs(np.linalg.eigvals(a)).max()
    assert 0.4 < rho < 0.6


def test_row_update_stream_uniform_rows_with_repeats_and_sigma():
    n, cnt = 64, 4000
    ups = li.row_update_stream(n, cnt, seed=1)
    rows = np.array([i for i, _ in ups])
    vs = np.stack([v for _, v in ups])
    assert rows.min() >= 0 and rows.max() < n
    assert len(np.unique(rows)) < cnt            # repeats occur (i.i.d. with replacement)
    counts = np.bincount(rows, minlength=n)
    assert counts.min() > 0 and counts.max() < 3 * cnt / n
    assert abs(vs.std() / 0.01 - 1) < 0.01       # sigma = 0.01, not variance 0.01
    assert [(i, v.tolist()) for i, v in li.row_update_stream(n, 5, seed=1)] == \
        [(i, v.tolist()) for i, v in ups[:5]]


def test_row_as_factors_is_the_unit_column():
    v = np.arange(6, dtype=np.float32)
    u, vv = li.row_as_factors(6, 2, v)
    assert np.array_equal(u @ vv.T, np.outer(np.eye(6, dtype=np.float32)[2], v))


def test_ols_inputs_scaled_columns_and_replacements():
    m, n, p, k = 2000, 100, 3, 7
    x, y, cols = li.ols_inputs(m, n, p, seed=2)
    assert x.shape == (m, n) and y.shape == (m, p)
    assert np.array_equal(cols, li.ols_scaled_columns(n, seed=2)) and len(cols) == 10
    other = np.setdiff1d(np.arange(n), cols)
    assert abs(x[:, cols].std() / 1e-2 - 1) < 0.05
    assert abs(x[:, other].std() - 1) < 0.02
    ups = li.ols_row_replacements(m, n, k, 20, seed=2)
    for rows, new in ups:
        assert len(np.unique(rows)) == k and rows.min() >= 0 and rows.max() < m
        assert new.shape == (k, n)
    allnew = np.concatenate([new for _, new in ups])
    assert abs(allnew[:, cols].std() / 1e-2 - 1) < 0.1   # the same column scaling
    assert abs(allnew[:, other].std() - 1) < 0.05
    # an update stream drawn with its own seed keeps X's scaled columns
    ups2 = li.ols_row_replacements(m, n, k, 20, seed=9, cols_seed=2)
    new2 = np.concatenate([new for _, new in ups2])
    assert abs(new2[:, cols].std() / 1e-2 - 1) < 0.1 and abs(new2[:, other].std() - 1) < 0.05
    # so the leverage of a replacement row stays near n / m (not ~ n / m x 1e4)
    w = np.linalg.inv(x.T @ x)
    lev = np.einsum("ij,jk,ik->i", new2, w, new2)
    assert lev.max() < 4 * n / m


@pytest.mark.parametrize("z", [0.0, 1.0, 3.0])
def test_zipf_row_batch_skew(z):
    n, cnt = 1000, 5000
    rows, vs = li.zipf_row_batch(n, cnt, z, seed=5)
    assert rows.shape == (cnt,) and vs.shape == (cnt, n)
    assert rows.min() >= 0 and rows.max() < n
    distinct = len(np.unique(rows))
    if z == 0.0:
        assert distinct > 0.95 * n                 # uniform: nearly every row is hit
    else:
        top = np.bincount(rows).max() / cnt
        # the most frequent row takes about 1 / H(n, z) of the updates
        h = (np.arange(1, n + 1, dtype=np.float64) ** -z).sum()
        assert abs(top - 1 / h) < 0.03
    assert np.array_equal(rows, li.zipf_row_batch(n, cnt, z, seed=5)[0])
