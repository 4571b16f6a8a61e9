"""Seeded synthetic inputs shared by the FP64 oracle, the tests and the bench.

This module only draws random numbers.  It holds none of the arithmetic of the
maintained programs (no products, no inverses, no delta rules), so both the
CUDA path and the oracle may import it without sharing any method code.

Recipes (all FP64 draws from numpy's PCG64 ``default_rng``; a workload-level
``seed`` is split into independent sub-streams with ``SeedSequence``):

* ``power_matrix``: dense A with i.i.d. N(0,1)/(2*sqrt(n)) entries, so the
  spectral radius is about 0.5 (circular law).  This stands in for the paper's
  "dense random matrices ... preconditioned appropriately" (Section 6,
  workload paragraph).
* ``row_update_stream``: rank-1 row updates dA = e_i v^T, i uniform in [0, n)
  drawn with replacement, v i.i.d. N(0, sigma^2) with sigma = 0.01 (the paper's
  "continuous random stream of rank-1 updates where each update affects one
  row", Section 6).
* ``lowrank_update_stream``: rank-r updates dA = U V^T, U and V i.i.d.
  N(0, sigma^2), n x r.
* ``iteration_inputs``: A as above, B and T_0 i.i.d. N(0,1), n x p (general
  form T_{i+1} = A T_i + B, Section 4.3).
* ``ols_inputs`` / ``ols_row_replacements``: X (m x n) i.i.d. N(0,1) with a
  fixed random 10% of the columns scaled by 1e-2, Y (m x p) i.i.d. N(0,1); an
  update replaces k distinct rows of X by fresh rows drawn the same way (same
  scaled columns), Y unchanged (OLS, Section 4.1).

* ``serving_views`` / ``serving_trace``: many maintained A^k views with n drawn
  uniformly from a size set, and an open-loop request trace: Poisson arrivals
  (exponential gaps at ``rate`` per second), target view uniform, rank
  uniform in 1..r_hi, U and V i.i.d. N(0, sigma^2); the factors of all
  requests packed in one float32 array (U_i then V_i, each n x rank
  row-major).  The paper streams rank-1 updates and batches of updates
  (Section 6); the rate sweep and the mix of sizes are this build's serving
  workload.

* ``zipf_row_batch``: a batch of row updates whose rows follow a Zipf law
  (frequency of the i-th most popular row proportional to i^-z over a random
  ordering of the n rows; z = 0 is uniform), v i.i.d. N(0, sigma^2): the
  batch-update workload of Section 6 (Table 4, batches of 1,000 updates,
  Zipf factors 5 to 0).

``dtype`` rounds the FP64 draw to nearest in the requested type; consumers that
compare against the FP64 oracle promote the rounded values back to FP64, so the
comparison measures the method's error and not input quantisation.
"""
from __future__ import annotations

import numpy as np

# Sub-stream identifiers, so that e.g. the matrix and the updates of one
# workload never share random numbers.
_STREAM_MATRIX = 1
_STREAM_UPDATES = 2
_STREAM_ITER_B = 3
_STREAM_ITER_T0 = 4
_STREAM_OLS_X = 5
_STREAM_OLS_Y = 6
_STREAM_OLS_COLS = 7
_STREAM_OLS_UPD = 8
_STREAM_MISC = 9
_STREAM_SERVE_SIZES = 10
_STREAM_SERVE_TRACE = 11
_STREAM_ZIPF = 12


def rng(seed: int, stream: int) -> np.random.Generator:
    """Independent PCG64 generator for (workload seed, sub-stream id)."""
    return np.random.default_rng(np.random.SeedSequence([int(seed), int(stream)]))


def _cast(x: np.ndarray, dtype) -> np.ndarray:
    return np.ascontiguousarray(x.astype(dtype))


def power_matrix(n: int, seed: int = 0, dtype=np.float64) -> np.ndarray:
    """Dense n x n matrix, entries i.i.d. N(0,1)/(2 sqrt(n))."""
    g = rng(seed, _STREAM_MATRIX)
    a = g.standard_normal((n, n)) / (2.0 * np.sqrt(max(n, 1)))
    return _cast(a, dtype)


def row_update_stream(n: int, count: int, seed: int = 0, sigma: float = 0.01,
                      dtype=np.float64):
    """List of ``count`` row updates (i, v): dA = e_i v^T."""
    g = rng(seed, _STREAM_UPDATES)
    out = []
    for _ in range(count):
        i = int(g.integers(0, n))
        v = _cast(sigma * g.standard_normal(n), dtype)
        out.append((i, v))
    return out


def lowrank_update_stream(n: int, r: int, count: int, seed: int = 0,
                          sigma: float = 0.01, dtype=np.float64, n_cols: int | None = None):
    """List of ``count`` factored updates (U, V), U n x r, V n_cols x r."""
    g = rng(seed, _STREAM_UPDATES)
    m = n if n_cols is None else n_cols
    out = []
    for _ in range(count):
        u = _cast(sigma * g.standard_normal((n, r)), dtype)
        v = _cast(sigma * g.standard_normal((m, r)), dtype)
        out.append((u, v))
    return out


def row_as_factors(n: int, i: int, v: np.ndarray):
    """Factored form (U, V) of the row update e_i v^T (U = e_i, V = v)."""
    u = np.zeros((n, 1), dtype=v.dtype)
    u[i, 0] = 1
    return u, v.reshape(n, 1).copy()


def iteration_inputs(n: int, p: int, seed: int = 0, dtype=np.float64):
    """(A, B, T0) for T_{i+1} = A T_i + B: A as ``power_matrix``, B, T0 ~ N(0,1)."""
    a = power_matrix(n, seed, dtype)
    b = _cast(rng(seed, _STREAM_ITER_B).standard_normal((n, p)), dtype)
    t0 = _cast(rng(seed, _STREAM_ITER_T0).standard_normal((n, p)), dtype)
    return a, b, t0


def ols_scaled_columns(n: int, seed: int = 0, frac: float = 0.1) -> np.ndarray:
    """Sorted indices of the fixed random subset of columns scaled by 1e-2."""
    g = rng(seed, _STREAM_OLS_COLS)
    cnt = int(round(frac * n))
    return np.sort(g.choice(n, size=cnt, replace=False))


def _ols_rows(g: np.random.Generator, k: int, n: int, cols: np.ndarray, scale: float):
    x = g.standard_normal((k, n))
    x[:, cols] *= scale
    return x


def ols_inputs(m: int, n: int, p: int, seed: int = 0, frac: float = 0.1,
               scale: float = 1e-2, dtype=np.float64):
    """(X, Y, scaled_cols): X m x n with 10% columns x1e-2, Y m x p."""
    cols = ols_scaled_columns(n, seed, frac)
    x = _ols_rows(rng(seed, _STREAM_OLS_X), m, n, cols, scale)
    y = rng(seed, _STREAM_OLS_Y).standard_normal((m, p))
    return _cast(x, dtype), _cast(y, dtype), cols


def ols_row_replacements(m: int, n: int, k: int, count: int, seed: int = 0,
                         frac: float = 0.1, scale: float = 1e-2, dtype=np.float64,
                         cols_seed: int | None = None):
    """List of ``count`` updates (rows, new_rows): k distinct rows in [0, m)
    replaced by fresh rows with the same column scaling as X: ``cols_seed`` is
    the seed X was drawn with (its scaled columns); None uses ``seed``."""
    cols = ols_scaled_columns(n, seed if cols_seed is None else cols_seed, frac)
    g = rng(seed, _STREAM_OLS_UPD)
    out = []
    for _ in range(count):
        rows = np.sort(g.choice(m, size=k, replace=False)).astype(np.int64)
        new = _cast(_ols_rows(g, k, n, cols, scale), dtype)
        out.append((rows, new))
    return out


def normal(shape, seed: int = 0, stream: int = _STREAM_MISC, scale: float = 1.0,
           dtype=np.float64) -> np.ndarray:
    """Generic i.i.d. N(0, scale^2) array (test helpers, FD directions)."""
    return _cast(scale * rng(seed, stream).standard_normal(shape), dtype)


def serving_views(count: int, sizes=(1024, 2048, 4096, 8192), seed: int = 0):
    """Sizes n of ``count`` views, each drawn uniformly from ``sizes``."""
    g = rng(seed, _STREAM_SERVE_SIZES)
    return [int(sizes[i]) for i in g.integers(0, len(sizes), size=count)]


def serving_trace(view_sizes, count: int, rate: float, seed: int = 0, r_hi: int = 8,
                  sigma: float = 0.01):
    """Open-loop trace of ``count`` requests over views with sizes
    ``view_sizes``: (t_s, views, ranks, factors, offsets), t_s in seconds
    from the start; request i's U is factors[offsets[i]:][:n*rank] (n x rank
    row-major) and its V the n*rank floats after it."""
    g = rng(seed, _STREAM_SERVE_TRACE)
    gaps = g.exponential(1.0 / rate, size=count)
    t_s = np.cumsum(gaps) - gaps[0]
    views = g.integers(0, len(view_sizes), size=count).astype(np.int32)
    ranks = g.integers(1, r_hi + 1, size=count).astype(np.int32)
    sizes = np.array([2 * view_sizes[v] * r for v, r in zip(views, ranks)], dtype=np.int64)
    offsets = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    factors = (sigma * g.standard_normal(int(sizes.sum()))).astype(np.float32)
    return t_s.astype(np.float64), views, ranks, factors, offsets


def trace_factors(view_sizes, views, ranks, factors, offsets, i: int):
    """(U_i, V_i) of request i of a ``serving_trace`` (views into ``factors``)."""
    n, r, o = view_sizes[views[i]], int(ranks[i]), int(offsets[i])
    return factors[o:o + n * r].reshape(n, r), factors[o + n * r:o + 2 * n * r].reshape(n, r)


def zipf_row_batch(n: int, count: int, z: float, seed: int = 0, sigma: float = 0.01,
                   dtype=np.float32):
    """(rows, vs): ``count`` row updates e_rows[j] vs[j]^T, rows Zipf(z)-distributed."""
    g = rng(seed, _STREAM_ZIPF)
    perm = g.permutation(n)
    w = np.arange(1, n + 1, dtype=np.float64) ** (-float(z))
    ranks = g.choice(n, size=count, p=w / w.sum())
    rows = perm[ranks].astype(np.int64)
    vs = _cast(sigma * g.standard_normal((count, n)), dtype)
    return rows, vs

