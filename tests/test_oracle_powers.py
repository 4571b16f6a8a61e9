"""Pins of the FP64 oracle for powers and sums (CPU only).

Every check compares the oracle against something other than itself: brute
force in exact integer arithmetic or by the linear model, closed forms, the
paper's multiplication counts, or invariants."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import linview_inputs as li
from oracle import powers as op
from oracle.metrics import rel_frob

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _brute_views(a, k):
    """A^h by k-1 plain products (linear model), and the running sums."""
    pw = op.linear_powers(a, k)
    sums = np.cumsum(np.stack(pw), axis=0)
    return {h: pw[h - 1] for h in op.levels(k)}, {h: sums[h - 1] for h in op.levels(k)}


@pytest.mark.parametrize("n,r,k", [(2, 1, 2), (5, 1, 4), (8, 2, 8), (12, 3, 16), (16, 1, 16), (9, 4, 8)])
def test_incremental_matches_brute_force(n, r, k):
    a = li.power_matrix(n, seed=n)
    inc = op.IncrementalPowers(a, k, sums=True)
    acur = a.copy()
    for (u, v) in li.lowrank_update_stream(n, r, 4, seed=n + 1, sigma=0.3):
        f = inc.apply(u, v)
        acur = acur + u @ v.T
        bp, bs = _brute_views(acur, k)
        for h in op.levels(k):
            assert rel_frob(inc.p[h], bp[h]) < 1e-12
            assert rel_frob(inc.s[h], bs[h]) < 1e-12
            # factor widths are exactly h*r (Appendix A: U_i is n x i for r = 1)
            assert f["U"][h].shape == (n, h * r) and f["V"][h].shape == (n, h * r)
            assert f["Z"][h].shape == (n, h * r) and f["W"][h].shape == (n, h * r)


def test_row_updates_match_brute_force():
    n, k = 10, 8
    a = li.power_matrix(n, seed=3)
    inc = op.IncrementalPowers(a, k, sums=True)
    acur = a.copy()
    for i, v in li.row_update_stream(n, 6, seed=4, sigma=0.2):
        inc.apply_row(i, v)
        acur[i, :] += v
        bp, bs = _brute_views(acur, k)
        for h in op.levels(k):
            assert rel_frob(inc.p[h], bp[h]) < 1e-12
            assert rel_frob(inc.s[h], bs[h]) < 1e-12


@pytest.mark.parametrize("lam,k", [(0.7, 8), (-1.3, 16), (0.0, 4), (1.0, 16)])
def test_closed_form_scalar_matrix(lam, k):
    # (lam I + u v^T)^h = lam^h I + ((lam+alpha)^h - lam^h)/alpha u v^T, alpha = v^T u
    n = 7
    g = np.random.default_rng(11)
    u = g.standard_normal((n, 1)) * 0.5
    v = g.standard_normal((n, 1)) * 0.5
    alpha = float((v.T @ u)[0, 0])
    inc = op.IncrementalPowers(lam * np.eye(n), k, sums=True)
    inc.apply(u, v)
    uv = u @ v.T
    ssum = np.zeros((n, n))
    for h in range(1, k + 1):
        coef = ((lam + alpha) ** h - lam ** h) / alpha
        ph = lam ** h * np.eye(n) + coef * uv
        ssum = ssum + ph
        if h in op.levels(k):
            assert rel_frob(inc.p[h], ph) < 1e-13
            assert rel_frob(inc.s[h], ssum) < 1e-13


def test_closed_form_alpha_zero():
    # alpha = v^T u = 0: (lam I + u v^T)^h = lam^h I + h lam^{h-1} u v^T
    n, k, lam = 6, 16, 0.9
    u = np.zeros((n, 1)); u[0, 0] = 1.0
    v = np.zeros((n, 1)); v[3, 0] = 2.0
    inc = op.IncrementalPowers(lam * np.eye(n), k)
    inc.apply(u, v)
    for h in op.levels(k):
        ph = lam ** h * np.eye(n) + h * lam ** (h - 1) * (u @ v.T)
        assert rel_frob(inc.p[h], ph) < 1e-14


def test_diagonal_stays_diagonal():
    n, k = 9, 16
    d = np.linspace(-0.9, 0.8, n)
    inc = op.IncrementalPowers(np.diag(d), k, sums=True)
    i, delta = 4, 0.35
    u = np.zeros((n, 1)); u[i, 0] = 1.0
    v = np.zeros((n, 1)); v[i, 0] = delta
    inc.apply(u, v)
    d2 = d.copy(); d2[i] += delta
    for h in op.levels(k):
        assert np.allclose(inc.p[h], np.diag(d2 ** h), atol=1e-15, rtol=1e-13)
        assert np.allclose(inc.s[h], np.diag(sum(d2 ** j for j in range(1, h + 1))),
                           atol=1e-15, rtol=1e-13)


def _int_matpow(m, e):
    n = len(m)
    out = [[int(i == j) for j in range(n)] for i in range(n)]
    for _ in range(e):
        out = [[sum(out[i][t] * m[t][j] for t in range(n)) for j in range(n)] for i in range(n)]
    return out


def test_nilpotent_exact_integers():
    # strict upper shift N: N^h = 0 for h >= n; small integer update -> exact in FP64
    n, k = 6, 16
    nmat = [[1 if j == i + 1 else 0 for j in range(n)] for i in range(n)]
    inc = op.IncrementalPowers(np.array(nmat, dtype=np.float64), k, sums=True)
    assert all(not inc.p[h].any() for h in op.levels(k) if h >= n)
    u = [1, 0, -1, 0, 0, 1]
    v = [0, 1, 0, 0, -1, 0]
    inc.apply(np.array(u, dtype=np.float64), np.array(v, dtype=np.float64))
    a2 = [[nmat[i][j] + u[i] * v[j] for j in range(n)] for i in range(n)]
    for h in op.levels(k):
        exact = np.array(_int_matpow(a2, h), dtype=np.float64)
        assert np.array_equal(inc.p[h], exact)
        s = sum(np.array(_int_matpow(a2, j), dtype=np.float64) for j in range(1, h + 1))
        assert np.array_equal(inc.s[h], s)


def test_sums_relation_to_paper_sums():
    # S'_k = S_k + P_k - I with the paper's S_k = I + A + ... + A^{k-1}
    n, k = 11, 16
    a = li.power_matrix(n, seed=5)
    s = op.reeval_sums(a, k)
    p = op.reeval_powers(a, k)
    assert rel_frob(s[k], op.paper_sums(a, k) + p[k] - np.eye(n)) < 1e-13


def test_delta_rank_bound():
    # rank(dP_h) <= h r  (Appendix A: U_i, V_i are n x i for r = 1)
    n, k, r = 24, 8, 2
    a = li.power_matrix(n, seed=6)
    inc = op.IncrementalPowers(a, k)
    before = {h: inc.p[h].copy() for h in op.levels(k)}
    (u, v), = li.lowrank_update_stream(n, r, 1, seed=7, sigma=0.5)
    inc.apply(u, v)
    for h in op.levels(k):
        sv = np.linalg.svd(inc.p[h] - before[h], compute_uv=False)
        rank = int(np.sum(sv > 1e-10 * sv[0]))
        assert rank <= h * r
        assert rank == min(h * r, n)  # generic inputs reach the bound


def test_op_counts_match_appendix_a():
    gold = json.load(open(os.path.join(GOLD, "opcounts_appendix_a.json")))
    for row in gold["exponential_total"]:
        n, k = row["n"], row["k"]
        inc = op.IncrementalPowers(li.power_matrix(n, seed=1), k)
        inc.apply(*li.lowrank_update_stream(n, 1, 1, seed=2)[0])
        assert inc.ops.mults == row["mults"], (n, k)
    # per level: run k = i/2 .. i programs and difference the totals
    n = 8
    prev = None
    for row in gold["exponential_per_level_n8"]:
        inc = op.IncrementalPowers(li.power_matrix(n, seed=1), row["i"])
        inc.apply(*li.lowrank_update_stream(n, 1, 1, seed=2)[0])
        tot = inc.ops.mults
        base = n * n if prev is None else prev
        assert tot - base == row["mults"]
        prev = tot
    for row in gold["linear_total"]:
        n, k = row["n"], row["k"]
        inc = op.LinearIncrementalPowers(li.power_matrix(n, seed=1), k)
        inc.apply(*li.lowrank_update_stream(n, 1, 1, seed=2)[0])
        assert inc.ops.mults == row["mults"], (n, k)


def test_linear_model_incremental_matches_brute_force():
    n, k = 7, 6
    a = li.power_matrix(n, seed=8)
    inc = op.LinearIncrementalPowers(a, k)
    acur = a.copy()
    for (u, v) in li.lowrank_update_stream(n, 2, 3, seed=9, sigma=0.3):
        inc.apply(u, v)
        acur += u @ v.T
        for h, ph in enumerate(op.linear_powers(acur, k), start=1):
            assert rel_frob(inc.p[h - 1], ph) < 1e-12


def test_example_3_8_trigger_exact_integers():
    gold = json.load(open(os.path.join(GOLD, "example_3_8_a4_trigger.json")))
    a = [[2, -1, 0], [1, 3, 1], [0, -2, 1]]
    u = [1, 0, 2]
    v = [0, 1, -1]
    inc = op.IncrementalPowers(np.array(a, dtype=np.float64), 8)
    f = inc.apply(np.array(u, dtype=np.float64), np.array(v, dtype=np.float64))
    a2 = [[Fraction(a[i][j] + u[i] * v[j]) for j in range(3)] for i in range(3)]
    for name, h in (("B", 2), ("C", 4), ("D", 8)):
        assert f["U"][h].shape[1] == gold["factor_width_rank1"][name]
        # the factors reproduce the brute-force delta exactly
        delta = np.array(_int_matpow(a2, h), dtype=np.float64) - np.array(_int_matpow(a, h), dtype=np.float64)
        assert np.array_equal(f["U"][h] @ f["V"][h].T, delta)
    assert np.linalg.matrix_rank(f["U"][2] @ f["V"][2].T) <= gold["max_rank_dB"]
    assert np.array_equal(f["U"][2][:, 0], np.array(u, dtype=np.float64))
    assert np.array_equal(f["V"][2][:, 1], np.array(v, dtype=np.float64))


def test_power_rows_match_reeval():
    n, k = 20, 16
    a = li.power_matrix(n, seed=10)
    rows = [0, 7, 19]
    pr, sr = op.power_rows(a, rows, k)
    lin = op.linear_powers(a, k)
    for h in op.levels(k):
        assert rel_frob(pr[h], lin[h - 1][rows]) < 1e-13
        assert rel_frob(sr[h], sum(lin[j][rows] for j in range(h))) < 1e-13


def test_power_rows_factored_against_library_power():
    """Rows of (A0 + U V^T)^h and of S'_h from the factored form vs
    numpy.linalg.matrix_power of the formed matrix (a library routine), for a
    row-update stream (U = unit columns) and a dense rank-12 sum."""
    n, k = 24, 16
    a0 = li.power_matrix(n, seed=11)
    rows = [0, 5, 23]
    ups = li.row_update_stream(n, 7, seed=12)
    u_row = np.zeros((n, len(ups)))
    v_row = np.zeros((n, len(ups)))
    for j, (i, v) in enumerate(ups):
        u_row[i, j] = 1.0
        v_row[:, j] = v
    g = np.random.default_rng(13)
    u_dense = g.standard_normal((n, 12)) * 0.05
    v_dense = g.standard_normal((n, 12)) * 0.05
    for u, v in ((u_row, v_row), (u_dense, v_dense)):
        a = a0 + u @ v.T
        pr, sr = op.power_rows_factored(a0, u, v, rows, k)
        for h in op.levels(k):
            ref = np.linalg.matrix_power(a, h)[rows]
            assert rel_frob(pr[h], ref) < 1e-13, h
            sref = sum(np.linalg.matrix_power(a, j)[rows] for j in range(1, h + 1))
            assert rel_frob(sr[h], sref) < 1e-13, h
    # a dropped factor term is visible: the update is not negligible
    pr0, _ = op.power_rows_factored(a0, u_dense * 0.0, v_dense, rows, k)
    assert rel_frob(pr0[16], np.linalg.matrix_power(a0 + u_dense @ v_dense.T, 16)[rows]) > 1e-6


def _fd_power_grad(a, k, g, e, step=1e-4):
    def loss(x):
        return float(np.sum(g * op.linear_powers(x, k)[-1]))
    return (loss(a + step * e) - loss(a - step * e)) / (2 * step)


@pytest.mark.parametrize("n,k", [(6, 4), (10, 16)])
def test_power_adjoint_chain_vs_sum_and_fd(n, k):
    a = li.power_matrix(n, seed=12)
    g = li.normal((n, n), seed=13)
    chain = op.adjoint_power_chain(a, k, g)
    direct = op.adjoint_power_sum(a, k, g)
    assert rel_frob(chain, direct) < 1e-12
    gscale = float(np.linalg.norm(chain))
    for t in range(6):
        e = li.normal((n, n), seed=20 + t)
        e /= np.linalg.norm(e)  # unit direction: O(h^2) truncation stays ~1e-6
        fd = _fd_power_grad(a, k, g, e)
        an = float(np.sum(chain * e))
        assert abs(fd - an) <= 1e-6 * gscale


# ---------------------------------------------------------------- skip-s model
@pytest.mark.parametrize("k,s,r", [(8, 2, 1), (12, 4, 2), (16, 4, 1), (16, 2, 3)])
def test_skip_model_incremental_matches_brute_force(k, s, r):
    """Appendix A skip-s rules against re-evaluation of the updated A after
    every update (products of the definition P_i = P_s P_{i-s})."""
    n = 9
    a = li.power_matrix(n, seed=k + s)
    inc = op.SkipIncrementalPowers(a, k, s)
    acur = a.copy()
    for (u, v) in li.lowrank_update_stream(n, r, 3, seed=k * s, sigma=0.3):
        inc.apply(u, v)
        acur += u @ v.T
        for h in op.skip_levels(k, s):
            assert rel_frob(inc.p[h], np.linalg.matrix_power(acur, h)) < 1e-12, h


def test_skip_model_special_cases():
    """s = 1 is the linear model and s = k/2 is the exponential model: the
    factors of the three rule sets coincide."""
    n, k = 6, 8
    a = li.power_matrix(n, seed=3)
    u, v = li.lowrank_update_stream(n, 2, 1, seed=4, sigma=0.2)[0]
    sk = op.SkipIncrementalPowers(a, k, 1)
    lin = op.LinearIncrementalPowers(a, k)
    U1, V1 = sk.apply(u, v)
    U2, V2 = lin.apply(u, v)
    for i in range(1, k + 1):
        assert np.allclose(U1[i], U2[i - 1], rtol=0, atol=1e-14)
        assert np.allclose(V1[i], V2[i - 1], rtol=0, atol=1e-14)
    sk = op.SkipIncrementalPowers(a, k, k // 2)
    ex = op.IncrementalPowers(a, k)
    U1, V1 = sk.apply(u, v)
    f = ex.apply(u, v)
    for h in op.levels(k):
        assert np.allclose(U1[h], f["U"][h], rtol=0, atol=1e-14)
        assert np.allclose(V1[h], f["V"][h], rtol=0, atol=1e-14)


@pytest.mark.parametrize("n,k,s", [(10, 8, 2), (16, 16, 4), (12, 12, 4)])
def test_skip_model_multiplication_count(n, k, s):
    """Appendix A, skip model: the levels above s cost
    sum_{i = 2s, 3s, .., k} (2 n^2 i + n (2s + 1)(i - s)) multiplications for
    a rank-1 update, on top of the exponential model's n^2 (4s - 3) +
    n (s - 1)(2s + 5) / 3 for P_1 .. P_s."""
    inc = op.SkipIncrementalPowers(li.power_matrix(n, seed=1), k, s)
    inc.apply(*li.lowrank_update_stream(n, 1, 1, seed=2)[0])
    exp_part = n * n * (4 * s - 3) + n * (s - 1) * (2 * s + 5) // 3
    skip_part = sum(2 * n * n * i + n * (2 * s + 1) * (i - s) for i in range(2 * s, k + 1, s))
    assert inc.ops.mults == exp_part + skip_part


@pytest.mark.parametrize("k,s", [(8, 2), (12, 4), (16, 4)])
def test_skip_sums_recurrence_is_the_definition(k, s):
    """The skip model's sum recurrence S'_i = P_s S'_{i-s} + S'_s gives
    A + A^2 + ... + A^i (brute force)."""
    n = 7
    a = li.power_matrix(n, seed=k * s)
    sm = op.skip_sums(a, k, s)
    assert sorted(sm) == op.skip_levels(k, s)[1:]
    for h, v in sm.items():
        ref = sum(np.linalg.matrix_power(a, i) for i in range(1, h + 1))
        assert rel_frob(v, ref) < 1e-13


def test_level_products_by_loops_and_the_squaring_rule():
    """One Appendix-A level, (P U, P^T V, P + U V^T), against explicit sums
    over small integers (exact), and its use in the rule for the next power:
    (P + U V^T)^2 - P^2 = U_2 V_2^T with U_2 = [U, P U + U (V^T U)],
    V_2 = [P^T V, V]."""
    g = np.random.default_rng(7)
    n, r = 5, 2
    p = g.integers(-3, 4, (n, n)).astype(np.float64)   # not symmetric
    u = g.integers(-3, 4, (n, r)).astype(np.float64)
    v = g.integers(-3, 4, (n, r)).astype(np.float64)
    assert not np.array_equal(p, p.T)
    x, y, p_new = op.level_products(p, u, v)
    for i in range(n):
        for c in range(r):
            assert x[i, c] == sum(p[i, j] * u[j, c] for j in range(n))
            assert y[i, c] == sum(p[j, i] * v[j, c] for j in range(n))
        for j in range(n):
            assert p_new[i, j] == p[i, j] + sum(u[i, c] * v[j, c] for c in range(r))
    u2 = np.concatenate([u, x + u @ (v.T @ u)], axis=1)
    v2 = np.concatenate([y, v], axis=1)
    assert np.array_equal(p_new @ p_new - p @ p, u2 @ v2.T)


@pytest.mark.parametrize("k,s", [(16, 4), (16, 2), (12, 4), (8, 8)])
def test_skip_powers_against_library_matrix_power(k, s):
    """Skip-s model views (squarings up to A^s, then A^i = A^s A^(i-s)) equal
    numpy.linalg.matrix_power at every maintained h; small integers keep the
    products exact."""
    g = np.random.default_rng(k * 10 + s)
    a = g.integers(-1, 2, (6, 6)).astype(np.float64)
    got = op.skip_powers(a, k, s)
    hs = sorted(got)
    assert hs == sorted(set([1 << j for j in range(s.bit_length()) if (1 << j) <= s] +
                            list(range(2 * s, k + 1, s))))
    for h in hs:
        assert np.array_equal(got[h], np.linalg.matrix_power(a, h)), h
