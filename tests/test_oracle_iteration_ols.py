"""Pins of the FP64 oracle for the general iteration and for OLS (CPU only)."""
import numpy as np
import pytest

import linview_inputs as li
from oracle import iteration as oi
from oracle import ols as oo
from oracle import powers as op
from oracle.metrics import rel_frob


# ---------------------------------------------------------------- iteration
@pytest.mark.parametrize("n,p,k,r", [(8, 3, 16, 1), (16, 5, 8, 2), (5, 1, 4, 3)])
def test_iteration_incremental_and_hybrid_match_reeval(n, p, k, r):
    a, b, t0 = li.iteration_inputs(n, p, seed=n)
    inc = oi.IncrementalIteration(a, b, t0, k)
    hyb = oi.HybridIteration(a, b, t0, k)
    acur = a.copy()
    for (u, v) in li.lowrank_update_stream(n, r, 3, seed=n + 7, sigma=0.2):
        U, V = inc.apply(u, v)
        hyb.apply(u, v)
        acur += u @ v.T
        ref = oi.reeval(acur, b, t0, k)
        for i in range(1, k + 1):
            assert rel_frob(inc.t[i], ref[i]) < 1e-12
            assert rel_frob(hyb.t[i], ref[i]) < 1e-12
            # Appendix B: U_i is n x i and V_i is p x i for a rank-1 update
            assert U[i].shape == (n, i * r) and V[i].shape == (p, i * r)


@pytest.mark.parametrize("n,p,k,rb", [(8, 3, 16, 1), (12, 7, 6, 2)])
def test_iteration_b_update_matches_reeval(n, p, k, rb):
    """Updates to B (dT_i = A dT_{i-1} + dB), interleaved with updates to A,
    against re-evaluation on the current inputs after every update."""
    a, b, t0 = li.iteration_inputs(n, p, seed=n + p)
    inc = oi.IncrementalIteration(a, b, t0, k)
    acur, bcur = a.copy(), b.copy()
    g = np.random.default_rng(n)
    for step in range(4):
        if step % 2:
            u, v = g.standard_normal((n, 1)) * 0.2, g.standard_normal((n, 1)) * 0.2
            inc.apply(u, v)
            acur += u @ v.T
        else:
            ub, vb = g.standard_normal((n, rb)), g.standard_normal((p, rb))
            U, V = inc.apply_b(ub, vb)
            bcur += ub @ vb.T
            assert U[k].shape == (n, k * rb) and V[k].shape == (p, k * rb)
        ref = oi.reeval(acur, bcur, t0, k)
        for i in range(1, k + 1):
            assert rel_frob(inc.t[i], ref[i]) < 1e-12


def test_iteration_b_update_closed_form():
    """A = lam I: dT_i = (1 + lam + ... + lam^(i-1)) dB exactly."""
    n, p, k, lam = 5, 3, 10, 0.7
    _, b, t0 = li.iteration_inputs(n, p, seed=4)
    inc = oi.IncrementalIteration(lam * np.eye(n), b, t0, k)
    before = [t.copy() for t in inc.t]
    g = np.random.default_rng(9)
    ub, vb = g.standard_normal((n, 1)), g.standard_normal((p, 1))
    inc.apply_b(ub, vb)
    for i in range(1, k + 1):
        geo = (1 - lam ** i) / (1 - lam)
        assert rel_frob(inc.t[i] - before[i], geo * (ub @ vb.T)) < 1e-13


def test_iteration_closed_form_scalar_plus_rank1():
    # A' = lam I + u v^T: A'^j = lam^j I + c_j u v^T, c_j = ((lam+alpha)^j - lam^j)/alpha,
    # T_i = A'^i T_0 + sum_{j<i} A'^j B  (unrolled form, Section 4.3)
    n, p, k, lam = 6, 2, 16, 0.8
    _, b, t0 = li.iteration_inputs(n, p, seed=3)
    g = np.random.default_rng(5)
    u = g.standard_normal((n, 1)) * 0.3
    v = g.standard_normal((n, 1)) * 0.3
    alpha = float((v.T @ u)[0, 0])
    inc = oi.IncrementalIteration(lam * np.eye(n), b, t0, k)
    inc.apply(u, v)

    def apow(j):
        return lam ** j * np.eye(n) + ((lam + alpha) ** j - lam ** j) / alpha * (u @ v.T)

    for i in range(1, k + 1):
        ti = apow(i) @ t0 + sum(apow(j) for j in range(i)) @ b
        assert rel_frob(inc.t[i], ti) < 1e-13


def test_iteration_unrolled_identity():
    # T_{i+s} = A^s T_i + (A^{s-1} + ... + I) B  (Section 4.3)
    n, p, k = 9, 4, 16
    a, b, t0 = li.iteration_inputs(n, p, seed=4)
    t = oi.reeval(a, b, t0, k)
    pw = op.reeval_powers(a, 8)
    for s in (1, 2, 4, 8):
        ssum = op.paper_sums(a, s) if s > 1 else np.eye(n)
        for i in (0, 3, 8):
            assert rel_frob(t[i + s], pw[s] @ t[i] + ssum @ b) < 1e-12


def _unit(x):
    return x / np.linalg.norm(x)


@pytest.mark.parametrize("n,p,k", [(12, 3, 16), (512, 64, 16)])
def test_iteration_adjoint_central_fd(n, p, k):
    # central differences, h = 1e-3, FP64; 8 random unit directions + single entries
    a, b, t0 = li.iteration_inputs(n, p, seed=21)
    da, db, dt0 = oi.adjoint(a, b, t0, k)
    h = 1e-3
    g = np.random.default_rng(22)
    dirs = [_unit(li.normal((n, n), seed=30 + t)) for t in range(8)]
    for _ in range(8 if n > 100 else 16):
        e = np.zeros((n, n)); e[g.integers(n), g.integers(n)] = 1.0
        dirs.append(e)
    # unit directions: |<dA, E>| <= ||dA||_F, and the O(h^2) truncation term is
    # far below 1e-6 ||dA||_F; a dropped or mis-signed term would be O(||dA||_F)
    gscale = float(np.linalg.norm(da))
    for e in dirs:
        fd = (oi.loss(a + h * e, b, t0, k) - oi.loss(a - h * e, b, t0, k)) / (2 * h)
        an = float(np.sum(da * e))
        assert abs(fd - an) <= 1e-6 * gscale, (fd, an)
    for t in range(3):
        e = _unit(li.normal((n, p), seed=40 + t))
        fd = (oi.loss(a, b + h * e, t0, k) - oi.loss(a, b - h * e, t0, k)) / (2 * h)
        assert abs(fd - float(np.sum(db * e))) <= 1e-6 * float(np.linalg.norm(db))
        fd = (oi.loss(a, b, t0 + h * e, k) - oi.loss(a, b, t0 - h * e, k)) / (2 * h)
        assert abs(fd - float(np.sum(dt0 * e))) <= 1e-6 * float(np.linalg.norm(dt0))


# ---------------------------------------------------------------------- OLS
def test_sherman_morrison_vs_library_inverse():
    n = 20
    g = np.random.default_rng(1)
    e = g.standard_normal((n, n)) + n * np.eye(n)
    u = g.standard_normal(n)
    v = g.standard_normal(n)
    einv = np.linalg.inv(e)
    got = einv + oo.sherman_morrison(einv, u, v)
    assert rel_frob(got, np.linalg.inv(e + np.outer(u, v))) < 1e-13


def test_sm_two_step_row_change():
    m, n, p = 60, 12, 2
    x, y, _ = li.ols_inputs(m, n, p, seed=2, frac=0.25)
    r = oo.reeval(x, y)
    d = np.random.default_rng(3).standard_normal(n)
    w2 = oo.sm_two_step(r["W"], x, 17, d)
    x2 = x.copy(); x2[17] += d
    assert rel_frob(w2, np.linalg.inv(x2.T @ x2)) < 1e-9


@pytest.mark.parametrize("k", [1, 4, 16])
def test_woodbury_row_blocks_vs_sm_and_lstsq(k):
    m, n, p = 400, 24, 3
    x, y, _ = li.ols_inputs(m, n, p, seed=5)
    a = oo.IncrementalOLS(x, y)
    b = oo.IncrementalOLS(x, y)
    for rows, new in li.ols_row_replacements(m, n, k, 3, seed=6, cols_seed=5):
        a.replace_rows(rows, new, "woodbury")
        b.replace_rows(rows, new, "sm")
    ref = oo.reeval(a.x, y)
    assert np.array_equal(a.x, b.x)
    assert rel_frob(a.w, ref["W"]) < 1e-9
    assert rel_frob(b.w, ref["W"]) < 1e-9
    assert rel_frob(a.z, ref["Z"]) < 1e-13
    assert rel_frob(a.xty, ref["XtY"]) < 1e-13
    beta_ls = np.linalg.lstsq(a.x, y, rcond=None)[0]   # independent library solver
    assert rel_frob(a.beta, beta_ls) < 1e-8


@pytest.mark.parametrize("k", [1, 3, 8])
def test_factored_beta_refresh_reaches_the_definition(k):
    """The CUDA path refreshes beta = W (X^T Y) by the delta of a product
    (Section 3.2) instead of recomputing W' C': with U = [X'_R^T, X_R^T],
    G = W U = [G_1, G_2], Wu = -G M^-1 (M = diag(I, -I) + U^T G),
    C' = X^T Y + (X'_R - X_R)^T Y_R and W' = W + G Wu^T,
        W' C' = beta + (G_1 - G_2) Y_R + G (Wu^T C').
    Checked against the oracle's beta (its definition W' C') over a few
    replacements, each starting from the previous refreshed beta."""
    m, n, p = 300, 20, 3
    x, y, _ = li.ols_inputs(m, n, p, seed=11)
    ref = oo.IncrementalOLS(x, y)
    w, beta, xty = ref.w.copy(), ref.beta.copy(), ref.xty.copy()
    for rows, new in li.ols_row_replacements(m, n, k, 4, seed=12, cols_seed=11):
        u = np.concatenate([new.T, ref.x[rows].T], axis=1)
        g = w @ u
        core = np.diag([1.0] * k + [-1.0] * k) + u.T @ g
        wu = -np.linalg.solve(core.T, g.T).T          # -G M^-1
        xty = xty + (new - ref.x[rows]).T @ y[rows]
        beta = beta + (g[:, :k] - g[:, k:]) @ y[rows] + g @ (wu.T @ xty)
        w = w + g @ wu.T
        ref.replace_rows(rows, new)
        assert rel_frob(w, ref.w) < 1e-12
        assert rel_frob(beta, ref.beta) < 1e-10


def test_ols_inputs_are_ill_conditioned():
    # 10% of columns scaled by 1e-2: kappa(X^T X) ~ 1e4 x ((sqrt m + sqrt n)/(sqrt m - sqrt n))^2
    m, n = 4096, 128
    x, _, cols = li.ols_inputs(m, n, 1, seed=0)
    assert len(cols) == round(0.1 * n)
    kappa = np.linalg.cond(x.T @ x)
    assert 5e3 < kappa < 1e5


def test_newton_schulz_step_pins():
    """The residual-correction step, pinned by what it must satisfy rather
    than by its formula: the exact inverse is a fixed point; from a perturbed
    inverse the new residual I - Z W' equals the square of the old one
    (quadratic convergence), so a few steps reach the library inverse; the
    beta refinement with the exact W lands on the solution of Z beta = X^T Y
    from any start.  A dropped factor W, a sign error or Z W for W Z breaks
    one of these (Z and W do not commute once W is perturbed)."""
    x, y, _ = li.ols_inputs(400, 30, 3, seed=5)
    z = x.T @ x
    w = np.linalg.inv(z)
    assert rel_frob(oo.newton_schulz_step(w, z), w) <= 1e-9
    g = np.random.default_rng(6)
    # W0 = W (I + d R): residual I - Z W0 = -d R (norm ~ 1e-2, inside the
    # iteration's region of convergence); not symmetric, so Z W0 != W0 Z
    w0 = w @ (np.eye(30) + 1e-3 * g.standard_normal((30, 30)))
    r0 = np.eye(30) - z @ w0
    w1 = oo.newton_schulz_step(w0, z)
    assert rel_frob(np.eye(30) - z @ w1, r0 @ r0) <= 1e-8
    wk = w0
    for _ in range(4):
        wk = oo.newton_schulz_step(wk, z)
    assert rel_frob(wk, w) <= 1e-9 < rel_frob(w0, w)
    xty = x.T @ y
    beta = np.linalg.lstsq(x, y, rcond=None)[0]
    start = beta + g.standard_normal(beta.shape)
    assert rel_frob(oo.refine_beta(w, start, xty, z), beta) <= 1e-8
    # with an approximate W the refinement contracts the error by I - W Z
    b1 = oo.refine_beta(w0, start, xty, z)
    assert rel_frob(b1 - beta, (np.eye(30) - w0 @ z) @ (start - beta)) <= 1e-8


# ------------------------------------------------- iteration, exponential model
@pytest.mark.parametrize("n,p,k", [(9, 3, 16), (6, 1, 2), (7, 4, 8)])
def test_exp_reeval_matches_linear_at_powers_of_two(n, p, k):
    """T_2h = P_h T_h + S_h B (S_h = I + ... + A^{h-1}) against the linear
    recurrence T_i = A T_{i-1} + B, and the A = lam I closed form
    T_h = lam^h T_0 + (1 + lam + ... + lam^{h-1}) B."""
    a, b, t0 = li.iteration_inputs(n, p, seed=3 * n)
    T, P, S = oi.exp_reeval(a, b, t0, k)
    lin = oi.reeval(a, b, t0, k)
    assert sorted(T) == [1 << j for j in range(k.bit_length())]
    for h in T:
        assert rel_frob(T[h], lin[h]) < 1e-12
    for h in P:
        assert rel_frob(P[h], np.linalg.matrix_power(a, h)) < 1e-12
        assert rel_frob(S[h], sum(np.linalg.matrix_power(a, i) for i in range(h))) < 1e-12
    lam = 0.7
    T, _, _ = oi.exp_reeval(lam * np.eye(n), b, t0, k)
    for h in T:
        assert rel_frob(T[h], lam ** h * t0 + sum(lam ** i for i in range(h)) * b) < 1e-13


@pytest.mark.parametrize("n,p,k,r", [(8, 3, 16, 1), (12, 5, 8, 2), (6, 1, 2, 1), (5, 2, 1, 1)])
def test_exp_incremental_matches_reeval(n, p, k, r):
    """The printed exponential rule (old P_h, S_h, T_h; every += last) keeps
    T_h, P_h and S_h equal to their re-evaluation on the updated A; the width
    of U_h follows the recurrence with dS_1 = 0: r * (1, 2, 5, 12, 27) for
    h = 1, 2, 4, 8, 16 (the paper's 2i - 1 is an upper bound)."""
    a, b, t0 = li.iteration_inputs(n, p, seed=n + 1)
    inc = oi.ExpIncrementalIteration(a, b, t0, k)
    acur = a.copy()
    widths = {1: 1, 2: 2, 4: 5, 8: 12, 16: 27}
    for (u, v) in li.lowrank_update_stream(n, r, 3, seed=n + 2, sigma=0.2):
        U, V = inc.apply(u, v)
        acur += u @ v.T
        T, P, S = oi.exp_reeval(acur, b, t0, k)
        for h in T:
            assert rel_frob(inc.t[h], T[h]) < 1e-12, h
            assert U[h].shape == (n, r * widths[h]) and V[h].shape == (p, r * widths[h])
            assert U[h].shape[1] <= r * (2 * h - 1) or h == 1
        for h in P:
            assert rel_frob(inc.p[h], P[h]) < 1e-12
            assert rel_frob(inc.s[h], S[h]) < 1e-12


# ------------------------------------------------------ iteration, skip model
@pytest.mark.parametrize("n,p,k,s,r", [(8, 3, 16, 4, 1), (9, 2, 8, 2, 2), (6, 1, 4, 1, 1),
                                       (7, 3, 16, 8, 1), (5, 2, 6, 2, 1)])
def test_skip_incremental_matches_reeval(n, p, k, s, r):
    """Skip-s model: re-evaluation T_i = P_s T_{i-s} + S_s B against the linear
    recurrence, and the printed incremental rule against it after updates."""
    a, b, t0 = li.iteration_inputs(n, p, seed=n + 5)
    inc = oi.SkipIncrementalIteration(a, b, t0, k, s)
    expect = sorted({1 << j for j in range(s.bit_length())} | set(range(2 * s, k + 1, s)))
    assert sorted(inc.t) == expect
    acur = a.copy()
    for (u, v) in li.lowrank_update_stream(n, r, 3, seed=n + 6, sigma=0.2):
        U, V = inc.apply(u, v)
        acur += u @ v.T
        T, P, S = oi.skip_reeval(acur, b, t0, k, s)
        lin = oi.reeval(acur, b, t0, k)
        for i in T:
            assert rel_frob(T[i], lin[i]) < 1e-12, i
            assert rel_frob(inc.t[i], T[i]) < 1e-12, i
        for h in P:
            assert rel_frob(inc.p[h], P[h]) < 1e-12
            assert rel_frob(inc.sv[h], S[h]) < 1e-12


def test_skip_special_cases_and_widths():
    """s = k/2 is the exponential model and s = 1 the linear model (same views,
    same factor widths); at s = 4, k = 16 the widths follow the recurrence
    w_i = r s + w_{i-s} + (width of Z_s): r * (1, 2, 5, 12, 19, 26)."""
    n, p = 7, 2
    a, b, t0 = li.iteration_inputs(n, p, seed=41)
    (u, v), = li.lowrank_update_stream(n, 1, 1, seed=42, sigma=0.2)
    sk = oi.SkipIncrementalIteration(a, b, t0, 16, 8)
    ex = oi.ExpIncrementalIteration(a, b, t0, 16)
    Us, _ = sk.apply(u, v)
    Ue, _ = ex.apply(u, v)
    assert sorted(Us) == sorted(Ue)
    for i in Us:
        assert Us[i].shape == Ue[i].shape
        assert rel_frob(sk.t[i], ex.t[i]) < 1e-13
    sk1 = oi.SkipIncrementalIteration(a, b, t0, 5, 1)
    lin = oi.IncrementalIteration(a, b, t0, 5)
    U1, _ = sk1.apply(u, v)
    Ul, _ = lin.apply(u, v)
    for i in range(1, 6):
        assert U1[i].shape == Ul[i].shape
        assert rel_frob(sk1.t[i], lin.t[i]) < 1e-13
    sk4 = oi.SkipIncrementalIteration(a, b, t0, 16, 4)
    U4, _ = sk4.apply(u, v)
    assert {i: U4[i].shape[1] for i in U4} == {1: 1, 2: 2, 4: 5, 8: 12, 12: 19, 16: 26}
    with pytest.raises(ValueError):
        oi.SkipIncrementalIteration(a, b, t0, 6, 4)


@pytest.mark.parametrize("k,s", [(16, 8), (16, 4), (8, 2), (5, 1)])
def test_exp_skip_b_updates_match_reeval(k, s):
    """Updates to B in the exponential / skip models (dT_1 = dB,
    dT_2h = P_h dT_h + S_h dB, dT_i = P_s dT_{i-s} + S_s dB), interleaved with
    updates to A, against re-evaluation on the current A and B; and the
    A = lam I closed form dT_i = (1 + lam + .. + lam^{i-1}) dB."""
    n, p = 9, 3
    a, b, t0 = li.iteration_inputs(n, p, seed=k + s)
    inc = (oi.ExpIncrementalIteration(a, b, t0, k) if s == k // 2
           else oi.SkipIncrementalIteration(a, b, t0, k, s))
    acur, bcur = a.copy(), b.copy()
    g = np.random.default_rng(k * s)
    for step in range(4):
        if step % 2:
            u, v = g.standard_normal((n, 2)) * 0.2, g.standard_normal((n, 2)) * 0.2
            inc.apply(u, v)
            acur += u @ v.T
        else:
            ub, vb = g.standard_normal((n, 2)), g.standard_normal((p, 2))
            inc.apply_b(ub, vb)
            bcur += ub @ vb.T
        T, _, _ = oi.skip_reeval(acur, bcur, t0, k, s)
        for i in T:
            assert rel_frob(inc.t[i], T[i]) < 1e-12, i
    lam = 0.6
    inc = oi.SkipIncrementalIteration(lam * np.eye(n), b, t0, k, s)
    before = {i: t.copy() for i, t in inc.t.items()}
    ub, vb = g.standard_normal((n, 1)), g.standard_normal((p, 1))
    inc.apply_b(ub, vb)
    for i in inc.t:
        assert rel_frob(inc.t[i] - before[i], sum(lam ** j for j in range(i)) * (ub @ vb.T)) < 1e-12
