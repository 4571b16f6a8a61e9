"""Matrix powers and sums of matrix powers -- FP64 oracle (test infrastructure).

Programs (Table 1 of the paper, exponential and linear models):

* powers, exponential model: P_1 = A, P_i = P_{i/2} P_{i/2} for i = 2, 4, ..., k;
* powers, linear model:      P_1 = A, P_i = A P_{i-1};
* sums of powers: the paper's S_k = I + A + ... + A^{k-1} (S_1 = I,
  S_i = P_{i/2} S_{i/2} + S_{i/2}); the maintained view is S'_h = A + ... + A^h,
  which obeys the same recurrence with S'_1 = A (so S'_k = S_k + P_k - I).

Incremental maintenance for a factored update dA = U V^T (Section 3.2):

* exponential model, Appendix A: with h = i/2,
      U_i = [U_h, P_h U_h + U_h (V_h^T U_h)],   V_i = [P_h^T V_h, V_h],
  all products taken on the views *before* the update; the view updates
  P_h += U_h V_h^T are applied after every factor is built (the trigger of
  Example 3.8 assigns all factors first and runs the += statements last);
* sums: the paper omits the rule (Section 4.2.3).  Applying the multi-matrix
  delta rule of Section 3.4 to S'_{2h} = P_h S'_h + S'_h gives
      dS'_{2h} = dP_h S'_h + P_h dS'_h + dP_h dS'_h + dS'_h,
  i.e. dS'_h = Z_h W_h^T with Z_1 = U_1, W_1 = V_1 and
      Z_{2h} = [U_h, P_h Z_h + U_h (V_h^T Z_h) + Z_h],  W_{2h} = [S'_h^T V_h, W_h];
* linear model, Appendix A: U_1 = U, V_1 = V and
      U_i = [U_1, A U_{i-1} + U_1 (V_1^T U_{i-1})],  V_i = [P_{i-1}^T V_1, V_{i-1}];
* skip-s model, Appendix A: P_1 .. P_s by the exponential model, then
  P_i = P_s P_{i-s} for i = 2s, 3s, ..., k, with
      U_i = [U_s, P_s U_{i-s} + U_s (V_s^T U_{i-s})],  V_i = [P_{i-s}^T V_s, V_{i-s}].

The instrumented ``ops`` counter tallies multiplications with the convention of
Appendix A (a product of an a x b by a b x c matrix costs a*b*c, the addition
inside U_i costs one per element, the += into the view itself is not counted);
the paper's closed forms for the totals are pinned against it in the tests.
"""
from __future__ import annotations

import numpy as np


def levels(k: int):
    """h = 1, 2, 4, ..., k (k a power of two)."""
    if k < 1 or (k & (k - 1)) != 0:
        raise ValueError("k must be a power of two")
    out, h = [], 1
    while h <= k:
        out.append(h)
        h *= 2
    return out


# --------------------------------------------------------------------------
# Re-evaluation (Table 1)
# --------------------------------------------------------------------------
def reeval_powers(a: np.ndarray, k: int) -> dict:
    """Exponential model: {h: A^h} for h = 1, 2, 4, ..., k."""
    a = np.asarray(a, dtype=np.float64)
    p = {1: a.copy()}
    for h in levels(k)[:-1]:
        p[2 * h] = p[h] @ p[h]
    return p


def skip_levels(k: int, s: int):
    """Views of the skip-s model: 1, 2, 4, ..., s, then 2s, 3s, ..., k."""
    if s < 1 or (s & (s - 1)) != 0 or k % s != 0 or k < 2 * s:
        raise ValueError("s must be a power of two and k a multiple of s with k >= 2s")
    return levels(s) + list(range(2 * s, k + 1, s))


def skip_powers(a: np.ndarray, k: int, s: int) -> dict:
    """Skip-s model: {h: A^h} for the views of ``skip_levels``: squarings up
    to P_s, then P_i = P_s P_{i-s}."""
    p = reeval_powers(a, s)
    for i in range(2 * s, k + 1, s):
        p[i] = p[s] @ p[i - s]
    return p


def skip_sums(a: np.ndarray, k: int, s: int) -> dict:
    """Sums S'_h = A + ... + A^h for the skip-s views h > 1, by the model's
    recurrences (Section 4.2.3): S'_{2h} = P_h S'_h + S'_h up to s, then
    S'_i = P_s S'_{i-s} + S'_s for i = 2s, 3s, ..., k (S'_1 = A)."""
    p = skip_powers(a, k, s)
    sm = {1: p[1].copy()}
    for h in levels(s)[:-1]:
        sm[2 * h] = p[h] @ sm[h] + sm[h]
    for i in range(2 * s, k + 1, s):
        sm[i] = p[s] @ sm[i - s] + sm[s]
    del sm[1]
    return sm


def linear_powers(a: np.ndarray, k: int) -> list:
    """Linear model: [A^1, A^2, ..., A^k] by k-1 products with A."""
    a = np.asarray(a, dtype=np.float64)
    out = [a.copy()]
    for _ in range(k - 1):
        out.append(a @ out[-1])
    return out


def reeval_sums(a: np.ndarray, k: int, p: dict | None = None) -> dict:
    """{h: S'_h = A + ... + A^h} by S'_1 = A, S'_{2h} = P_h S'_h + S'_h."""
    a = np.asarray(a, dtype=np.float64)
    if p is None:
        p = reeval_powers(a, k)
    s = {1: a.copy()}
    for h in levels(k)[:-1]:
        s[2 * h] = p[h] @ s[h] + s[h]
    return s


def paper_sums(a: np.ndarray, k: int) -> np.ndarray:
    """The paper's S_k = I + A + ... + A^{k-1} (S_1 = I, S_i = P_{i/2} S_{i/2} + S_{i/2})."""
    a = np.asarray(a, dtype=np.float64)
    p = reeval_powers(a, k)
    s = np.eye(a.shape[0])
    for h in levels(k)[:-1]:
        s = p[h] @ s + s
    return s


def power_rows(a: np.ndarray, rows, k: int):
    """Rows ``rows`` of every A^h (h = 1..k) and of S'_h, one row at a time:
    r <- e_i^T A, then r <- r A repeatedly (the plain definition).

    Returns (powers, sums): dicts h -> (len(rows) x n) arrays for h in levels(k).
    """
    a = np.asarray(a, dtype=np.float64)
    rows = np.asarray(rows, dtype=np.int64)
    cur = a[rows, :].copy()
    acc = cur.copy()
    want = set(levels(k))
    pw, sm = {}, {}
    for e in range(1, k + 1):
        if e > 1:
            cur = cur @ a
            acc = acc + cur
        if e in want:
            pw[e] = cur.copy()
            sm[e] = acc.copy()
    return pw, sm


def power_rows_factored(a0: np.ndarray, u: np.ndarray, v: np.ndarray, rows, k: int):
    """Rows ``rows`` of every A^h and S'_h (h in levels(k)) for the matrix
    A = A0 + U V^T held in factored form (U, V: n x q, the sum of the updates
    applied so far, Sec. 3.2), by the plain definition of power_rows:
    r <- e_i^T A, then r <- r A, where each product with A is taken as
    r A0 + (r U) V^T (the product distributes over the sum).  The n x n
    matrix A is never formed, so a long stream of rank-r updates at large n
    costs q extra columns instead of an n^2 update per step.

    Returns (powers, sums) as power_rows does.
    """
    a0 = np.asarray(a0, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64).reshape(a0.shape[0], -1)
    v = np.asarray(v, dtype=np.float64).reshape(a0.shape[0], -1)
    rows = np.asarray(rows, dtype=np.int64)

    def times_a(x):
        return x @ a0 + (x @ u) @ v.T

    cur = a0[rows, :] + u[rows, :] @ v.T
    acc = cur.copy()
    want = set(levels(k))
    pw, sm = {}, {}
    for e in range(1, k + 1):
        if e > 1:
            cur = times_a(cur)
            acc = acc + cur
        if e in want:
            pw[e] = cur.copy()
            sm[e] = acc.copy()
    return pw, sm


def level_products(p, u, v):
    """One level of Appendix A on a view P_h with factors U_h, V_h:
    (P_h U_h, P_h^T V_h, P_h + U_h V_h^T), products on the view before the
    update (the plain definitions)."""
    p = np.asarray(p, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    return p @ u, p.T @ v, p + u @ v.T


# --------------------------------------------------------------------------
# Incremental maintenance
# --------------------------------------------------------------------------
class _Ops:
    def __init__(self):
        self.mults = 0

    def mul(self, x, y):
        self.mults += x.shape[0] * x.shape[1] * (y.shape[1] if y.ndim == 2 else 1)
        return x @ y

    def add(self, x, y):
        self.mults += x.size
        return x + y


class IncrementalPowers:
    """Views P_h (and optionally S'_h) for h = 1, 2, ..., k, exponential model.

    ``apply(U, V)`` refreshes every view for dA = U V^T by the rules in the
    module docstring and returns the factors {h: (U_h, V_h)} (and Z_h, W_h).
    """

    def __init__(self, a: np.ndarray, k: int, sums: bool = False):
        self.k = k
        self.sums = sums
        self.p = reeval_powers(a, k)
        self.s = reeval_sums(a, k, self.p) if sums else None
        if sums:
            self.s[1] = self.p[1]  # S'_1 is the view A itself
        self.ops = _Ops()

    @property
    def a(self):
        return self.p[1]

    def apply(self, u: np.ndarray, v: np.ndarray):
        u = np.asarray(u, dtype=np.float64).reshape(self.a.shape[0], -1)
        v = np.asarray(v, dtype=np.float64).reshape(self.a.shape[1], -1)
        o = self.ops
        U, V = {1: u}, {1: v}
        Z, W = {1: u}, {1: v}
        hs = levels(self.k)
        # all factors from the views as they are before the update
        for h in hs[:-1]:
            ph = self.p[h]
            c = o.mul(V[h].T, U[h])                       # V_h^T U_h
            right = o.add(o.mul(ph, U[h]), o.mul(U[h], c))  # P_h U_h + U_h (V_h^T U_h)
            U[2 * h] = np.hstack([U[h], right])
            V[2 * h] = np.hstack([o.mul(ph.T, V[h]), V[h]])
            if self.sums:
                d = V[h].T @ Z[h]
                zr = ph @ Z[h] + U[h] @ d + Z[h]
                Z[2 * h] = np.hstack([U[h], zr])
                W[2 * h] = np.hstack([self.s[h].T @ V[h], W[h]])
        # update statements last (Example 3.8)
        for h in hs:
            self.p[h] += o.mul(U[h], V[h].T)
            if self.sums and h > 1:
                self.s[h] += Z[h] @ W[h].T
        return {"U": U, "V": V, "Z": Z, "W": W}

    def apply_row(self, i: int, v: np.ndarray):
        n = self.a.shape[0]
        u = np.zeros((n, 1))
        u[i, 0] = 1.0
        return self.apply(u, np.asarray(v, dtype=np.float64).reshape(n, 1))


class LinearIncrementalPowers:
    """Views P_1..P_k, linear model of Appendix A (``ops`` counts multiplications)."""

    def __init__(self, a: np.ndarray, k: int):
        self.k = k
        self.p = linear_powers(a, k)  # p[i-1] = A^i
        self.ops = _Ops()

    def apply(self, u: np.ndarray, v: np.ndarray):
        n = self.p[0].shape[0]
        u = np.asarray(u, dtype=np.float64).reshape(n, -1)
        v = np.asarray(v, dtype=np.float64).reshape(n, -1)
        o = self.ops
        a = self.p[0]
        U, V = [u], [v]
        for i in range(2, self.k + 1):
            prev_u = U[-1]
            c = o.mul(v.T, prev_u)                             # V_1^T U_{i-1}
            right = o.add(o.mul(a, prev_u), o.mul(u, c))       # A U_{i-1} + U_1 (.)
            U.append(np.hstack([u, right]))
            V.append(np.hstack([o.mul(self.p[i - 2].T, v), V[-1]]))  # P_{i-1}^T V_1
        for i in range(1, self.k + 1):
            self.p[i - 1] += o.mul(U[i - 1], V[i - 1].T)
        return U, V


class SkipIncrementalPowers:
    """Views of the skip-s model (``skip_levels``), Appendix A: the
    exponential rules up to P_s, then the skip rule for i = 2s, ..., k; all
    factors from the views before the update, the += statements last."""

    def __init__(self, a: np.ndarray, k: int, s: int):
        self.k, self.step = k, s
        self.hs = skip_levels(k, s)
        self.p = skip_powers(a, k, s)
        self.ops = _Ops()

    def apply(self, u: np.ndarray, v: np.ndarray):
        n = self.p[1].shape[0]
        u = np.asarray(u, dtype=np.float64).reshape(n, -1)
        v = np.asarray(v, dtype=np.float64).reshape(n, -1)
        o, s = self.ops, self.step
        U, V = {1: u}, {1: v}
        for h in levels(s)[:-1]:
            ph = self.p[h]
            c = o.mul(V[h].T, U[h])
            U[2 * h] = np.hstack([U[h], o.add(o.mul(ph, U[h]), o.mul(U[h], c))])
            V[2 * h] = np.hstack([o.mul(ph.T, V[h]), V[h]])
        ps = self.p[s]
        for i in range(2 * s, self.k + 1, s):
            c = o.mul(V[s].T, U[i - s])                              # V_s^T U_{i-s}
            right = o.add(o.mul(ps, U[i - s]), o.mul(U[s], c))       # P_s U_{i-s} + U_s (.)
            U[i] = np.hstack([U[s], right])
            V[i] = np.hstack([o.mul(self.p[i - s].T, V[s]), V[i - s]])  # P_{i-s}^T V_s
        for h in self.hs:
            self.p[h] += o.mul(U[h], V[h].T)
        return U, V


# --------------------------------------------------------------------------
# Adjoint (reverse mode) of a loss of P_k
# --------------------------------------------------------------------------
def adjoint_power_chain(a: np.ndarray, k: int, g: np.ndarray) -> np.ndarray:
    """dL/dA for L(P_k) with G = dL/dP_k, back through the squaring chain:
    P_{2h} = P_h P_h gives  Gbar_h = Gbar_{2h} P_h^T + P_h^T Gbar_{2h}."""
    p = reeval_powers(a, k)
    gb = np.asarray(g, dtype=np.float64).copy()
    for h in reversed(levels(k)[:-1]):
        gb = gb @ p[h].T + p[h].T @ gb
    return gb


def adjoint_power_sum(a: np.ndarray, k: int, g: np.ndarray) -> np.ndarray:
    """dL/dA = sum_{j=0}^{k-1} (A^T)^j G (A^T)^{k-1-j} (from d(A^k))."""
    a = np.asarray(a, dtype=np.float64)
    n = a.shape[0]
    pw = [np.eye(n)]
    for _ in range(k - 1):
        pw.append(pw[-1] @ a.T)
    out = np.zeros((n, n))
    for j in range(k):
        out += pw[j] @ g @ pw[k - 1 - j]
    return out
