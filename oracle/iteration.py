"""General form T_{i+1} = A T_i + B -- FP64 oracle (test infrastructure).

Section 4.3 and Appendix B of the paper.  A is n x n, B and T_i are n x p.

* re-evaluation, linear model (Table 1): T_1 = A T_0 + B, T_i = A T_{i-1} + B;
* incremental, linear model (Appendix B) for dA = U V^T: U_1 = U, V_1 = T_0^T V,
      U_i = [U, A U_{i-1} + U (V^T U_{i-1})],   V_i = [T_{i-1}^T V, V_{i-1}],
  dT_i = U_i V_i^T (Appendix B prints "U_i V_i"; the transpose is implied by
  the factored form of Section 3.2), with A and T_{i-1} taken before the update
  and every += applied last;
* hybrid, linear model (Appendix B): dT_1 = dA T_0,
      dT_i = U V^T T_{i-1} + A dT_{i-1} + U V^T dT_{i-1}   (dense n x p deltas);
* exponential model (Section 3.3, Appendix B) for k a power of two: views
  T_h, h = 1, 2, 4, ..., k, with the auxiliary views P_h = A^h and
  S_h = I + A + ... + A^{h-1} (h = 1, 2, ..., k/2):
      T_1 = A T_0 + B,  T_2h = P_h T_h + S_h B,
      P_2h = P_h P_h,   S_2h = S_h + P_h S_h   (S_1 = I);
  incremental for dA = u v^T, with dP_h = Q_h R_h^T, dS_h = Z_h W_h^T and
  dT_h = U_h V_h^T from the old views (Appendix B, exponential model):
      U_1 = u, V_1 = T_0^T v;
      U_2h = [Q_h, P_h U_h + Q_h (R_h^T U_h), Z_h],
      V_2h = [T_h^T R_h, V_h, B^T W_h];
  Q_h, R_h as in Appendix A (powers), and Z_h, W_h from
  S_2h = S_h + P_h S_h:  dS_2h = dS_h + dP_h S_h + P_h dS_h + dP_h dS_h, i.e.
      Z_2h = [Q_h, Z_h + P_h Z_h + Q_h (R_h^T Z_h)],  W_2h = [S_h^T R_h, W_h],
  with Z_1, W_1 empty (dS_1 = 0).  (The paper prints "dW_{i/2}" for W_{i/2}
  and gives the width of U_i as 2i - 1, an upper bound: with dS_1 = 0 the
  widths are 1, 2, 5, 12, 27 for i = 1, 2, 4, 8, 16 at rank 1.)
* skip-s model (Section 3.3, Appendix B), s a power of two, k a multiple of s,
  k >= 2s: T_1, T_2, .., T_s by the exponential model, then
      T_i = P_s T_{i-s} + S_s B   (i = 2s, 3s, .., k),
  and incrementally, from the old views,
      U_i = [Q_s, P_s U_{i-s} + Q_s (R_s^T U_{i-s}), Z_s],
      V_i = [T_{i-s}^T R_s, V_{i-s}, B^T W_s];
* adjoint of L = ||T_k||_F^2: G_k = 2 T_k, G_i = A^T G_{i+1},
      dL/dB = sum_{i=1..k} G_i,   dL/dA = sum_{i=1..k} G_i T_{i-1}^T,
      dL/dT_0 = A^T G_1.
"""
from __future__ import annotations

import numpy as np


def reeval(a, b, t0, k: int) -> list:
    """[T_0, T_1, ..., T_k] by the linear model."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    t = [np.asarray(t0, dtype=np.float64).copy()]
    for _ in range(k):
        t.append(a @ t[-1] + b)
    return t


def loss(a, b, t0, k: int) -> float:
    """L = ||T_k||_F^2."""
    tk = reeval(a, b, t0, k)[-1]
    return float(np.sum(tk * tk))


class IncrementalIteration:
    """Views T_1..T_k maintained under dA = U V^T (Appendix B, linear model)."""

    def __init__(self, a, b, t0, k: int):
        self.k = k
        self.a = np.asarray(a, dtype=np.float64).copy()
        self.b = np.asarray(b, dtype=np.float64).copy()
        self.t = reeval(self.a, self.b, t0, k)  # t[0] = T_0 (input), t[i] = T_i

    def apply(self, u, v):
        n = self.a.shape[0]
        u = np.asarray(u, dtype=np.float64).reshape(n, -1)
        v = np.asarray(v, dtype=np.float64).reshape(n, -1)
        U = {1: u}
        V = {1: self.t[0].T @ v}
        for i in range(2, self.k + 1):
            right = self.a @ U[i - 1] + u @ (v.T @ U[i - 1])
            U[i] = np.hstack([u, right])
            V[i] = np.hstack([self.t[i - 1].T @ v, V[i - 1]])
        self.a += u @ v.T
        for i in range(1, self.k + 1):
            self.t[i] += U[i] @ V[i].T
        return U, V


    def apply_b(self, ub, vb):
        """dB = U_b V_b^T (U_b n x r_b, V_b p x r_b) with A unchanged: dT_i =
        A dT_{i-1} + dB, dT_0 = 0, i.e. dT_i = U_i V_i^T with
        U_i = [U_b, A U_{i-1}], V_i = [V_b, V_{i-1}] (derived from the
        recurrence; the paper omits changes in B, Section 4.3.2)."""
        n, p = self.b.shape
        ub = np.asarray(ub, dtype=np.float64).reshape(n, -1)
        vb = np.asarray(vb, dtype=np.float64).reshape(p, -1)
        U, V = {1: ub}, {1: vb}
        for i in range(2, self.k + 1):
            U[i] = np.hstack([ub, self.a @ U[i - 1]])
            V[i] = np.hstack([vb, V[i - 1]])
        self.b += ub @ vb.T
        for i in range(1, self.k + 1):
            self.t[i] += U[i] @ V[i].T
        return U, V


class HybridIteration:
    """Views T_1..T_k maintained with dense deltas (Appendix B, hybrid linear)."""

    def __init__(self, a, b, t0, k: int):
        self.k = k
        self.a = np.asarray(a, dtype=np.float64).copy()
        self.b = np.asarray(b, dtype=np.float64).copy()
        self.t = reeval(self.a, self.b, t0, k)

    def apply(self, u, v):
        n = self.a.shape[0]
        u = np.asarray(u, dtype=np.float64).reshape(n, -1)
        v = np.asarray(v, dtype=np.float64).reshape(n, -1)
        d = [None, u @ (v.T @ self.t[0])]
        for i in range(2, self.k + 1):
            d.append(u @ (v.T @ self.t[i - 1]) + self.a @ d[i - 1] + u @ (v.T @ d[i - 1]))
        self.a += u @ v.T
        for i in range(1, self.k + 1):
            self.t[i] += d[i]


def adjoint(a, b, t0, k: int):
    """(dL/dA, dL/dB, dL/dT0) for L = ||T_k||_F^2 (reverse mode over the k steps)."""
    a = np.asarray(a, dtype=np.float64)
    t = reeval(a, b, t0, k)
    g = {k: 2.0 * t[k]}
    for i in range(k - 1, 0, -1):
        g[i] = a.T @ g[i + 1]
    da = np.zeros_like(a)
    db = np.zeros_like(t[0])
    for i in range(1, k + 1):
        da += g[i] @ t[i - 1].T
        db += g[i]
    dt0 = a.T @ g[1]
    return da, db, dt0


def exp_reeval(a, b, t0, k: int):
    """Exponential model: ({h: T_h} for h = 1, 2, 4, ..., k, {h: P_h},
    {h: S_h}) with P_h, S_h for h = 1, 2, ..., k/2 (k a power of two)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = a.shape[0]
    P, S = {1: a.copy()}, {1: np.eye(n)}
    h = 1
    while 2 * h <= k // 2:
        P[2 * h] = P[h] @ P[h]
        S[2 * h] = S[h] + P[h] @ S[h]
        h *= 2
    T = {1: a @ np.asarray(t0, dtype=np.float64) + b}
    h = 1
    while 2 * h <= k:
        T[2 * h] = P[h] @ T[h] + S[h] @ b
        h *= 2
    return T, P, S


class ExpIncrementalIteration:
    """Views T_1, T_2, T_4, ..., T_k (with P_h, S_h, h <= k/2) maintained
    under dA = u v^T (Appendix B, exponential model)."""

    def __init__(self, a, b, t0, k: int):
        if k < 1 or k & (k - 1):
            raise ValueError("k must be a power of two")
        self.k = k
        self.a = np.asarray(a, dtype=np.float64).copy()
        self.b = np.asarray(b, dtype=np.float64).copy()
        self.t0 = np.asarray(t0, dtype=np.float64).copy()
        self.t, self.p, self.s = exp_reeval(self.a, self.b, self.t0, k)

    def apply(self, u, v):
        """Returns the factors {h: U_h}, {h: V_h} of dT_h."""
        n = self.a.shape[0]
        u = np.asarray(u, dtype=np.float64).reshape(n, -1)
        v = np.asarray(v, dtype=np.float64).reshape(n, -1)
        Q, R = {1: u}, {1: v}
        Z, W = {1: np.zeros((n, 0))}, {1: np.zeros((n, 0))}
        U, V = {1: u}, {1: self.t0.T @ v}
        h = 1
        while 2 * h <= self.k:
            P, S, T = self.p[h], self.s[h], self.t[h]
            U[2 * h] = np.hstack([Q[h], P @ U[h] + Q[h] @ (R[h].T @ U[h]), Z[h]])
            V[2 * h] = np.hstack([T.T @ R[h], V[h], self.b.T @ W[h]])
            if 2 * h <= self.k // 2:
                Q[2 * h] = np.hstack([Q[h], P @ Q[h] + Q[h] @ (R[h].T @ Q[h])])
                R[2 * h] = np.hstack([P.T @ R[h], R[h]])
                Z[2 * h] = np.hstack([Q[h], Z[h] + P @ Z[h] + Q[h] @ (R[h].T @ Z[h])])
                W[2 * h] = np.hstack([S.T @ R[h], W[h]])
            h *= 2
        self.a += u @ v.T
        for h in self.p:
            self.p[h] += Q[h] @ R[h].T
            self.s[h] += Z[h] @ W[h].T
        for h in self.t:
            self.t[h] += U[h] @ V[h].T
        return U, V

    def apply_b(self, ub, vb):
        """dB = U_b V_b^T with A unchanged (derived from the recurrence; the
        paper omits changes in B, Section 4.3.2): P_h and S_h are unchanged,
        dT_1 = dB and dT_2h = P_h dT_h + S_h dB, i.e.
        U_1 = U_b, V_1 = V_b, U_2h = [P_h U_h, S_h U_b], V_2h = [V_h, V_b]."""
        n, p = self.b.shape
        ub = np.asarray(ub, dtype=np.float64).reshape(n, -1)
        vb = np.asarray(vb, dtype=np.float64).reshape(p, -1)
        U, V = {1: ub}, {1: vb}
        h = 1
        while 2 * h <= self.k:
            U[2 * h] = np.hstack([self.p[h] @ U[h], self.s[h] @ ub])
            V[2 * h] = np.hstack([V[h], vb])
            h *= 2
        self.b += ub @ vb.T
        for h in self.t:
            self.t[h] += U[h] @ V[h].T
        return U, V


def skip_reeval(a, b, t0, k: int, s: int):
    """Skip-s model: ({i: T_i} for i = 1, 2, 4, .., s, 2s, 3s, .., k,
    {h: P_h}, {h: S_h}) with P_h, S_h for h = 1, 2, .., s."""
    if s < 1 or s & (s - 1) or k % s or k < 2 * s:
        raise ValueError("s a power of two, k a multiple of s, k >= 2s")
    T, P, S = exp_reeval(a, b, t0, s)
    h = max(P)
    if 2 * h == s:  # exp_reeval stops at s/2: P_s, S_s by one more squaring
        P[s] = P[h] @ P[h]
        S[s] = S[h] + P[h] @ S[h]
    b = np.asarray(b, dtype=np.float64)
    for i in range(2 * s, k + 1, s):
        T[i] = P[s] @ T[i - s] + S[s] @ b
    return T, P, S


class SkipIncrementalIteration:
    """Views T_1, T_2, .., T_s (powers of two), T_2s, .., T_k with P_h, S_h
    (h = 1, 2, .., s) maintained under dA = u v^T (Appendix B, skip model)."""

    def __init__(self, a, b, t0, k: int, s: int):
        self.k, self.s = k, s
        self.a = np.asarray(a, dtype=np.float64).copy()
        self.b = np.asarray(b, dtype=np.float64).copy()
        self.t0 = np.asarray(t0, dtype=np.float64).copy()
        self.t, self.p, self.sv = skip_reeval(self.a, self.b, self.t0, k, s)

    def apply(self, u, v):
        """Returns the factors {i: U_i}, {i: V_i} of dT_i."""
        n = self.a.shape[0]
        u = np.asarray(u, dtype=np.float64).reshape(n, -1)
        v = np.asarray(v, dtype=np.float64).reshape(n, -1)
        Q, R = {1: u}, {1: v}
        Z, W = {1: np.zeros((n, 0))}, {1: np.zeros((n, 0))}
        U, V = {1: u}, {1: self.t0.T @ v}
        h = 1
        while 2 * h <= self.s:  # exponential part: factors up to h = s
            P, S, T = self.p[h], self.sv[h], self.t[h]
            U[2 * h] = np.hstack([Q[h], P @ U[h] + Q[h] @ (R[h].T @ U[h]), Z[h]])
            V[2 * h] = np.hstack([T.T @ R[h], V[h], self.b.T @ W[h]])
            Q[2 * h] = np.hstack([Q[h], P @ Q[h] + Q[h] @ (R[h].T @ Q[h])])
            R[2 * h] = np.hstack([P.T @ R[h], R[h]])
            Z[2 * h] = np.hstack([Q[h], Z[h] + P @ Z[h] + Q[h] @ (R[h].T @ Z[h])])
            W[2 * h] = np.hstack([S.T @ R[h], W[h]])
            h *= 2
        s = self.s
        Ps = self.p[s]
        for i in range(2 * s, self.k + 1, s):
            U[i] = np.hstack([Q[s], Ps @ U[i - s] + Q[s] @ (R[s].T @ U[i - s]), Z[s]])
            V[i] = np.hstack([self.t[i - s].T @ R[s], V[i - s], self.b.T @ W[s]])
        self.a += u @ v.T
        for h in self.p:
            self.p[h] += Q[h] @ R[h].T
            self.sv[h] += Z[h] @ W[h].T
        for i in self.t:
            self.t[i] += U[i] @ V[i].T
        return U, V

    def apply_b(self, ub, vb):
        """dB = U_b V_b^T with A unchanged (derived from the recurrences):
        dT_1 = dB, dT_2h = P_h dT_h + S_h dB (h < s), dT_i = P_s dT_{i-s} + S_s dB
        (i > s), i.e. U_i = [P U_j, S U_b], V_i = [V_j, V_b]."""
        n, p = self.b.shape
        ub = np.asarray(ub, dtype=np.float64).reshape(n, -1)
        vb = np.asarray(vb, dtype=np.float64).reshape(p, -1)
        U, V = {1: ub}, {1: vb}
        h = 1
        while 2 * h <= self.s:
            U[2 * h] = np.hstack([self.p[h] @ U[h], self.sv[h] @ ub])
            V[2 * h] = np.hstack([V[h], vb])
            h *= 2
        s = self.s
        for i in range(2 * s, self.k + 1, s):
            U[i] = np.hstack([self.p[s] @ U[i - s], self.sv[s] @ ub])
            V[i] = np.hstack([V[i - s], vb])
        self.b += ub @ vb.T
        for i in self.t:
            self.t[i] += U[i] @ V[i].T
        return U, V

