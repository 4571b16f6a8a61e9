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
