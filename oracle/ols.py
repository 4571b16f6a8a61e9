"""Ordinary least squares -- FP64 oracle (test infrastructure).

beta* = (X^T X)^{-1} X^T Y with X m x n, Y m x p (Section 4.1, Example 3.1).
Z = X^T X and W = Z^{-1}.

* re-evaluation: Z, W = inv(Z), beta = W X^T Y (numpy.linalg.inv as the
  library inverse);
* Sherman-Morrison (Section 3.1): for E + u v^T,
      d(E^{-1}) = -E^{-1} u v^T E^{-1} / (1 + v^T E^{-1} u);
* two-step Sherman-Morrison (Example 3.3): for dX = u v^T,
      dZ = v (u^T X) + (X^T u + v (u^T u)) v^T = p1 q1^T + p2 q2^T,
  W <- W + d_{Z1}(W), then W <- W + d_{Z2}(W) using the once-updated W;
* block Woodbury (the k x k generalisation used for row blocks): for
  dZ = U diag(c) U^T and symmetric W,
      W' = W - G (diag(1/c) + U^T G)^{-1} G^T,   G = W U.
  Replacing rows R of X by X'_R gives U = [X'_R^T, X_R^T], c = (+1..., -1...),
  since dZ = X'_R^T X'_R - X_R^T X_R.  The 2k x 2k core is solved by LU with
  partial pivoting (numpy.linalg.solve); it is indefinite, so not Cholesky.
* residual correction of the maintained W (the paper maintains W = Z^{-1},
  Section 4.1, and leaves its rounding drift open; the correction is the
  Newton-Schulz iteration for a matrix inverse, Schulz 1933): one step
      W <- W + W (I - Z W),
  whose residual is the square of the old one, I - Z W' = (I - Z W)^2; and
  the matching refinement of beta = W X^T Y:
      beta <- beta + W (X^T Y - Z beta).
"""
from __future__ import annotations

import numpy as np


def reeval(x, y):
    """dict(Z, W, XtY, beta) from scratch."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    z = x.T @ x
    w = np.linalg.inv(z)
    xty = x.T @ y
    return {"Z": z, "W": w, "XtY": xty, "beta": w @ xty}


def sherman_morrison(e_inv, u, v):
    """d(E^{-1}) for the rank-1 change u v^T of E."""
    e_inv = np.asarray(e_inv, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64).reshape(-1)
    v = np.asarray(v, dtype=np.float64).reshape(-1)
    left = e_inv @ u
    right = v @ e_inv
    den = 1.0 + v @ left
    return -np.outer(left, right) / den


def sm_two_step(w, x, i: int, d):
    """W after the row change X[i] += d (dX = e_i d^T) by Example 3.3."""
    x = np.asarray(x, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64).reshape(-1)
    xi = x[i, :]                  # u^T X for u = e_i; also X^T u
    p1, q1 = d, xi
    p2, q2 = xi + d, d            # X^T u + v (u^T u), u^T u = 1
    w1 = w + sherman_morrison(w, p1, q1)
    return w1 + sherman_morrison(w1, p2, q2)


def woodbury(w, u, c):
    """(Z + U diag(c) U^T)^{-1} from W = Z^{-1} (W symmetric)."""
    w = np.asarray(w, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    g = w @ u
    m = np.diag(1.0 / c) + u.T @ g
    return w - g @ np.linalg.solve(m, g.T)


def newton_schulz_step(w, z):
    """One Newton-Schulz step toward Z^{-1}: W + W (I - Z W)."""
    w = np.asarray(w, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    return w + w @ (np.eye(w.shape[0]) - z @ w)


def refine_beta(w, beta, xty, z):
    """One refinement step of beta for Z beta = X^T Y with the approximate
    inverse W: beta + W (X^T Y - Z beta)."""
    w = np.asarray(w, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    return beta + w @ (np.asarray(xty, dtype=np.float64) - np.asarray(z, dtype=np.float64) @ beta)


class IncrementalOLS:
    """X, X^T Y, W and beta under row-block replacements (Y unchanged)."""

    def __init__(self, x, y):
        self.x = np.asarray(x, dtype=np.float64).copy()
        self.y = np.asarray(y, dtype=np.float64).copy()
        r = reeval(self.x, self.y)
        self.z, self.w, self.xty, self.beta = r["Z"], r["W"], r["XtY"], r["beta"]

    def replace_rows(self, rows, new_rows, method: str = "woodbury"):
        rows = np.asarray(rows, dtype=np.int64)
        new = np.asarray(new_rows, dtype=np.float64).reshape(len(rows), -1)
        old = self.x[rows, :].copy()
        if method == "woodbury":
            k = len(rows)
            u = np.hstack([new.T, old.T])
            c = np.concatenate([np.ones(k), -np.ones(k)])
            self.w = woodbury(self.w, u, c)
            self.x[rows, :] = new
        elif method == "sm":
            for j, i in enumerate(rows):
                d = new[j] - self.x[i]
                self.w = sm_two_step(self.w, self.x, int(i), d)
                self.x[i, :] = new[j]
        else:
            raise ValueError(method)
        self.z += new.T @ new - old.T @ old
        self.xty += (new - old).T @ self.y[rows, :]
        self.beta = self.w @ self.xty
