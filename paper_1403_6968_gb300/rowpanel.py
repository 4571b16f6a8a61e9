"""Row-panel sharding of one maintained program over W GPUs: the plan
(power programs below; the general iteration and OLS in iteration_exchanges
and ols_exchanges).

Host logic only (no arithmetic of the method).  Each rank owns the rows
[r0, r1) of every view P_h and S'_h of the exponential model; the factor
arenas (U_h, V_h and the suffix sums W^_h of the sums views) are replicated.
One trigger (Appendix A, the level rule of Example 3.8) then needs exactly
two exchanges per level h = 1, 2, 4, .., k/2, both of n x r_h factor blocks:

* X_h = P_h U_h: every rank computes its row block from its rows of P_h
  and the replicated U_h, then an all-gather (row blocks in rank order)
  gives every rank the whole X_h;
* Y_h = P_h^T V_h: every rank computes the partial sum over its rows,
  (P_h rows)^T (V_h rows), then an all-reduce (sum) gives the whole Y_h.

Everything else is local: the core C_h = V_h^T U_h and the assembly of
U_2h = [U_h, X_h + U_h C_h], V_2h = [Y_h, V_h] run redundantly on every rank
from the replicated factors; the refreshes P_h += U_h V_h^T and
S'_h += U_h W^_h^T (the sums' delta in Krylov form, whose W^_h are suffix
block sums of V_h) touch only the owned rows.  The final level P_k needs no
products, so no exchange.  The paper's own cluster design stores both a row
and a column block of each view to avoid the reduction at twice the memory
(Section 5); on NVLink-connected GPUs the all-reduce of an n x r_h block is
cheaper than a second copy of every view.
"""
from __future__ import annotations


def panels(n: int, world: int):
    """Row ranges [(r0, r1)] of the W ranks: contiguous, sizes differing by
    at most one row, rank order."""
    if n < 1 or world < 1:
        raise ValueError("need n >= 1 and world >= 1")
    base, extra = divmod(n, world)
    out, r0 = [], 0
    for w in range(world):
        r1 = r0 + base + (1 if w < extra else 0)
        out.append((r0, r1))
        r0 = r1
    return out


def level_exchanges(n: int, k: int, r: int, world: int, elem_bytes: int = 4):
    """The exchanges of one rank-r update of A^k (exponential model, k a power
    of two): one entry per level h = 1, 2, .., k/2 with the factor width
    r_h = h r and the collectives' payloads (whole-result bytes)."""
    if k < 1 or k & (k - 1):
        raise ValueError("k must be a power of two")
    out = []
    h = 1
    while h < k:
        rh = h * r
        block = n * rh * elem_bytes
        out.append({"h": h, "r_h": rh,
                    "allgather": {"op": "all_gather", "what": "X_h = P_h U_h row blocks",
                                  "rows_per_rank": [b - a for a, b in panels(n, world)],
                                  "cols": rh, "bytes": block},
                    "allreduce": {"op": "all_reduce_sum", "what": "partial P_h^T V_h",
                                  "rows": n, "cols": rh, "bytes": block}})
        h *= 2
    return out


def update_exchange_bytes(n: int, k: int, r: int, world: int, elem_bytes: int = 4) -> int:
    """Total payload of the collectives of one update (all levels)."""
    return sum(e["allgather"]["bytes"] + e["allreduce"]["bytes"]
               for e in level_exchanges(n, k, r, world, elem_bytes))


def iteration_exchanges(n: int, p: int, k: int, r: int, world: int, elem_bytes: int = 4):
    """The exchanges of one rank-r update of A in the general iteration
    T_i = A T_{i-1} + B (linear model, Appendix B) with the rows of A and of
    every T_i sharded like the views above and the factors replicated.

    The Krylov blocks K_j = A' K_{j-1} (A' = A + U V^T; K_0 = U) are the only
    products with A: each rank computes its row block from its rows of A,
    the replicated K_{j-1} and (V^T K_{j-1}), then an all-gather gives every
    rank K_j (j = 1 .. k-1).  The right factors T_i^T V (i = 0 .. k-1, p x r
    each) are partial sums over the owned rows: one all-reduce of all k of
    them.  T_i += [K_0 .. K_{i-1}] [M_{i-1} .. M_0]^T and A += U V^T touch
    only the owned rows."""
    if n < 1 or p < 1 or k < 1 or r < 1:
        raise ValueError("need n, p, k, r >= 1")
    rows = [b - a for a, b in panels(n, world)]
    out = [{"op": "all_gather", "what": f"K_{j} row blocks", "rows_per_rank": rows, "cols": r,
            "bytes": n * r * elem_bytes} for j in range(1, k)]
    out.append({"op": "all_reduce_sum", "what": "partial T_i^T V, i = 0 .. k-1",
                "rows": k * r, "cols": p, "bytes": k * r * p * elem_bytes})
    return out


def ols_exchanges(n: int, p: int, kr: int, world: int, elem_bytes: int = 4):
    """The exchanges of one replacement of kr rows of X (Section 4.1, block
    Woodbury) with the rows of W, beta and X^T Y sharded and the update's
    data (the old and new rows of X, their rows of Y) replicated.

    G = W U (U = [X'_R^T, X_R^T], n x 2kr): row blocks from the owned rows of
    W, then an all-gather; the core C^-1 + U^T G, its inverse and
    Wu = -G M^-1 follow redundantly on every rank.  W += G Wu^T and
    X^T Y += (X'_R - X_R)^T Y_R touch only the owned rows.  The refresh of
    beta needs H = Wu^T (X^T Y)' (2kr x p), partial sums over the owned rows:
    one all-reduce; then beta += (G_1 - G_2) Y_R + G H on the owned rows."""
    if n < 1 or p < 1 or kr < 1:
        raise ValueError("need n, p, kr >= 1")
    rows = [b - a for a, b in panels(n, world)]
    return [{"op": "all_gather", "what": "G = W U row blocks", "rows_per_rank": rows,
             "cols": 2 * kr, "bytes": n * 2 * kr * elem_bytes},
            {"op": "all_reduce_sum", "what": "partial H = Wu^T (X^T Y)'", "rows": 2 * kr,
             "cols": p, "bytes": 2 * kr * p * elem_bytes}]
