"""Row-panel sharding of one maintained power program over W GPUs: the plan.

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
