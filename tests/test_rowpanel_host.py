"""Row-panel sharding of a power program (A^k and S'_h) on CPU gloo ranks.

Each rank owns a row panel of every view (paper_1403_6968_gb300.rowpanel);
the factors are replicated.  One update runs the exponential-model level rule
(Appendix A) with exactly the plan's two collectives per level -- an
all-gather of the X_h = P_h U_h row blocks and an all-reduce of the partial
P_h^T V_h -- and refreshes only the owned rows (sums views by the Krylov form
S'_h += U_h W^_h^T, W^_h the suffix block sums of V_h).  After several updates
every rank's panels must equal the FP64 oracle's re-evaluation on the updated
A (brute force), and the bytes exchanged must be the plan's.  The per-rank
arithmetic here is numpy FP64 (test infrastructure): this checks the sharded
design and its exchange schedule; no multi-GPU path is built.
"""
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, outdir, n, k, r, nupd):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import linview_inputs as li
    from oracle import powers as op
    from paper_1403_6968_gb300 import rowpanel
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    pan = rowpanel.panels(n, ws)
    r0, r1 = pan[rank]
    maxrows = max(b - a for a, b in pan)
    a = li.power_matrix(n, seed=7)
    full_p = op.reeval_powers(a, k)
    full_s = op.reeval_sums(a, k, full_p)
    levels = op.levels(k)                      # 1, 2, 4, .., k
    P = {h: full_p[h][r0:r1].copy() for h in levels}
    S = {h: full_s[h][r0:r1].copy() for h in levels if h > 1}
    acur = a.copy()
    sent = []

    def all_gather_rows(x_loc):
        buf = np.zeros((maxrows, x_loc.shape[1]))
        buf[:x_loc.shape[0]] = x_loc
        parts = [torch.zeros(maxrows, x_loc.shape[1], dtype=torch.float64) for _ in range(ws)]
        dist.all_gather(parts, torch.from_numpy(buf))
        return np.concatenate([parts[w].numpy()[:b - e] for w, (e, b) in enumerate(pan)])

    def all_reduce_sum(y_part):
        t = torch.from_numpy(y_part.copy())
        dist.all_reduce(t)
        return t.numpy()

    for u, v in li.lowrank_update_stream(n, r, nupd, seed=8):
        acur += u @ v.T
        uh, vh = u.copy(), v.copy()
        fac = {}
        for h in levels[:-1]:
            x = all_gather_rows(P[h] @ uh)                      # X_h = P_h U_h
            y = all_reduce_sum(P[h].T @ vh[r0:r1])              # Y_h = P_h^T V_h
            sent.append({"h": h, "r_h": uh.shape[1], "allgather": x.nbytes, "allreduce": y.nbytes})
            c = vh.T @ uh                                       # replicated core
            fac[h] = (uh, vh)
            uh, vh = np.hstack([uh, x + uh @ c]), np.hstack([y, vh])
        fac[k] = (uh, vh)
        for h in levels:                                        # owned rows only
            uh, vh = fac[h]
            P[h] += uh[r0:r1] @ vh.T
            if h > 1:
                nb = vh.shape[1] // r                           # W^_h: suffix block sums of V_h
                what = np.zeros_like(vh)
                acc = np.zeros((n, r))
                for b in range(nb - 1, -1, -1):
                    acc = acc + vh[:, b * r:(b + 1) * r]
                    what[:, b * r:(b + 1) * r] = acc
                S[h] += uh[r0:r1] @ what.T
    ref_p = op.reeval_powers(acur, k)
    ref_s = op.reeval_sums(acur, k, ref_p)
    err = max([float(np.linalg.norm(P[h] - ref_p[h][r0:r1]) / np.linalg.norm(ref_p[h][r0:r1]))
               for h in levels] +
              [float(np.linalg.norm(S[h] - ref_s[h][r0:r1]) / np.linalg.norm(ref_s[h][r0:r1]))
               for h in levels if h > 1])
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
        json.dump({"rank": rank, "rows": [r0, r1], "err": err, "sent": sent}, f)
    dist.destroy_process_group()


@pytest.mark.parametrize("ws,n", [(2, 37), (3, 64)])
def test_sharded_views_equal_the_oracle(tmp_path, ws, n):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    from paper_1403_6968_gb300 import rowpanel
    k, r, nupd = 8, 2, 3
    mp.spawn(_rank_main, args=(ws, _free_port(), str(tmp_path), n, k, r, nupd), nprocs=ws,
             join=True)
    got = [json.load(open(tmp_path / f"rank{w}.json")) for w in range(ws)]
    assert [tuple(g["rows"]) for g in got] == rowpanel.panels(n, ws)
    plan = rowpanel.level_exchanges(n, k, r, ws, elem_bytes=8)
    for g in got:
        assert g["err"] <= 1e-11, g
        # every update made exactly the plan's exchanges, level by level
        assert len(g["sent"]) == nupd * len(plan)
        for i, s in enumerate(g["sent"]):
            e = plan[i % len(plan)]
            assert (s["h"], s["r_h"]) == (e["h"], e["r_h"])
            assert s["allgather"] == e["allgather"]["bytes"]
            assert s["allreduce"] == e["allreduce"]["bytes"]


def test_panels_and_plan():
    from paper_1403_6968_gb300 import rowpanel
    assert rowpanel.panels(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert rowpanel.panels(8192, 8)[-1] == (7168, 8192)
    with pytest.raises(ValueError):
        rowpanel.panels(0, 2)
    plan = rowpanel.level_exchanges(8192, 16, 1, 8)
    assert [e["r_h"] for e in plan] == [1, 2, 4, 8]
    # n = 8192, rank 1, A^16: 2 x 8192 x 15 x 4 bytes per update
    assert rowpanel.update_exchange_bytes(8192, 16, 1, 8) == 2 * 8192 * 15 * 4
    with pytest.raises(ValueError):
        rowpanel.level_exchanges(100, 12, 1, 2)


def _gloo(rank, ws, port):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    return dist


def _collectives(dist, pan, ws, sent):
    import torch
    maxrows = max(b - a for a, b in pan)

    def all_gather_rows(x_loc):
        buf = np.zeros((maxrows, x_loc.shape[1]))
        buf[:x_loc.shape[0]] = x_loc
        parts = [torch.zeros(maxrows, x_loc.shape[1], dtype=torch.float64) for _ in range(ws)]
        dist.all_gather(parts, torch.from_numpy(buf))
        out = np.concatenate([parts[w].numpy()[:b - e] for w, (e, b) in enumerate(pan)])
        sent.append(("all_gather", out.nbytes))
        return out

    def all_reduce_sum(y_part):
        t = torch.from_numpy(np.ascontiguousarray(y_part))
        dist.all_reduce(t)
        sent.append(("all_reduce_sum", t.numpy().nbytes))
        return t.numpy()

    return all_gather_rows, all_reduce_sum


def _rank_iteration(rank, ws, port, outdir, n, p, k, r, nupd):
    """Linear model of the general iteration with the rows of A and every T_i
    owned: K_j from the owned rows of A and an all-gather, the right factors
    T_i^T V from one all-reduce, the refreshes on the owned rows."""
    dist = _gloo(rank, ws, port)
    import linview_inputs as li
    from oracle import iteration as oi
    from paper_1403_6968_gb300 import rowpanel
    pan = rowpanel.panels(n, ws)
    r0, r1 = pan[rank]
    sent = []
    gather, reduce = _collectives(dist, pan, ws, sent)
    a, b, t0 = li.iteration_inputs(n, p, seed=11)
    full = oi.reeval(a, b, t0, k)
    T = {i: full[i][r0:r1].copy() for i in range(k + 1)}
    A = a[r0:r1].copy()
    acur = a.copy()
    for u, v in li.lowrank_update_stream(n, r, nupd, seed=12, sigma=0.2):
        acur += u @ v.T
        # M_i = T_i^T v (old T_i), i = 0 .. k-1: one all-reduce of all of them
        M = reduce(np.stack([T[i].T @ v[r0:r1] for i in range(k)]))
        K = [u]
        for j in range(1, k):                      # K_j = (A + u v^T) K_{j-1}
            K.append(gather(A @ K[j - 1] + u[r0:r1] @ (v.T @ K[j - 1])))
        A += u[r0:r1] @ v.T
        for i in range(1, k + 1):                  # T_i += sum_a K_a M_{i-1-a}^T
            T[i] += sum(K[q][r0:r1] @ M[i - 1 - q].T for q in range(i))
    ref = oi.reeval(acur, b, t0, k)
    err = max(float(np.linalg.norm(T[i] - ref[i][r0:r1]) / np.linalg.norm(ref[i][r0:r1]))
              for i in range(1, k + 1))
    err = max(err, float(np.linalg.norm(A - acur[r0:r1]) / np.linalg.norm(acur[r0:r1])))
    with open(os.path.join(outdir, f"it{rank}.json"), "w") as f:
        json.dump({"err": err, "sent": sent}, f)
    dist.destroy_process_group()


def _rank_ols(rank, ws, port, outdir, m, n, p, kr, nupd):
    """Block Woodbury with the rows of W, beta and X^T Y owned: G from the
    owned rows of W and an all-gather, H = Wu^T (X^T Y)' from one all-reduce,
    every refresh on the owned rows (X and the replaced rows replicated)."""
    dist = _gloo(rank, ws, port)
    import linview_inputs as li
    from oracle import ols as oo
    from paper_1403_6968_gb300 import rowpanel
    pan = rowpanel.panels(n, ws)
    r0, r1 = pan[rank]
    sent = []
    gather, reduce = _collectives(dist, pan, ws, sent)
    x, y, _ = li.ols_inputs(m, n, p, seed=13)
    ref = oo.reeval(x, y)
    W, beta, xty = ref["W"][r0:r1].copy(), ref["beta"][r0:r1].copy(), ref["XtY"][r0:r1].copy()
    for rows, new in li.ols_row_replacements(m, n, kr, nupd, seed=14, cols_seed=13):
        old = x[rows].copy()
        U = np.hstack([new.T, old.T])                          # n x 2kr
        c = np.concatenate([np.ones(kr), -np.ones(kr)])
        G = gather(W @ U)
        wu = -G @ np.linalg.inv(np.diag(1.0 / c) + U.T @ G)
        W += G[r0:r1] @ wu.T
        yr = y[rows]
        xty += (new - old).T[r0:r1] @ yr
        H = reduce(wu[r0:r1].T @ xty)                          # 2kr x p
        beta += (G[r0:r1, :kr] - G[r0:r1, kr:]) @ yr + G[r0:r1] @ H
        x[rows] = new
    fresh = oo.reeval(x, y)
    err = max(float(np.linalg.norm(W - fresh["W"][r0:r1]) / np.linalg.norm(fresh["W"][r0:r1])),
              float(np.linalg.norm(beta - fresh["beta"][r0:r1]) /
                    np.linalg.norm(fresh["beta"][r0:r1])))
    with open(os.path.join(outdir, f"ols{rank}.json"), "w") as f:
        json.dump({"err": err, "sent": sent}, f)
    dist.destroy_process_group()


@pytest.mark.parametrize("ws,n", [(2, 29), (3, 48)])
def test_sharded_iteration_equals_the_oracle(tmp_path, ws, n):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    from paper_1403_6968_gb300 import rowpanel
    p, k, r, nupd = 3, 8, 2, 3
    mp.spawn(_rank_iteration, args=(ws, _free_port(), str(tmp_path), n, p, k, r, nupd),
             nprocs=ws, join=True)
    plan = rowpanel.iteration_exchanges(n, p, k, r, ws, elem_bytes=8)
    # the all-reduce of the right factors comes first in an update, then the gathers
    want = [(plan[-1]["op"], plan[-1]["bytes"])] + [(e["op"], e["bytes"]) for e in plan[:-1]]
    for w in range(ws):
        got = json.load(open(tmp_path / f"it{w}.json"))
        assert got["err"] <= 1e-11, got["err"]
        assert [tuple(s) for s in got["sent"]] == want * nupd


@pytest.mark.parametrize("ws,kr", [(2, 1), (3, 4)])
def test_sharded_ols_equals_the_oracle(tmp_path, ws, kr):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    from paper_1403_6968_gb300 import rowpanel
    m, n, p, nupd = 200, 20, 3, 3
    mp.spawn(_rank_ols, args=(ws, _free_port(), str(tmp_path), m, n, p, kr, nupd),
             nprocs=ws, join=True)
    plan = rowpanel.ols_exchanges(n, p, kr, ws, elem_bytes=8)
    for w in range(ws):
        got = json.load(open(tmp_path / f"ols{w}.json"))
        assert got["err"] <= 1e-9, got["err"]
        assert [tuple(s) for s in got["sent"]] == [(e["op"], e["bytes"]) for e in plan] * nupd


def test_iteration_and_ols_plans():
    from paper_1403_6968_gb300 import rowpanel
    it = rowpanel.iteration_exchanges(8192, 64, 16, 2, 8)
    assert [e["op"] for e in it] == ["all_gather"] * 15 + ["all_reduce_sum"]
    # n = 8192, p = 64, k = 16, rank 2: 15 x 64 KB gathers + one 8 KB reduction
    assert sum(e["bytes"] for e in it) == 15 * 8192 * 2 * 4 + 16 * 2 * 64 * 4
    ols = rowpanel.ols_exchanges(4096, 16, 16, 8)
    assert [e["bytes"] for e in ols] == [4096 * 32 * 4, 32 * 16 * 4]
    with pytest.raises(ValueError):
        rowpanel.ols_exchanges(0, 1, 1, 2)
