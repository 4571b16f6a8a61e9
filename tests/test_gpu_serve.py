"""GPU: the serving loop (linview_server_*) -- continuous batching of factored
updates over many resident A^k views.

* alone vs mix: every view refreshed by the server from an open-loop trace
  (requests coalesced while their view is busy, several views refreshing at
  once) equals the same view refreshed alone, one request at a time, and the
  FP64 oracle's re-evaluation on the updated A, within the FP32 bound 1e-4;
* admission by memory: a view that does not fit the budget waits with its
  requests queued and is admitted when a removed view frees memory;
* the device-bytes estimate used for admission equals what a program holds.

The server runs a scheduler thread inside the library, so each server test
body runs in a child process with a time limit: a stuck scheduler fails its
own test instead of holding the whole session.
"""
import os
import subprocess
import sys
import time

import numpy as np
import pytest

import linview_inputs as li
from oracle import powers as op
from oracle.metrics import rel_frob

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4
K = 16
L = 4  # view id of A^16


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _pkg():
    import paper_1403_6968_gb300 as P
    return P


def _final_a(a0, reqs):
    a = a0.astype(np.float64).copy()
    for u, v in reqs:
        a += u.astype(np.float64) @ v.astype(np.float64).T
    return a


def _body_serve_alone_vs_mix():
    P = _pkg()
    sizes = [256, 512, 384, 1000]
    a0 = [li.power_matrix(n, seed=10 + i, dtype=np.float32) for i, n in enumerate(sizes)]
    count = 80
    # ~20 us between arrivals: most requests find their view busy
    t_s, views, ranks, factors, offsets = li.serving_trace(sizes, count, rate=5e4, seed=3)
    srv = P.Server(max_inflight=3, r_cap=8)
    try:
        ids = [srv.add_view(a, K) for a in a0]
        assert ids == list(range(len(sizes)))
        assert all(srv.view_state(i) == "resident" for i in ids)
        srv.replay(t_s, views, ranks, factors, offsets)
        srv.drain(timeout_s=120)
        recs = srv.poll()
        st = srv.stats()
        assert len(recs) == count and st["completed"] == count and st["failed"] == 0
        assert sorted(r["ticket"] for r in recs) == list(range(1, count + 1))
        for r in recs:
            assert r["status"] == 0
            assert r["arrival_s"] <= r["start_s"] + 1e-9 <= r["done_s"] + 1e-9
            assert 1 <= r["batch_rank"] <= 8 and r["rank"] <= r["batch_rank"]
        # the mix really coalesced and overlapped
        assert max(r["batch_size"] for r in recs) > 1
        assert st["refreshes"] < count
        assert st["max_inflight_seen"] >= 2
        mixed = {i: srv.program(i).read_view(L).cpu().numpy().astype(np.float64) for i in ids}
        mixed_a = {i: srv.program(i).read_view(0).cpu().numpy().astype(np.float64) for i in ids}
    finally:
        srv.close()
    # the same requests, each view alone, one request at a time, in ticket order
    for i, n in enumerate(sizes):
        reqs = [li.trace_factors(sizes, views, ranks, factors, offsets, j)
                for j in range(count) if views[j] == i]
        prog = P.Program("power", [a0[i]], k=K, r_max=8)
        for u, v in reqs:
            prog.apply_delta(u, v)
        alone = prog.read_view(L).cpu().numpy().astype(np.float64)
        prog.close()
        af = _final_a(a0[i], reqs)
        ref = op.reeval_powers(af, K)[K]
        assert rel_frob(mixed_a[i], af) <= TOL
        assert rel_frob(mixed[i], alone) <= TOL, (i, n)
        assert rel_frob(mixed[i], ref) <= TOL, (i, n)
        assert rel_frob(alone, ref) <= TOL, (i, n)


def _body_serve_alone_vs_mix_full_sizes():
    """The serving workload's own view sizes (n in {1024, 2048, 4096, 8192},
    A^16, FP32): the mixed, coalesced result of every view equals the view
    refreshed alone (whole A^16 view) and the FP64 oracle on 16 sampled rows,
    computed row by row on A0 + sum_j U_j V_j^T."""
    P = _pkg()
    sizes = [4096, 8192, 1024, 2048]
    a0 = [li.power_matrix(n, seed=60 + i, dtype=np.float32) for i, n in enumerate(sizes)]
    count = 40
    t_s, views, ranks, factors, offsets = li.serving_trace(sizes, count, rate=5e4, seed=61)
    srv = P.Server(max_inflight=3, r_cap=8)
    try:
        ids = [srv.add_view(a, K) for a in a0]
        assert all(srv.view_state(i) == "resident" for i in ids)
        srv.replay(t_s, views, ranks, factors, offsets)
        srv.drain(timeout_s=180)
        recs = srv.poll()
        st = srv.stats()
        assert len(recs) == count and st["failed"] == 0
        assert all(r["status"] == 0 for r in recs)
        assert max(r["batch_size"] for r in recs) > 1 and st["max_inflight_seen"] >= 2
        mixed = {i: srv.program(i).read_view(L).cpu().numpy() for i in ids}
    finally:
        srv.close()
    g = np.random.default_rng(62)
    for i, n in enumerate(sizes):
        reqs = [li.trace_factors(sizes, views, ranks, factors, offsets, j)
                for j in range(count) if views[j] == i]
        prog = P.Program("power", [a0[i]], k=K, r_max=8)
        for u, v in reqs:
            prog.apply_delta(u, v)
        alone = prog.read_view(L).cpu().numpy()
        prog.close()
        assert rel_frob(mixed[i], alone) <= TOL, (i, n)
        rows = sorted(set(int(x) for x in g.choice(n, 16, replace=False)))
        if reqs:
            uall = np.concatenate([u for u, _ in reqs], axis=1)
            vall = np.concatenate([v for _, v in reqs], axis=1)
        else:
            uall = vall = np.zeros((n, 1))
        pr, _ = op.power_rows_factored(a0[i], uall, vall, rows, K)
        assert rel_frob(mixed[i][rows], pr[K]) <= TOL, (i, n)
        assert rel_frob(alone[rows], pr[K]) <= TOL, (i, n)


def _body_serve_admission_by_memory():
    P = _pkg()
    n = 512
    est = P.estimate_device_bytes(n, K, r_max=8)
    srv = P.Server(max_inflight=2, r_cap=8, hbm_budget_bytes=2 * est + est // 2)
    try:
        a0 = [li.power_matrix(n, seed=20 + i, dtype=np.float32) for i in range(3)]
        ids = [srv.add_view(a, K) for a in a0]
        assert [srv.view_state(i) for i in ids] == ["resident", "resident", "waiting"]
        st = srv.stats()
        assert st["views_resident"] == 2 and st["views_waiting"] == 1
        assert st["bytes_used"] == 2 * est
        reqs = {i: li.lowrank_update_stream(n, 2, 3, seed=30 + i, dtype=np.float32) for i in ids}
        for i in ids:
            for u, v in reqs[i]:
                srv.submit(i, u, v)
        # the resident views finish; the waiting one keeps its requests queued
        deadline = time.time() + 60
        done = []
        while time.time() < deadline and len(done) < 6:
            done += srv.poll()
            time.sleep(0.01)
        assert len(done) == 6 and {r["view"] for r in done} == {0, 1}
        assert srv.view_state(2) == "waiting"
        srv.remove_view(0)
        srv.drain(timeout_s=120)
        recs = srv.poll()
        assert len(recs) == 3 and {r["view"] for r in recs} == {2}
        assert all(r["status"] == 0 for r in recs)
        assert srv.view_state(0) == "removed" and srv.view_state(2) == "resident"
        got = srv.program(2).read_view(L).cpu().numpy().astype(np.float64)
        ref = op.reeval_powers(_final_a(a0[2], reqs[2]), K)[K]
        assert rel_frob(got, ref) <= TOL
        with pytest.raises(P.LinviewError):
            srv.submit(0, *reqs[0][0])
    finally:
        srv.close()


def _body_serve_remove_cancels_queue_and_errors():
    P = _pkg()
    n = 256
    srv = P.Server(max_inflight=1, r_cap=4)
    try:
        v = srv.add_view(li.power_matrix(n, seed=5, dtype=np.float32), 8)
        u, w = li.lowrank_update_stream(n, 5, 1, seed=6, dtype=np.float32)[0]
        wide = np.zeros((n, n + 1), np.float32)
        with pytest.raises(P.LinviewError) as e:
            srv.submit(v, wide, wide)  # rank n + 1 > n (a rank past r_cap is re-evaluation)
        assert e.value.name == "ERANK"
        with pytest.raises(P.LinviewError) as e:
            srv.submit(7, u[:, :1], w[:, :1])
        assert e.value.name == "EINVAL"
        with pytest.raises(P.LinviewError):
            srv.add_view(li.power_matrix(n, seed=5, dtype=np.float32), 6)  # k not a power of 2
        for _ in range(20):
            srv.submit(v, u[:, :2], w[:, :2])
        srv.remove_view(v)
        srv.drain(timeout_s=60)
        recs = srv.poll()
        assert len(recs) == 20
        # whatever was still queued at the removal completes with EINVAL
        assert all(r["status"] in (0, 1) for r in recs)
        assert srv.view_state(v) == "removed"
    finally:
        srv.close()


def _body_serve_row_coalescing():
    """Queued row updates to one view merge by row: each delta's rank is the
    number of distinct rows of the requests it carries (Section 6, batch
    updates), and the view equals the oracle on A + sum_j e_{i_j} v_j^T."""
    P = _pkg()
    n, count = 512, 60
    a0 = li.power_matrix(n, seed=50, dtype=np.float32)
    rows, vs = li.zipf_row_batch(n, count, 2.0, seed=51)
    assert len(np.unique(rows)) < count  # the batch repeats rows
    srv = P.Server(max_inflight=1, r_cap=8)
    try:
        v = srv.add_view(a0, K)
        srv.replay(np.zeros(count), np.zeros(count, np.int32), np.ones(count, np.int32),
                   np.ascontiguousarray(vs.reshape(-1)), np.arange(count) * n, rows=rows)
        srv.drain(timeout_s=120)
        recs = srv.poll()
        assert len(recs) == count and all(r["status"] == 0 for r in recs)
        batches = {}
        for r in recs:
            batches.setdefault(r["start_s"], []).append(r)
        merged = False
        for group in batches.values():
            distinct = {int(rows[r["ticket"] - 1]) for r in group}
            assert all(r["batch_rank"] == len(distinct) for r in group)
            assert all(r["batch_size"] == len(group) for r in group)
            merged |= len(group) > len(distinct)
        assert merged
        assert srv.stats()["refreshes"] == len(batches)
        got = srv.program(v).read_view(L).cpu().numpy().astype(np.float64)
    finally:
        srv.close()
    af = a0.astype(np.float64).copy()
    for i, w in zip(rows, vs):
        af[i] += w.astype(np.float64)
    assert rel_frob(got, op.reeval_powers(af, K)[K]) <= TOL


def _body_serve_over_cap_reeval():
    """A request of rank above r_cap is served by re-evaluation (Sec. 4.2.2):
    it and everything queued behind it go into A, every view is recomputed.
    Mixed with in-cap requests and row updates on one view; the view equals
    the oracle on A + all deltas, later in-cap requests refresh it
    incrementally again, and factors of the wrong shape are refused."""
    P = _pkg()
    n = 384
    a0 = li.power_matrix(n, seed=60, dtype=np.float32)
    g = np.random.default_rng(61)
    srv = P.Server(max_inflight=1, r_cap=2)
    reqs = []
    try:
        v = srv.add_view(a0, K)
        for rank in (1, 5, 2, 70, 1):   # 5 and 70 exceed r_cap; 70 spans two 64-column passes
            u = (g.standard_normal((n, rank)) * 0.01).astype(np.float32)
            w = (g.standard_normal((n, rank)) * 0.01).astype(np.float32)
            srv.submit(v, u, w)
            reqs.append((u, w))
        i = 17
        row = (g.standard_normal(n) * 0.01).astype(np.float32)
        srv.submit_row(v, i, row)
        e = np.zeros((n, 1), np.float32)
        e[i] = 1
        reqs.append((e, row.reshape(-1, 1)))
        srv.drain(timeout_s=120)
        recs = srv.poll()
        st = srv.stats()
        assert len(recs) == len(reqs) and all(r["status"] == 0 for r in recs), recs
        assert st["reevals"] >= 1 and st["failed"] == 0
        got = srv.program(v).read_view(L).cpu().numpy().astype(np.float64)
        assert rel_frob(got, op.reeval_powers(_final_a(a0, reqs), K)[K]) <= TOL
        # incremental refreshes resume after the re-evaluation
        u = (g.standard_normal((n, 2)) * 0.01).astype(np.float32)
        w = (g.standard_normal((n, 2)) * 0.01).astype(np.float32)
        srv.submit(v, u, w)
        reqs.append((u, w))
        srv.drain(timeout_s=120)
        assert srv.stats()["reevals"] == st["reevals"]
        got = srv.program(v).read_view(L).cpu().numpy().astype(np.float64)
        assert rel_frob(got, op.reeval_powers(_final_a(a0, reqs), K)[K]) <= TOL
        for bad in ((np.zeros((n - 1, 2), np.float32),) * 2,
                    (np.zeros((n, 2), np.float32), np.zeros((n, 3), np.float32))):
            try:
                srv.submit(v, *bad)
            except ValueError:
                pass
            else:
                raise AssertionError("wrong factor shapes accepted")
    finally:
        srv.close()


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run_child(body, timeout=300):
    env = dict(os.environ, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, os.path.abspath(__file__), body], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=timeout)
    assert r.returncode == 0, f"{body} failed:\n{r.stdout[-3000:]}\n{r.stderr[-3000:]}"


def test_serve_alone_vs_mix():
    _run_child("serve_alone_vs_mix")


def test_serve_alone_vs_mix_full_sizes():
    _run_child("serve_alone_vs_mix_full_sizes", timeout=600)


def test_serve_admission_by_memory():
    _run_child("serve_admission_by_memory")


def test_serve_remove_cancels_queue_and_errors():
    _run_child("serve_remove_cancels_queue_and_errors")


def test_serve_row_coalescing():
    _run_child("serve_row_coalescing")


def test_serve_over_cap_reeval():
    _run_child("serve_over_cap_reeval")


@pytest.mark.parametrize("kind,n,k,r_max,model", [
    ("power", 1000, 16, 8, "exp"), ("power", 256, 8, 1, "exp"), ("power_sum", 777, 16, 4, "exp"),
    ("power_sum", 512, 4, 2, "exp"), ("power", 300, 16, 4, "linear"),
    ("power_sum", 300, 5, 1, "linear"), ("power", 300, 16, 2, "skip"),
    ("power_sum", 300, 16, 4, "skip")])
def test_estimate_equals_program_bytes(kind, n, k, r_max, model):
    P = _pkg()
    a = li.power_matrix(n, seed=1, dtype=np.float32)
    skip = 4 if model == "skip" else 0
    prog = P.Program(kind, [a], k=k, r_max=r_max, model=model, skip=skip)
    try:
        assert P.program_device_bytes(prog) == P.estimate_device_bytes(n, k, r_max=r_max, kind=kind,
                                                                       model=model, skip=skip)
    finally:
        prog.close()


if __name__ == "__main__":  # child process of _run_child
    globals()["_body_" + sys.argv[1]]()
    print("ok", sys.argv[1])
