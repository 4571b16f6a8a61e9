#!/usr/bin/env python
"""Benchmark: incremental view refresh of A^16 and S' = A + ... + A^16 on one GB300.

Workload (the paper's powers / sums-of-powers experiments, Section 6, at the
GPU-sized configuration): A is 8192 x 8192 FP32 with i.i.d. N(0,1)/(2 sqrt n)
entries; a stream of rank-1 row updates dA = e_i v^T (i uniform, v ~
N(0, 0.01^2)) arrives; after every update all nine views (A, A^2, A^4, A^8,
A^16, S'_2, S'_4, S'_8, S'_16) are refreshed in place by the exponential-model
trigger.  A step is one update = one refresh of every view.

Printed JSON line: refreshes/s (device-timed, inputs resident), e2e through the
public API with host buffers, p50/p99 step latency, the view-pass kernels'
achieved HBM bandwidth against the measured copy bandwidth, GPU re-evaluation of
the same views in three GEMM arithmetics, and the FP64 CPU oracle on a bounded
sample (``cpu_baseline``).  ``--impl reference`` times the FP64 oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("view refreshes/s incremental vs GPU re-eval, 1 GB300, rel err≤1e-4; "
          "p99 latency")
UNIT = "refreshes/s"
WORKLOAD = ("A^16 and S'=sum_{i=1..16} A^i (9 views) maintained under rank-1 row updates "
            "dA=e_i v^T, n=8192, FP32, A~N(0,1)/(2 sqrt n), v~N(0,0.01^2)")


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    # --matrix-n: the same option under a name that no torchrun option starts
    # with (torchrun's parser rejects "--n" as an ambiguous abbreviation)
    ap.add_argument("--n", "--matrix-n", dest="n", type=int, default=8192)
    ap.add_argument("--k", type=int, default=16)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--reeval-steps", type=int, default=3)
    ap.add_argument("--cpu-sample", type=int, default=12,
                    help="oracle updates timed (about 10 s of host work at n = 8192)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--serve-rates", default="1e2,1e3,3e3,1e4,3e4,1e5",
                    help="request rates (per s) of the serving sweep")
    ap.add_argument("--serve-views", type=int, default=32)
    ap.add_argument("--serve-inflight", type=int, default=8,
                    help="views refreshing at once in the serving sweep")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-rank4", action="store_true")
    ap.add_argument("--no-ksweep", action="store_true")
    ap.add_argument("--no-ols", action="store_true", help="skip the OLS row-block section")
    ap.add_argument("--no-general", action="store_true")
    ap.add_argument("--gemm-n", type=int, default=8192, help="size of the gemm section's products")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the general form at the paper's n = 30000")
    ap.add_argument("--no-gemm", action="store_true")
    ap.add_argument("--no-drift", action="store_true",
                    help="skip the residual-correction drift section (two 200-update streams)")
    ap.add_argument("--only", default=None,
                    choices=["rank4_stream", "k_sweep", "iteration_p_sweep", "gd_regression",
                             "small_fp64", "ols_row_blocks", "iteration_adjoint", "serving",
                             "zipf_batches", "drift", "gemm", "iteration_p_sweep_n30000",
                             "gd_regression_n30000", "ols_drift", "serving_inflight"],
                    help="run one secondary section alone (no headline line): profiling")
    return ap.parse_args()


# ---------------------------------------------------------------- distributed
def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _dist_init(ws, local, use_cuda):
    import torch
    import torch.distributed as dist
    if ws > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        if use_cuda:
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if use_cuda else "gloo")
    return dist if ws > 1 else None


def _barrier(dist):
    if dist is not None:
        dist.barrier()


def _weak_value(ws, steps, max_ms):
    """Whole-job throughput of ``ws`` replicas that each ran ``steps`` steps,
    the slowest in ``max_ms`` milliseconds (weak scaling: units of all ranks
    over the max-over-ranks time)."""
    return ws * steps / (max_ms / 1e3)


def _max_over_ranks(dist, x, use_cuda):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if use_cuda else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampling during the timed region (200 ms period)."""

    def __init__(self, uuid, enabled=True):
        self.uuid = uuid
        self.proc = None
        self.path = None
        self.enabled = enabled

    def start(self):
        if not self.enabled:
            return
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        q = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            if self.uuid and self.uuid not in f[0]:
                continue
            rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def _uuid():
    try:
        import torch
        u = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def _pass_source_hash():
    """Hash of the view-pass kernel sources and of the parameter block they
    take (a capture is stale once either changes)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1403_6968_gb300", "csrc")
    for f in ("lv_pass.cu", "lv_pass_ws.cuh", "lv_device.cuh"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    hdr = open(os.path.join(csrc, "lv_internal.h"), "rb").read()
    a = hdr.index(b"struct PassParams {")
    h.update(hdr[a:hdr.index(b"};", a)])
    return h.hexdigest()[:16]


def _traffic(kernel):
    """DRAM bytes per launch of ``kernel`` from the committed ncu summary, or
    None when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    h = _pass_source_hash()
    e = d.get(kernel)
    if not e or e.get("pass_source_sha256_16") != h:
        return None
    return e.get("dram_bytes_per_launch_full_size")


# ---------------------------------------------------------------- CPU oracle
def cpu_oracle_rate(n, k, updates, seed=0):
    """The FP64 oracle's incremental refresh (as it stands) on ``updates`` row
    updates of the same workload; returns (refreshes/s, seconds, setup s)."""
    import numpy as np
    import linview_inputs as li
    from oracle import powers as op
    a = li.power_matrix(n, seed=seed, dtype=np.float32).astype(np.float64)
    t0 = time.perf_counter()
    inc = op.IncrementalPowers(a, k, sums=True)
    setup = time.perf_counter() - t0
    ups = li.row_update_stream(n, updates, seed=seed + 1000, dtype=np.float32)
    t0 = time.perf_counter()
    for i, v in ups:
        inc.apply_row(i, v.astype(np.float64))
    dt = time.perf_counter() - t0
    return updates / dt, dt, setup


def cpu_oracle_errors(a32, ups, rows, row_sets, k):
    """Part of the CPU-baseline leg: the FP64 oracle's rows ``rows`` of every
    view after the row updates ``ups`` (applied in order to the FP32-rounded
    A promoted to FP64), against each set of the same rows read back from the
    GPU (``row_sets``: set name -> {view name -> array}).  Returns, per set,
    the per-view relative Frobenius errors."""
    import numpy as np
    from oracle import powers as op
    from oracle.metrics import rel_frob
    a = a32.astype(np.float64)
    for i, v in ups:
        a[i] += v.astype(np.float64)
    pr, sr = op.power_rows(a, rows, k)
    out = {}
    for set_name, gpu_rows in row_sets.items():
        errs = {}
        for name, got in gpu_rows.items():
            h = int(name[1:])
            errs[name] = rel_frob(got, (pr if name[0] == "P" else sr)[h])
        out[set_name] = errs
    return out


def drift_oracle_errors(d, a32, k):
    """Part of the CPU-baseline leg: the FP64 oracle's rows at every checked
    update of a drift_streams run, against the GPU rows of both runs."""
    import numpy as np
    from oracle import powers as op
    from oracle.metrics import rel_frob
    a0 = a32.astype(np.float64)
    out = {}
    for name, st in d["streams"].items():
        ups = st["ups"]
        res = {cp: {} for cp in st["runs"]}
        for t in d["checks"]:
            rows = st["runs"][0]["rows_at"][t]["rows"]
            if name == "rank1":
                a = a0.copy()
                for i, v in ups[:t]:
                    a[i] += v.astype(np.float64)
                pr, sr = op.power_rows(a, rows, k)
            else:
                u = np.concatenate([x for x, _ in ups[:t]], axis=1)
                v = np.concatenate([y for _, y in ups[:t]], axis=1)
                pr, sr = op.power_rows_factored(a0, u, v, rows, k)
            for cp, run in st["runs"].items():
                got = run["rows_at"][t]
                assert got["rows"] == rows
                res[cp][t] = {nm: rel_frob(x, (pr if nm[0] == "P" else sr)[int(nm[1:])])
                              for nm, x in got["views"].items()}
        out[name] = res
    return out


def _cores():
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(var):
            return int(os.environ[var])
    return os.cpu_count()


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import numpy as np
    import linview_inputs as li
    from oracle import powers as op
    n, k = args.n, args.k
    a = li.power_matrix(n, seed=0, dtype=np.float32).astype(np.float64)
    inc = op.IncrementalPowers(a, k, sums=True)
    ups = li.row_update_stream(n, args.warmup + args.steps, seed=0, dtype=np.float32)
    for i, v in ups[:args.warmup]:
        inc.apply_row(i, v.astype(np.float64))
    lat = []
    t0 = time.perf_counter()
    for i, v in ups[args.warmup:]:
        s = time.perf_counter()
        inc.apply_row(i, v.astype(np.float64))
        lat.append(time.perf_counter() - s)
    dt = time.perf_counter() - t0
    val = args.steps / dt
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "strategy": "FP64 CPU oracle, incremental "
                      "exponential model (numpy BLAS)"},
           "latency_ms": {"p50": 1e3 * statistics.median(lat),
                          "p99": 1e3 * float(np.percentile(lat, 99))},
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": _cores(), "kind": "oracle",
                            "sample": f"{args.steps} row updates at n={n} after {args.warmup} "
                                      "warm-up updates (views initialised by the oracle's own "
                                      "re-evaluation, untimed)"},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch
    ws, rank, local = _dist()
    dist = _dist_init(ws, local, True)
    torch.cuda.set_device(local)
    import __graft_entry__ as g
    g.build()
    import linview_inputs as li
    from paper_1403_6968_gb300 import Program

    n, k = args.n, args.k
    L = k.bit_length() - 1
    K, W, E = args.steps, args.warmup, args.e2e_steps
    a = li.power_matrix(n, seed=rank, dtype=np.float32)
    KR = min(K, 16)  # updates of the roofline region (one per instrumented graph copy)
    ups = li.row_update_stream(n, W + 1 + K + KR + E + 4 * args.reeval_steps + 1, seed=rank,
                               dtype=np.float32)
    dev_v = [torch.from_numpy(v).cuda() for _, v in ups]
    rows = [i for i, _ in ups]
    prog = Program("power_sum", [torch.from_numpy(a).cuda()], k=k, r_max=1)
    stream = torch.cuda.current_stream()
    for t in range(W):
        prog.apply_row_delta(rows[t], dev_v[t])
    # one more warm-up update with per-pass timing on: the library captures the
    # instrumented copies of the propagation graph here, outside both regions
    prog.set_profiling(True)
    prog.apply_row_delta(rows[W], dev_v[W])
    prog.set_profiling(False)
    W1 = W + 1  # first update of the timed region
    torch.cuda.synchronize()
    _barrier(dist)
    clocks = Clocks(_uuid(), enabled=not args.no_clocks)
    clocks.start()
    prog.reset_stats()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    torch.cuda.synchronize()
    evs[0].record(stream)
    for t in range(K):
        prog.apply_row_delta(rows[W1 + t], dev_v[W1 + t])
        evs[t + 1].record(stream)
    torch.cuda.synchronize()
    _barrier(dist)
    clk = clocks.stop()
    lat = [evs[t].elapsed_time(evs[t + 1]) for t in range(K)]
    tot_ms = evs[0].elapsed_time(evs[K])
    launches_timed = prog.pass_stats(0)["all_launches"]
    prog.sync()
    # roofline region: KR more updates, the same graph replays with an event
    # pair recorded around every view pass on the stream the passes run on
    # (kept apart from the region above: the event nodes add launch gaps)
    prog.reset_stats()
    prog.set_profiling(True)
    er0, er1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    er0.record(stream)
    for t in range(KR):
        prog.apply_row_delta(rows[W1 + K + t], dev_v[W1 + K + t])
    er1.record(stream)
    torch.cuda.synchronize()
    roof_region_ms = er0.elapsed_time(er1)
    st_all = prog.pass_stats(0)
    st_f = prog.pass_stats(1)
    st_u = prog.pass_stats(2)
    prog.set_profiling(False)
    prog.reset_stats()
    prog.sync()
    max_ms = _max_over_ranks(dist, tot_ms, True)
    value = _weak_value(ws, K, max_ms)

    # roofline of the dominant view-pass kernel (per-launch algorithmic bytes:
    # one read + one write of an n x n FP32 view)
    peaks = _peaks()
    peak = peaks.get("hbm_gbs") if peaks else 6800.0
    peak_src = "measured" if peaks else "fallback"
    dom, st = ("lv::update_ws_kernel", st_u) if st_u["ms"] >= st_f["ms"] else \
        ("lv::fused_ws_kernel", st_f)
    per_launch = st["bytes"] / max(st["launches"], 1)
    avg_s = st["ms"] / 1e3 / max(st["launches"], 1)
    achieved = per_launch / avg_s / 1e9
    other = st_f if st is st_u else st_u
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": _traffic(dom), "kernel": dom,
            "peak_source": f"{peak_src} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
            "algorithmic_bytes_per_launch": per_launch,
            "launches": st["launches"], "avg_launch_us": avg_s * 1e6,
            "window": f"a second timed region of {KR} updates right after the first: the same "
                      "propagation replays with a CUDA event pair recorded around each view "
                      "pass, on the stream the passes run on; here the sums passes run on the "
                      "main stream, each pass alone (in the timed region they overlap the level "
                      "passes on a side stream)",
            "window_ms_per_step": roof_region_ms / KR,
            "all_view_passes": {"launches": st_all["launches"],
                                "achieved_gbs": st_all["bytes"] / (st_all["ms"] / 1e3) / 1e9},
            "other_pass_kernel": {"launches": other["launches"],
                                  "achieved_gbs": (other["bytes"] / (other["ms"] / 1e3) / 1e9)
                                  if other["ms"] > 0 else None}}
    bytes_per_refresh = (2 * L + 1) * 2.0 * n * n * 4
    step_s = max_ms / 1e3 / K

    # e2e through the public API: host v (pinned) in, one refreshed row of
    # A^16 out, every step.  Two steps in flight: step t's row is copied out
    # asynchronously into its own pinned buffer, and the host waits for step
    # t-1's row (which it then holds) before issuing step t+1, so the GPU is
    # not idle while the host issues the next step; every step's copies are
    # inside the timed region, which ends when the last row is on the host.
    e2e = None
    if E > 0:
        E0 = W1 + K + KR  # first update of the e2e region
        pin_v = [torch.from_numpy(v).pin_memory() for _, v in ups[E0:E0 + E]]
        row_out = [torch.empty((1, n), dtype=torch.float32).pin_memory() for _ in range(2)]
        got = [torch.cuda.Event() for _ in range(2)]
        cur = torch.cuda.current_stream()
        torch.cuda.synchronize()
        _barrier(dist)
        t0 = time.perf_counter()
        for t in range(E):
            i = rows[E0 + t]
            b = t % 2
            prog.apply_row_delta(i, pin_v[t])
            prog.read_view_rows(L, i, 1, out=row_out[b], sync=False)
            got[b].record(cur)
            if t >= 1:
                got[1 - b].synchronize()   # step t-1's row is on the host
        got[(E - 1) % 2].synchronize()
        e2e_s = _max_over_ranks(dist, time.perf_counter() - t0, True)
        # the last row read back is the refreshed row of A^16 (checked below
        # against a synchronous read of the same row)
        last = rows[E0 + E - 1]
        ref_row = prog.read_view_rows(L, last, 1)
        e2e = {"value": ws * E / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 4 * n,
               "d2h_bytes_per_step": 4 * n, "steps": E, "in_flight": 2,
               "last_row_matches": bool(np.array_equal(row_out[(E - 1) % 2].numpy(), ref_row))}

    # rows of every view after all the updates so far (the timed stream, the
    # roofline window and the e2e region), for the error against the FP64
    # oracle: the last 8 updated rows and 8 fixed ones
    applied = W1 + K + KR + (E if E > 0 else 0)
    chk_rows = sorted(set(rows[applied - 8:applied]) |
                      {0, 1, n // 7, n // 3, n // 2, (2 * n) // 3, n - 2, n - 1})
    torch.cuda.synchronize()
    gpu_rows = {}
    for j in range(L + 1):
        gpu_rows[f"P{1 << j}"] = np.stack([prog.read_view_rows(j, i, 1)[0] for i in chk_rows])
    for j in range(1, L + 1):
        gpu_rows[f"S{1 << j}"] = np.stack([prog.read_view_rows(L + j, i, 1)[0]
                                           for i in chk_rows])

    # GPU re-evaluation of the same views (the paper's re-evaluation strategy:
    # apply dA to A, recompute every view): the library's own split-TF32
    # tensor-core GEMM first, then the cuBLAS arithmetics as comparison
    # denominators.  Each mode's views at the current A (sampled rows) are
    # compared with the FP64 oracle in the CPU-baseline leg below.
    reeval, speed = {}, {}
    modes = ("tc3", "bf16x9", "tf32", "fp32")
    reeval_rows = {}
    if args.reeval_steps > 0:
        for mode in modes:
            prog.set_reeval_mode(mode)
            prog.reeval()
            torch.cuda.synchronize()
            rr = {}
            for j in range(L + 1):
                rr[f"P{1 << j}"] = np.stack([prog.read_view_rows(j, i, 1)[0] for i in chk_rows])
            for j in range(1, L + 1):
                rr[f"S{1 << j}"] = np.stack([prog.read_view_rows(L + j, i, 1)[0]
                                             for i in chk_rows])
            reeval_rows[mode] = rr
        # re-evaluation strategy per update: apply dA to A (a level pass,
        # 0.3 ms, untimed), then recompute every view (timed with CUDA events);
        # each arithmetic warmed up once first (library set-up, work space)
        aptr, ald = prog.view_device_ptr(0)
        ti = W1 + K + KR + E
        for mode in modes:
            prog.set_reeval_mode(mode)
            prog.reeval()
            tot = 0.0
            for t in range(args.reeval_steps):
                u = torch.zeros((1, n), dtype=torch.float32, device="cuda")
                u[0, rows[ti]] = 1.0
                _apply_to_a(aptr, ald, n, u, dev_v[ti].reshape(1, n))
                ti += 1
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                prog.reeval()
                e1.record(stream)
                torch.cuda.synchronize()
                tot += e0.elapsed_time(e1)
            ms = tot / args.reeval_steps
            reeval[mode] = {"refreshes_per_s": 1e3 / ms, "ms_per_refresh": ms,
                            "gemm": "own tcgen05 split TF32" if mode == "tc3" else "cuBLAS"}
        prog.set_reeval_mode("default")

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K,
           "warmup": W, "ms_per_step": max_ms / K, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n": n, "k": k, "views": 2 * L + 1,
                      "update": "rank-1 row", "parallelism": "replicas" if ws > 1 else "single",
                      "l2": "inputs larger than L2: 9 views x 268 MB = 2.4 GB per refresh",
                      "bytes_per_refresh_algorithmic": bytes_per_refresh},
           "latency_ms": {"p50": statistics.median(lat), "p99": float(np.percentile(lat, 99)),
                          "max": max(lat)},
           "achieved_refresh_gbs": bytes_per_refresh / step_s / 1e9,
           # the whole refresh (all 9 view passes, the sums passes overlapping the
           # level passes) against the same measured copy bandwidth
           "achieved_refresh_frac": bytes_per_refresh / step_s / 1e9 / peak,
           "roofline": roof, "e2e": e2e, "gpu_launches": launches_timed,
           "reeval": reeval, "speedup": speed, "clocks": clk}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        errs_all = cpu_oracle_errors(a, ups[:applied], chk_rows,
                                     dict(incremental=gpu_rows, **reeval_rows), k)
        errs = errs_all["incremental"]
        out["oracle_rel_err"] = {
            "per_view": errs, "max": max(errs.values()), "tolerance": 1e-4,
            "rows": len(chk_rows), "after_updates": applied,
            "how": "sampled rows (the last 8 updated rows and 8 fixed ones) of every view "
                   "after all the updates of the run so far, against the FP64 oracle's rows "
                   "of A^h and S'_h computed row by row on the updated A"}
        for mode in reeval:
            reeval[mode]["oracle_rel_err_max"] = max(errs_all[mode].values())
            reeval[mode]["oracle_rel_err"] = errs_all[mode]
        if reeval:
            acc = [m for m in reeval if reeval[m]["oracle_rel_err_max"] <= 1e-4]
            fastest_acc = max(acc, key=lambda m: reeval[m]["refreshes_per_s"]) if acc else None
            fastest_any = max(reeval, key=lambda m: reeval[m]["refreshes_per_s"])
            out["speedup"] = {
                "vs_fastest_accurate_reeval":
                    (value / ws) / reeval[fastest_acc]["refreshes_per_s"] if fastest_acc else None,
                "fastest_accurate_reeval": fastest_acc,
                "vs_own_reeval": (value / ws) / reeval["tc3"]["refreshes_per_s"],
                "vs_fastest_any_reeval": (value / ws) / reeval[fastest_any]["refreshes_per_s"],
                "fastest_any_reeval": fastest_any,
                "accurate": "oracle_rel_err_max <= 1e-4 on the sampled rows of every view"}
        rate, dt, setup = cpu_oracle_rate(n, k, args.cpu_sample)
        out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": _cores(), "kind": "oracle",
                               "sample": f"{args.cpu_sample} rank-1 row updates of the same "
                                         f"workload at n={n} (FP64 numpy oracle; its own "
                                         f"re-evaluation setup of {setup:.1f} s untimed)"}
    prog.close()
    # secondary workloads: a failure in one is recorded in its field and does
    # not take the headline line down with it
    def section(name, fn):
        try:
            out[name] = fn()
        except Exception as e:  # noqa: BLE001
            out[name] = {"error": f"{type(e).__name__}: {e}"}

    if not args.no_rank4:
        section("rank4_stream", lambda: rank_stream(args, 4, seed=rank))
    if not args.no_gemm:
        section("gemm", lambda: gemm_section(args))
    if not args.no_drift and ws == 1:
        section("drift", lambda: drift_report(drift_streams(args), _drift_a(args), k,
                                              not args.no_cpu_baseline))
        if not args.no_ols:
            section("ols_drift", lambda: ols_drift_report(ols_drift_streams(seed=rank),
                                                          not args.no_cpu_baseline))
    if not args.no_ksweep:
        section("k_sweep", lambda: k_sweep(args, seed=rank))
    if not args.no_general:
        section("iteration_p_sweep", lambda: iteration_p_sweep(args, seed=rank))
        section("gd_regression", lambda: gd_regression(seed=rank))
    if not args.no_general and not args.no_large:
        # the paper's sizes for the general form (Section 6: n = 30K, p up to 1000)
        section("iteration_p_sweep_n30000",
                lambda: iteration_p_sweep(args, seed=rank, steps=3, n=30000))
        section("gd_regression_n30000", lambda: gd_regression_device(seed=rank))
    section("small_fp64", lambda: small_fp64(seed=rank))
    if not args.no_ols:
        section("ols_row_blocks", lambda: ols_sweep(seed=rank))
    if not args.no_general:
        section("iteration_adjoint", lambda: iteration_adjoint(seed=rank))
    if rank == 0 and not args.no_serving:
        section("serving", lambda: serving_sweep(args, seed=rank))
        section("serving_inflight", lambda: serving_inflight(args, seed=rank))
        section("zipf_batches", lambda: zipf_batches(args, seed=rank))
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def rank_stream(args, r, seed=0, steps=20, warmup=3):
    """The same powers + sums program under the rank-r stream dA = U V^T
    (U, V ~ N(0, 0.01^2), n x r): refreshes/s with inputs resident."""
    import numpy as np
    import torch
    import linview_inputs as li
    from paper_1403_6968_gb300 import Program

    n, k = args.n, args.k
    a = li.power_matrix(n, seed=seed, dtype=np.float32)
    ups = [(torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda())
           for u, v in li.lowrank_update_stream(n, r, warmup + steps, seed=seed, dtype=np.float32)]
    prog = Program("power_sum", [torch.from_numpy(a).cuda()], k=k, r_max=r)
    for u, v in ups[:warmup]:
        prog.apply_delta(u, v)
    stream = torch.cuda.current_stream()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    prog.reset_stats()
    torch.cuda.synchronize()
    evs[0].record(stream)
    for t, (u, v) in enumerate(ups[warmup:]):
        prog.apply_delta(u, v)
        evs[t + 1].record(stream)
    torch.cuda.synchronize()
    launches = prog.pass_stats(0)["all_launches"]
    prog.sync()
    lat = [evs[t].elapsed_time(evs[t + 1]) for t in range(steps)]
    tot_ms = evs[0].elapsed_time(evs[steps])
    prog.close()
    L = k.bit_length() - 1
    alg = (2 * L + 1) * 2.0 * n * n * 4
    return {"rank": r, "steps": steps, "refreshes_per_s": steps / (tot_ms / 1e3),
            "ms_per_step": tot_ms / steps, "p50_ms": statistics.median(lat),
            "p99_ms": float(np.percentile(lat, 99)), "gpu_launches": launches,
            "achieved_refresh_gbs": alg / (tot_ms / steps / 1e3) / 1e9,
            "note": "achieved GB/s counts each of the 9 views read and written once per "
                    "refresh (the method's minimum traffic)"}


def drift_streams(args, seed=0, count=200, period=64, checks=(1, 50, 100, 150, 200)):
    """Residual correction, measured: the powers + sums program (A^16 and S',
    n = 8192, FP32) under the 200-update rank-1 row stream and the 200-update
    rank-4 stream, once without correction and once re-evaluated every
    ``period`` updates (the library's own split-TF32 GEMM).  At the checked
    updates, sampled rows of every view are read back; the CPU-baseline leg
    compares them with the FP64 oracle (drift_oracle_errors).  Reports the
    time of an ordinary update and of a correcting one."""
    import numpy as np
    import torch
    import linview_inputs as li
    from paper_1403_6968_gb300 import Program

    n, k = args.n, args.k
    L = k.bit_length() - 1
    a = li.power_matrix(n, seed=seed, dtype=np.float32)
    g = np.random.default_rng(4321)
    fixed = sorted(set(int(i) for i in g.choice(n, 14, replace=False)) | {0, n - 1})
    vnames = [f"P{1 << j}" for j in range(L + 1)] + [f"S{1 << j}" for j in range(1, L + 1)]
    vids = list(range(L + 1)) + [L + j for j in range(1, L + 1)]
    streams = {}
    for rank in (1, 4):
        if rank == 1:
            ups = li.row_update_stream(n, count, seed=seed, dtype=np.float32)
            dev = [(int(i), torch.from_numpy(v).cuda()) for i, v in ups]
        else:
            ups = li.lowrank_update_stream(n, 4, count, seed=seed, dtype=np.float32)
            dev = [(torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda()) for u, v in ups]
        runs = {}
        for cp in (0, period):
            prog = Program("power_sum", [torch.from_numpy(a).cuda()], k=k, r_max=rank,
                           correction_period=cp)
            stream = torch.cuda.current_stream()
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(count + 1)]
            rows_at = {}
            torch.cuda.synchronize()
            evs[0].record(stream)
            for t in range(1, count + 1):
                if rank == 1:
                    prog.apply_row_delta(*dev[t - 1])
                else:
                    prog.apply_delta(*dev[t - 1])
                evs[t].record(stream)
                if t in checks:
                    rows = sorted(set(fixed) | ({dev[t - 1][0]} if rank == 1 else set()))
                    torch.cuda.synchronize()
                    rows_at[t] = {"rows": rows, "views": {
                        nm: np.stack([prog.read_view_rows(vid, i, 1)[0] for i in rows])
                        for nm, vid in zip(vnames, vids)}}
                    evs[t].synchronize()
            torch.cuda.synchronize()
            # per-update times (an event pair per update; the checks happen
            # outside the measured intervals only for the update they follow)
            ms = [evs[t - 1].elapsed_time(evs[t]) for t in range(1, count + 1)
                  if (t - 1) not in checks]
            corr = [evs[t - 1].elapsed_time(evs[t]) for t in range(1, count + 1)
                    if cp and t % cp == 0 and (t - 1) not in checks]
            plain = [evs[t - 1].elapsed_time(evs[t]) for t in range(1, count + 1)
                     if not (cp and t % cp == 0) and (t - 1) not in checks]
            runs[cp] = {"rows_at": rows_at,
                        "ms_per_update": float(np.mean(ms)),
                        "ms_plain_update": float(np.median(plain)),
                        "ms_correcting_update": float(np.median(corr)) if corr else None}
            prog.close()
        streams[f"rank{rank}"] = {"ups": ups, "runs": runs}
    return {"n": n, "k": k, "updates": count, "correction_period": period,
            "checks": list(checks), "streams": streams}


def drift_report(d, a32, k, with_oracle):
    """The JSON form of a drift_streams result; with_oracle: add the FP64
    oracle errors (part of the CPU-baseline leg)."""
    out = {"n": d["n"], "k": d["k"], "updates": d["updates"],
           "correction_period": d["correction_period"], "checks": d["checks"], "streams": {}}
    errs = drift_oracle_errors(d, a32, k) if with_oracle else None
    for name, st in d["streams"].items():
        rep = {}
        for cp, run in st["runs"].items():
            key = "no_correction" if cp == 0 else f"corrected_every_{cp}"
            r = {"ms_per_update": run["ms_per_update"], "ms_plain_update": run["ms_plain_update"],
                 "ms_correcting_update": run["ms_correcting_update"]}
            if errs is not None:
                e = errs[name][cp]
                r["oracle_rel_err_max_at"] = {str(t): max(v.values()) for t, v in e.items()}
                last = max(e)
                r["oracle_rel_err_per_view_at_last"] = e[last]
            rep[key] = r
        out["streams"][name] = rep
    out["how"] = ("sampled rows (14 fixed, plus the updated row for row updates) of all 9 views "
                  "at the checked updates vs the FP64 oracle's rows computed from the plain "
                  "definition on the updated A; times are CUDA-event intervals per update")
    return out


def ols_drift_streams(seed=0, m=65536, n=4096, p=16, ks=(1, 4, 16), count=100, period=50,
                      checks=(1, 49, 50, 99, 100), nrows=16):
    """Residual correction of OLS, measured: per k, 100 row-block updates of
    the OLS workload (m = 65536, n = 4096, p = 16, FP32) through a program
    without correction and through one created with correction="newton" and
    correction_period = ``period`` (a Newton-Schulz step W <- W + W (I - Z W)
    from the maintained Z = X^T X after every ``period``-th update).  At the
    checked updates ``nrows`` sampled rows of W and all of beta are read back;
    the CPU-baseline leg compares them with the FP64 oracle
    (ols_drift_oracle_errors).  Also times an update of each program and a
    correction alone."""
    import numpy as np
    import torch
    import linview_inputs as li
    from paper_1403_6968_gb300 import Program

    x, y, _ = li.ols_inputs(m, n, p, seed=seed, dtype=np.float32)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    g = np.random.default_rng(97)
    rows_s = sorted(set(int(i) for i in g.choice(n, nrows - 2, replace=False)) | {0, n - 1})
    out = {}
    for k in ks:
        ups = li.ols_row_replacements(m, n, k, count, seed=seed + 100 + k, dtype=np.float32,
                                      cols_seed=seed)
        dev = [(r_, torch.from_numpy(nw).cuda()) for r_, nw in ups]
        runs = {}
        for variant in ("no_correction", "newton"):
            kw = {"correction": "newton", "correction_period": period} if variant == "newton" else {}
            prog = Program("ols", [xd, yd], k=k, **kw)
            prog.sync()
            stream = torch.cuda.current_stream()
            # an event pair around every update (the checks' host reads fall
            # outside every interval)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(count + 1)]
            at = {}
            for t in range(1, count + 1):
                ev[t][0].record(stream)
                prog.apply_row_block(*dev[t - 1])
                ev[t][1].record(stream)
                if t in checks:
                    prog.sync()
                    at[t] = {"W_rows": np.stack([prog.read_view_rows(0, i, 1)[0] for i in rows_s]),
                             "beta": prog.read_view_host(1)}
            prog.sync()
            corrects = variant == "newton"
            plain = [ev[t][0].elapsed_time(ev[t][1]) for t in range(1, count + 1)
                     if not (corrects and t % period == 0)]
            r = {"at": at, "ms_update": float(np.median(plain))}
            if corrects:
                # the updates that end in a correction: the update, Z brought up to
                # date with the history since the last correction, the step
                r["ms_correcting_update"] = float(np.median(
                    [ev[t][0].elapsed_time(ev[t][1]) for t in range(period, count + 1, period)]))
                r["ms_correction_alone"] = _event_ms(lambda j: prog.correct(), 2)
                # (the timed corrections changed W: nothing is read after them)
            runs[variant] = r
            prog.close()
        out[k] = {"ups": ups, "runs": runs}
    return {"m": m, "n": n, "p": p, "updates": count, "correction_period": period,
            "checks": list(checks), "rows": rows_s, "x": x, "y": y, "ks": out}


def ols_drift_oracle_errors(d):
    """Part of the CPU-baseline leg: the FP64 oracle (IncrementalOLS: X, Z =
    X^T X and X^T Y carried exactly under the same replacements) at every
    checked update, W = inv(Z) and beta = W X^T Y from the definition; the
    relative Frobenius error of the program's sampled W rows and beta."""
    import copy
    import numpy as np
    from oracle import ols as oo
    from oracle.metrics import rel_frob

    base = oo.IncrementalOLS(d["x"], d["y"])
    rows = d["rows"]
    errs = {}
    for k, kd in d["ks"].items():
        ref = copy.deepcopy(base)
        e = {v: {} for v in kd["runs"]}
        for t, (r_, nw) in enumerate(kd["ups"], start=1):
            ref.replace_rows(r_, nw.astype(np.float64))
            if t in d["checks"]:
                w = np.linalg.inv(ref.z)
                beta = w @ ref.xty
                for v, run in kd["runs"].items():
                    got = run["at"][t]
                    e[v][t] = {"W": rel_frob(got["W_rows"], w[rows]),
                               "beta": rel_frob(got["beta"], beta)}
        errs[k] = e
    return errs


def ols_drift_report(d, with_oracle):
    out = {"m": d["m"], "n": d["n"], "p": d["p"], "updates": d["updates"],
           "correction_period": d["correction_period"], "checks": d["checks"], "k": {}}
    errs = ols_drift_oracle_errors(d) if with_oracle else None
    for k, kd in d["ks"].items():
        rep = {}
        for v, run in kd["runs"].items():
            r = {k2: v2 for k2, v2 in run.items() if k2.startswith("ms_")}
            if errs is not None:
                r["oracle_rel_err_at"] = {str(t): errs[k][v][t] for t in d["checks"]}
            rep[v] = r
        out["k"][str(k)] = rep
    out["how"] = (f"{len(d['rows'])} sampled rows of W and all of beta after the checked "
                  "updates vs the FP64 oracle (Z = X^T X carried exactly, W = inv(Z)); newton: "
                  "correction=\"newton\" (Z = X^T X kept as double-float pairs, "
                  "W <- W + W (I - Z W) and beta <- beta + W (X^T Y - Z beta) after every "
                  "correction_period-th update); times: median CUDA-event interval of an "
                  "update without a correction, of an update that ends in one (Z brought up "
                  "to date with the period's replaced rows, then the step), and of a "
                  "correction alone (no rows pending)")
    return out


def gemm_section(args, reps=3):
    """The library's own GEMM on the workloads' products: the n^3 squaring of
    re-evaluation, dA = [G][T]^T of the adjoint (inner dimension k p = 1024)
    and the n x n x p product of the iteration (p = 64), FP32 in split TF32
    on tcgen05.  Effective TFLOP/s counts 2 M N K; the tensor pipe runs three
    TF32 products per output, so its roofline is 3 x that against the TF32
    peak (the measured dense BF16 peak x 1/2, the nominal TF32 : BF16 ratio).
    cuBLAS TF32 (one product, ~1e-3 relative) and IEEE FP32 are timed beside
    it for context."""
    import torch
    from paper_1403_6968_gb300 import gemm
    peaks = _peaks()
    bf16 = peaks.get("bf16_tflops") if peaks else 1900.0
    tf32_peak = 0.5 * bf16
    n = args.gemm_n
    shapes = [(n, n, n), (n, n, 1024), (n, 64, n)]
    g = torch.Generator(device="cuda").manual_seed(0)
    rows = []
    for (M, N, K) in shapes:
        a = torch.randn(M, K, device="cuda", generator=g)
        b = torch.randn(K, N, device="cuda", generator=g)
        c = torch.empty(M, N, device="cuda")
        gemm(a, b, c)  # warm-up: tensor maps, kernel attributes, the memory pool
        own = _event_ms(lambda j: gemm(a, b, c), reps)
        ref = a.double() @ b.double()
        err = float((c.double() - ref).norm() / ref.norm())
        del ref
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = True
        torch.matmul(a, b, out=c)  # warm-up
        t_tf32 = _event_ms(lambda j: torch.matmul(a, b, out=c), reps)
        torch.backends.cuda.matmul.allow_tf32 = False
        torch.matmul(a, b, out=c)
        t_fp32 = _event_ms(lambda j: torch.matmul(a, b, out=c), reps)
        torch.backends.cuda.matmul.allow_tf32 = prev
        eff = 2.0 * M * N * K / (own / 1e3) / 1e12
        rows.append({"M": M, "N": N, "K": K, "own_ms": own, "own_tflops_effective": eff,
                     "tensor_pipe_tflops": 3 * eff, "tensor_frac_of_tf32_peak": 3 * eff / tf32_peak,
                     "rel_err_vs_fp64": err, "cublas_tf32_ms": t_tf32, "cublas_fp32_ms": t_fp32})
    return {"rows": rows, "tf32_peak_tflops": tf32_peak,
            "peak_source": ("measured bf16 x 0.5" if peaks else "fallback bf16 x 0.5"),
            "note": "own_ms includes splitting both operands into [hi | lo] rows (one pass each)"}


def k_sweep(args, seed=0, steps=8, warmup=2, ks=(2, 4, 8, 16, 32)):
    """Iterative models of A^k (Section 3.3, Appendix A) against k: per-update
    refresh time of the exponential model (views A^(2^j)), the linear model
    (views A^1..A^k) and the skip-4 model (A, A^2, A^4, A^8, A^12, ..) under
    rank-1 row updates, beside the re-evaluation of each (BF16x9 GEMMs)."""
    import numpy as np
    import torch
    import linview_inputs as li
    from paper_1403_6968_gb300 import Program

    n = args.n
    a = torch.from_numpy(li.power_matrix(n, seed=seed, dtype=np.float32)).cuda()
    ups = li.row_update_stream(n, warmup + steps, seed=seed + 7, dtype=np.float32)
    dv = [(i, torch.from_numpy(v).cuda()) for i, v in ups]
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for j in range(reps):
            fn(j)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    rows = []
    for k in ks:
        row = {"k": k}
        for model in ("exp", "linear", "skip4"):
            if model == "skip4" and k < 8:
                continue
            kw = {"model": "skip", "skip": 4} if model == "skip4" else {"model": model}
            prog = Program("power", [a], k=k, r_max=1, **kw)
            for i, v in dv[:warmup]:
                prog.apply_row_delta(i, v)
            row[f"{model}_ms"] = timed(lambda j: prog.apply_row_delta(*dv[warmup + j]), steps)
            row[f"{model}_views"] = prog.num_views()
            prog.set_reeval_mode("tc3")   # the library's own split-TF32 GEMM
            prog.reeval()
            row[f"{model}_reeval_ms"] = timed(lambda j: prog.reeval(), 2)
            prog.sync()
            prog.close()
        rows.append(row)
    return {"n": n, "update": "rank-1 row", "steps": steps, "rows": rows,
            "note": "per-update refresh of all views of the model; re-evaluation recomputes "
                    "the same views from A"}


def _event_ms(fn, reps):
    import torch
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for j in range(reps):
        fn(j)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def iteration_p_sweep(args, seed=0, k=16, steps=6, ps=(1, 16, 128, 1024), n=None):
    """General form with B = 0 (Section 6, "B=0"): T_{i+1} = A T_i, n = 8192
    (or ``n``), k = 16, against the width p of T: per-update refresh of
    T_1..T_k (rank-1 row updates of A) vs re-evaluation (k products A T_i)."""
    import numpy as np
    import torch
    import linview_inputs as li
    from paper_1403_6968_gb300 import Program

    n = n or args.n
    if n > 16384:  # the paper's size: A and T_0 drawn by a seeded device generator
        gen = torch.Generator(device="cuda").manual_seed(2000 + seed)
        a = torch.randn((n, n), generator=gen, device="cuda") / (2.0 * np.sqrt(n))
    else:
        gen = None
        a = torch.from_numpy(li.power_matrix(n, seed=seed, dtype=np.float32)).cuda()
    ups = [(i, torch.from_numpy(v).cuda())
           for i, v in li.row_update_stream(n, steps + 2, seed=seed + 3, dtype=np.float32)]
    rows = []
    for p in ps:
        if gen is not None:
            t0 = torch.randn((n, p), generator=gen, device="cuda")
        else:
            t0 = torch.from_numpy(li.normal((n, p), seed=seed + p, dtype=np.float32)).cuda()
        b = torch.zeros((n, p), dtype=torch.float32, device="cuda")
        prog = Program("iteration", [a, b, t0], k=k, r_max=1)
        for i, v in ups[:2]:
            prog.apply_row_delta(i, v)
        inc = _event_ms(lambda j: prog.apply_row_delta(*ups[2 + j]), steps)
        row = {"p": p, "incremental_ms": inc}
        for mode in ("tc3", "bf16x9", "tf32"):
            prog.set_reeval_mode(mode)
            prog.reeval()
            row[f"reeval_{mode}_ms"] = _event_ms(lambda j: prog.reeval(), 2)
        prog.sync()
        prog.close()
        # hybrid strategy (dense dT_i, one n x n x p product with A per step)
        hyb = Program("iteration", [a, b, t0], k=k, r_max=1, strategy="hybrid")
        for i, v in ups[:2]:
            hyb.apply_row_delta(i, v)
        row["hybrid_ms"] = _event_ms(lambda j: hyb.apply_row_delta(*ups[2 + j]), steps)
        hyb.sync()
        hyb.close()
        # exponential model (views T_1, T_2, T_4, .., T_k) and skip-4 model (T_1,
        # T_2, T_4, T_8, T_12, T_16), with their auxiliary P_h, S'_h views
        for key, kw in (("exp_model_ms", {"model": "exp"}),
                        ("skip4_model_ms", {"model": "skip", "skip": 4})):
            ex = Program("iteration", [a, b, t0], k=k, r_max=1, **kw)
            for i, v in ups[:2]:
                ex.apply_row_delta(i, v)
            row[key] = _event_ms(lambda j: ex.apply_row_delta(*ups[2 + j]), steps)
            ex.sync()
            ex.close()
        rows.append(row)
    return {"n": n, "k": k, "B": "0", "update": "rank-1 row of A", "steps": steps, "rows": rows,
            "note": "incremental = factored deltas, linear model (Krylov reuse); hybrid = "
                    "dense deltas D_i = A D_{i-1} + rank-1 term; exp_model / skip4_model = "
                    "factored deltas, exponential / skip-4 model (views T_1, T_2, T_4, .., T_k "
                    "/ T_1, T_2, T_4, T_8, T_12, T_16, with P_h and S'_h views); "
                    "re-evaluation = k products A T_i"}


def gd_regression_device(seed=0, n=30000, m=30000, p=1000, k=16, steps=3):
    """The gradient-descent workload of gd_regression at the paper's size
    (Section 6: n = 30K, p = 1000, k = 16), built on the device: X (m x n) and
    Y (m x p) ~ N(0, 1) from a seeded device generator, X^T X and X^T Y on the
    library's own GEMM (split TF32), lambda_max by power iteration, A = I -
    eta X^T X, B = eta X^T Y.  Incremental row replacements (rank-2 dA, rank-1
    dB) in the linear, exponential and skip-4 models against re-evaluating the
    k iterations (own GEMM, cuBLAS BF16x9 and TF32)."""
    import torch
    from paper_1403_6968_gb300 import Program, gemm

    gen = torch.Generator(device="cuda").manual_seed(1000 + seed)
    t_set = time.perf_counter()
    x = torch.randn((m, n), generator=gen, device="cuda")
    y = torch.randn((m, p), generator=gen, device="cuda")
    g = torch.empty((n, n), device="cuda")
    gemm(x, x, g, ta=True)                     # X^T X, own GEMM
    xty = torch.empty((n, p), device="cuda")
    gemm(x, y, xty, ta=True)                   # X^T Y
    z = torch.randn((n, 1), generator=gen, device="cuda")
    for _ in range(30):                        # lambda_max by power iteration
        z = g @ z
        z /= z.norm()
    eta = 1.0 / (1.05 * float((z.T @ (g @ z)).item()))
    a = -eta * g
    a.diagonal().add_(1.0)
    del g
    b = eta * xty
    del xty
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_set
    newx = torch.randn((steps + 2, n), generator=gen, device="cuda")
    rowsel = torch.randint(0, m, (steps + 2,), generator=gen, device="cuda").tolist()
    deltas = []
    for j in range(steps + 2):
        i = int(rowsel[j])
        xo, xn = x[i].clone(), newx[j]
        x[i] = xn
        u = torch.stack([xn, xo], dim=1).contiguous()
        v = torch.stack([-eta * xn, eta * xo], dim=1).contiguous()
        ub = (xn - xo).reshape(n, 1).contiguous()
        vb = (eta * y[i]).reshape(p, 1).contiguous()
        deltas.append((u, v, ub, vb))
    del x
    out = {"n": n, "m": m, "p": p, "k": k, "eta": eta, "setup_s": setup_s,
           "inputs": "X, Y ~ N(0,1) from a seeded device generator; X^T X, X^T Y on the own GEMM"}
    for key, kw in (("linear", {"model": "linear"}), ("exp_model", {"model": "exp"}),
                    ("skip4_model", {"model": "skip", "skip": 4})):
        prog = Program("iteration", [a, b, torch.zeros((n, p), device="cuda")], k=k, r_max=2,
                       **kw)

        def replace_row(j):
            u, v, ub, vb = deltas[j]
            prog.apply_delta(u, v)
            prog.apply_delta(ub, vb, input_id=1)

        replace_row(0)
        replace_row(1)
        out[f"{key}_ms_per_row_replacement"] = _event_ms(lambda j: replace_row(2 + j), steps)
        if key == "linear":
            for mode in ("tc3", "bf16x9", "tf32"):
                prog.set_reeval_mode(mode)
                prog.reeval()
                out[f"reeval_{mode}_ms"] = _event_ms(lambda j: prog.reeval(), 1)
        prog.sync()
        prog.close()
    best = min(out[f"{m_}_ms_per_row_replacement"] for m_ in ("linear", "exp_model", "skip4_model"))
    out["speedup_best_model_vs_own_reeval"] = out["reeval_tc3_ms"] / best
    out["speedup_best_model_vs_bf16x9_reeval"] = out["reeval_bf16x9_ms"] / best
    out["note"] = ("per row replacement of X: the rank-2 dA and rank-1 dB; re-evaluation: "
                   "T_i = A T_{i-1} + B for i = 1..k")
    return out


def gd_regression(seed=0, n=4096, m=4096, p=1024, k=16, steps=6):
    """Batch gradient descent for least squares as the general form (Section
    6, "B != 0"): Theta_{i+1} = Theta_i - eta X^T (X Theta_i - Y), i.e.
    A = I - eta X^T X, B = eta X^T Y, Theta_0 = 0.  An update replaces one row
    of X: dA = -eta (x' x'^T - x x^T) (rank 2) and dB = eta (x' - x) y^T
    (rank 1), applied as two factored deltas; compared with re-evaluating the
    k iterations.  X, Y ~ N(0, 1); eta = 1 / (1.05 lambda_max(X^T X))."""
    import numpy as np
    import torch
    import linview_inputs as li
    from paper_1403_6968_gb300 import Program

    x = li.normal((m, n), seed=seed + 11)
    y = li.normal((m, p), seed=seed + 12)
    t_host = time.perf_counter()
    g = x.T @ x                                   # workload construction on the host
    z = li.normal((n, 1), seed=seed + 13)
    for _ in range(30):                           # lambda_max by power iteration
        z = g @ z
        z /= np.linalg.norm(z)
    eta = 1.0 / (1.05 * (z.T @ g @ z).item())
    a = (np.eye(n) - eta * g).astype(np.float32)
    b = (eta * (x.T @ y)).astype(np.float32)
    host_s = time.perf_counter() - t_host
    prog = Program("iteration", [torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(),
                                 torch.zeros((n, p), dtype=torch.float32, device="cuda")],
                   k=k, r_max=2)
    newx = li.normal((steps + 2, n), seed=seed + 14)
    rowsel = np.random.default_rng(seed + 15).integers(0, m, size=steps + 2)
    deltas = []
    for j in range(steps + 2):
        i = int(rowsel[j])
        xo, xn = x[i].copy(), newx[j]
        x[i] = xn
        u = np.stack([xn, xo], axis=1).astype(np.float32)
        v = np.stack([-eta * xn, eta * xo], axis=1).astype(np.float32)
        ub = (xn - xo).reshape(n, 1).astype(np.float32)
        vb = (eta * y[i]).reshape(p, 1).astype(np.float32)
        deltas.append(tuple(torch.from_numpy(t).cuda() for t in (u, v, ub, vb)))

    def replace_row(j):
        u, v, ub, vb = deltas[j]
        prog.apply_delta(u, v)
        prog.apply_delta(ub, vb, input_id=1)

    replace_row(0)
    replace_row(1)
    inc = _event_ms(lambda j: replace_row(2 + j), steps)
    out = {"n": n, "m": m, "p": p, "k": k, "eta": eta, "incremental_ms_per_row_replacement": inc,
           "host_setup_s": host_s}
    for mode in ("tc3", "bf16x9", "tf32", "fp32"):
        prog.set_reeval_mode(mode)
        prog.reeval()
        out[f"reeval_{mode}_ms"] = _event_ms(lambda j: prog.reeval(), 2)
    prog.sync()
    prog.close()
    # the same row replacements in the exponential and skip-4 models (views
    # T_1, T_2, T_4, .., T_16 / T_1, T_2, T_4, T_8, T_12, T_16; Section 6's
    # comparison of the iterative models), each on its own program
    a_dev, b_dev = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    for key, kw in (("exp_model", {"model": "exp"}),
                    ("skip4_model", {"model": "skip", "skip": 4})):
        prog = Program("iteration", [a_dev, b_dev,
                                     torch.zeros((n, p), dtype=torch.float32, device="cuda")],
                       k=k, r_max=2, **kw)
        replace_row(0)
        replace_row(1)
        out[f"{key}_ms_per_row_replacement"] = _event_ms(lambda j: replace_row(2 + j), steps)
        prog.sync()
        prog.close()
    out["speedup_vs_bf16x9_reeval"] = out["reeval_bf16x9_ms"] / inc
    out["note"] = ("incremental: the rank-2 dA and rank-1 dB of a row replacement; "
                   "re-evaluation: T_i = A T_{i-1} + B for i = 1..k")
    return out


def small_fp64(seed=0, n=256, k=8, steps=20):
    """The small FP64 case: A^8 (views A, A^2, A^4, A^8), n = 256, rank-1 row
    updates; everything is L2-resident, so this is latency (launches and
    dependent small kernels), reported per refresh."""
    import numpy as np
    import torch
    import linview_inputs as li
    from paper_1403_6968_gb300 import Program

    a = li.power_matrix(n, seed=seed, dtype=np.float64)
    prog = Program("power", [torch.from_numpy(a).cuda()], k=k, precision="f64")
    ups = [(i, torch.from_numpy(v).cuda())
           for i, v in li.row_update_stream(n, steps + 3, seed=seed + 1, dtype=np.float64)]
    for i, v in ups[:3]:
        prog.apply_row_delta(i, v)
    stream = torch.cuda.current_stream()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    torch.cuda.synchronize()
    evs[0].record(stream)
    for t in range(steps):
        prog.apply_row_delta(*ups[3 + t])
        evs[t + 1].record(stream)
    torch.cuda.synchronize()
    lat = [evs[t].elapsed_time(evs[t + 1]) * 1e3 for t in range(steps)]
    prog.close()
    return {"n": n, "k": k, "precision": "f64", "p50_us": float(np.median(lat)),
            "p99_us": float(np.percentile(lat, 99)), "steps": steps}


def iteration_adjoint(seed=0, n=8192, p=64, k=16, r=2, steps=6):
    """The differentiation workload: T_i = A T_{i-1} + B, n = 8192, p = 64,
    k = 16, rank-2 updates of A (U, V ~ N(0, 0.01^2)): the incremental
    refresh of T_1..T_16, the re-evaluation, and the adjoint of
    L = ||T_16||_F^2 (dL/dA and dL/dB: 15 products A^T G and one
    n x n x k p GEMM)."""
    import numpy as np
    import torch
    import linview_inputs as li
    from paper_1403_6968_gb300 import Program

    a, b, t0 = li.iteration_inputs(n, p, seed=seed, dtype=np.float32)
    prog = Program("iteration", [torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(),
                                 torch.from_numpy(t0).cuda()], k=k, r_max=r)
    ups = [tuple(torch.from_numpy(x).cuda() for x in uv)
           for uv in li.lowrank_update_stream(n, r, steps + 2, seed=seed + 1, dtype=np.float32)]
    for u, v in ups[:2]:
        prog.apply_delta(u, v)
    inc = _event_ms(lambda j: prog.apply_delta(*ups[2 + j]), steps)
    dA = torch.empty((n, n), dtype=torch.float32, device="cuda")
    dB = torch.empty((n, p), dtype=torch.float32, device="cuda")
    prog.adjoint_iteration(dA, dB)
    adj = _event_ms(lambda j: prog.adjoint_iteration(dA, dB), 3)
    out = {"n": n, "p": p, "k": k, "rank": r, "incremental_ms": inc, "adjoint_ms": adj}
    for mode in ("tc3", "bf16x9", "tf32", "fp32"):
        prog.set_reeval_mode(mode)
        prog.reeval()
        out[f"reeval_{mode}_ms"] = _event_ms(lambda j: prog.reeval(), 2)
    prog.sync()
    prog.close()
    out["note"] = ("incremental: rank-2 dA, linear model with Krylov reuse (15 products of A "
                   "with the newest 2 columns); adjoint: dL/dA and dL/dB of ||T_16||_F^2")
    return out


def ols_sweep(seed=0, m=65536, n=4096, p=16, ks=(1, 4, 16), steps=6):
    """OLS (Section 4.1) at m = 65536, n = 4096, p = 16: X ~ N(0, 1) with a
    fixed 10% of its columns scaled by 1e-2 (kappa(X^T X) ~ 3e4), Y ~ N(0, 1);
    an update replaces k rows of X by fresh rows with the same scaling.  Per
    k: the incremental refresh of W = (X^T X)^-1 and beta (block Woodbury,
    FP32 views, double-float 2k x 2k core) against the re-evaluation (FP64
    X^T X by row chunks, Cholesky inverse)."""
    import numpy as np
    import torch
    import linview_inputs as li
    from paper_1403_6968_gb300 import Program

    x, y, _ = li.ols_inputs(m, n, p, seed=seed, dtype=np.float32)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    rows = []
    for k in ks:
        prog = Program("ols", [xd, yd], k=k)
        ups = li.ols_row_replacements(m, n, k, steps + 2, seed=seed + k, dtype=np.float32,
                                      cols_seed=seed)
        dev = [(r_, torch.from_numpy(nw).cuda()) for r_, nw in ups]
        for r_, nw in dev[:2]:
            prog.apply_row_block(r_, nw)
        inc = _event_ms(lambda j: prog.apply_row_block(*dev[2 + j]), steps)
        prog.sync()
        w_inc, b_inc = prog.read_view_host(0), prog.read_view_host(1)
        prog.reeval()
        re = _event_ms(lambda j: prog.reeval(), 1)
        prog.sync()
        w_re, b_re = prog.read_view_host(0), prog.read_view_host(1)
        prog.close()
        errs = {name: float(np.linalg.norm((a.astype(np.float64) - b.astype(np.float64)).ravel())
                            / np.linalg.norm(b.astype(np.float64).ravel()))
                for name, a, b in (("W", w_inc, w_re), ("beta", b_inc, b_re))}
        # W read twice and written once (two passes), 4 bytes per entry
        gbs = 3.0 * n * n * 4 / (inc / 1e3) / 1e9
        rows.append({"k": k, "incremental_ms": inc, "reeval_fp64_ms": re,
                     "speedup": re / inc, "w_pass_gbs": gbs,
                     "rel_err_vs_reeval": errs})
    return {"m": m, "n": n, "p": p, "rows": rows,
            "note": "incremental: block Woodbury on W (FP32, two passes: G = W^T U by column "
                    "sums, W += G Wu^T) with a double-float 2k x 2k core (Newton-Schulz, "
                    "Gauss-Jordan fallback) and the factored beta refresh (no pass over W); "
                    "re-evaluation: FP64 "
                    "X^T X, Cholesky inverse, beta = W X^T Y; rel_err_vs_reeval: the views after "
                    f"{steps + 2} updates against the re-evaluation that follows them"}


def serving_sweep(args, seed=0):
    """Serving workload: resident A^16 views with n uniform in
    {1024, 2048, 4096, 8192}; for each rate an open-loop Poisson trace of
    rank-1..8 updates (target view uniform) replayed through the server;
    latency = completion - arrival per request."""
    import numpy as np
    import torch
    import linview_inputs as li
    from paper_1403_6968_gb300 import Server

    sizes = li.serving_views(args.serve_views, seed=seed)
    srv = Server(max_inflight=args.serve_inflight, r_cap=8)
    t0 = time.perf_counter()
    for i, n in enumerate(sizes):
        srv.add_view(torch.from_numpy(li.power_matrix(n, seed=100 + i, dtype=np.float32)).cuda(),
                     16)
    setup_s = time.perf_counter() - t0
    st0 = srv.stats()
    sweep = []
    for j, rate in enumerate(float(x) for x in args.serve_rates.split(",")):
        count = int(max(50, min(2000, rate * 0.5)))
        t_s, views, ranks, factors, offsets = li.serving_trace(sizes, count, rate, seed=seed + j)
        before = srv.stats()
        srv.replay(t_s, views, ranks, factors, offsets)
        srv.drain(timeout_s=300)
        recs = srv.poll()
        after = srv.stats()
        lat = np.array([r["done_s"] - r["arrival_s"] for r in recs]) * 1e3
        span = max(r["done_s"] for r in recs) - min(r["arrival_s"] for r in recs)
        nref = after["refreshes"] - before["refreshes"]
        sweep.append({
            "rate_per_s": rate, "requests": count,
            "failed": after["failed"] - before["failed"],
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "requests_per_s": count / span, "refreshes": nref,
            "mean_coalesced_rank": (after["coalesced_rank_sum"] - before["coalesced_rank_sum"])
            / max(nref, 1),
            "mean_request_rank": float(ranks.mean()),
            "max_inflight_seen": after["max_inflight_seen"],
            "_recs": recs, "_span": span})
    srv.close()
    # what a refresh of each view size costs alone, per coalesced rank, and
    # hence how the GPU time of each sweep point splits over the view sizes
    cost = serving_view_costs(sorted(set(sizes)), seed=seed)
    for pt in sweep:
        recs, span = pt.pop("_recs"), pt.pop("_span")
        seen = {}
        for rc in recs:  # one refresh per (view, issue time)
            seen[(rc["view"], rc["start_s"])] = rc["batch_rank"]
        busy = {}
        for (v, _), r in seen.items():
            nv = sizes[v]
            busy[nv] = busy.get(nv, 0.0) + cost[str(nv)][str(min(max(int(r), 1), 8))]
        pt["gpu_busy_share_by_n"] = {str(nv): busy[nv] / 1e3 / span for nv in sorted(busy)}
    return {"views": len(sizes), "n_counts": {str(n): sizes.count(n) for n in sorted(set(sizes))},
            "k": 16, "resident_bytes": st0["bytes_used"], "setup_s": setup_s,
            "max_inflight": args.serve_inflight, "r_cap": 8, "sweep": sweep,
            "refresh_ms_alone": cost,
            "note": "open-loop Poisson arrivals replayed by the library; queued requests to a "
                    "busy view coalesce up to rank 8; latency = completion seen by the "
                    "scheduler - arrival; refresh_ms_alone: one refresh of an A^16 view of "
                    "each size per coalesced rank, timed alone (CUDA events); "
                    "gpu_busy_share_by_n: the sum of those costs over a sweep point's "
                    "refreshes, per view size, divided by the point's wall time"}


def serving_inflight(args, seed=0, rate=1e5, count=2000, levels=(4, 8, 16, 32)):
    """The serving workload past saturation (one open-loop trace at ``rate``)
    for several bounds on the number of views refreshing at once: a server of
    the same views per bound, the same trace replayed through each."""
    import numpy as np
    import torch
    import linview_inputs as li
    from paper_1403_6968_gb300 import Server

    sizes = li.serving_views(args.serve_views, seed=seed)
    mats = [li.power_matrix(n, seed=100 + i, dtype=np.float32) for i, n in enumerate(sizes)]
    t_s, views, ranks, factors, offsets = li.serving_trace(sizes, count, rate, seed=seed + 7)
    rows = []
    for m in levels:
        srv = Server(max_inflight=m, r_cap=8)
        for a in mats:
            srv.add_view(torch.from_numpy(a).cuda(), 16)
        before = srv.stats()
        srv.replay(t_s, views, ranks, factors, offsets)
        srv.drain(timeout_s=300)
        recs = srv.poll()
        after = srv.stats()
        srv.close()
        torch.cuda.empty_cache()
        lat = np.array([r["done_s"] - r["arrival_s"] for r in recs]) * 1e3
        span = max(r["done_s"] for r in recs) - min(r["arrival_s"] for r in recs)
        nref = after["refreshes"] - before["refreshes"]
        rows.append({"max_inflight": m, "requests_per_s": count / span,
                     "p50_ms": float(np.percentile(lat, 50)),
                     "p99_ms": float(np.percentile(lat, 99)), "refreshes": nref,
                     "mean_coalesced_rank": (after["coalesced_rank_sum"]
                                             - before["coalesced_rank_sum"]) / max(nref, 1),
                     "max_inflight_seen": after["max_inflight_seen"],
                     "failed": after["failed"] - before["failed"]})
    return {"views": len(sizes), "rate_per_s": rate, "requests": count, "r_cap": 8,
            "rows": rows,
            "note": "the same open-loop trace past saturation replayed through a server per "
                    "bound on the views refreshing at once (each view on its own stream)"}


def serving_view_costs(ns, seed=0, reps=5):
    """ms of one refresh of an A^16 view (the server's program: power, k = 16,
    r_max = 8) per view size and delta rank 1..8, each timed alone."""
    import numpy as np
    import torch
    import linview_inputs as li
    from paper_1403_6968_gb300 import Program

    out = {}
    for n in ns:
        prog = Program("power", [torch.from_numpy(li.power_matrix(n, seed=seed, dtype=np.float32))
                                 .cuda()], k=16, r_max=8)
        ups = li.lowrank_update_stream(n, 8, 1, seed=seed + 1, dtype=np.float32)[0]
        u8, v8 = torch.from_numpy(ups[0]).cuda(), torch.from_numpy(ups[1]).cuda()
        row = {}
        for r in range(1, 9):
            u, v = u8[:, :r].contiguous(), v8[:, :r].contiguous()
            for _ in range(2):
                prog.apply_delta(u, v)
            row[str(r)] = _event_ms(lambda j: prog.apply_delta(u, v), reps)
        out[str(n)] = row
        prog.close()
    return out


def zipf_batches(args, seed=0, count=1000):
    """Batch updates (Section 6, Table 4): a batch of ``count`` row updates
    with Zipf-distributed rows arrives at once for one A^16 view; the server
    merges repeated rows and splits the batch into deltas of rank <= 8.
    Reported beside the re-evaluation of the view after the whole batch."""
    import numpy as np
    import torch
    import linview_inputs as li
    from paper_1403_6968_gb300 import Server

    n, k = args.n, 16
    srv = Server(max_inflight=1, r_cap=8)
    v = srv.add_view(torch.from_numpy(li.power_matrix(n, seed=seed, dtype=np.float32)).cuda(), k)
    out = []
    for j, z in enumerate((5.0, 4.0, 3.0, 2.0, 1.0, 0.0)):
        rows, vs = li.zipf_row_batch(n, count, z, seed=seed + j)
        before = srv.stats()
        srv.replay(np.zeros(count), np.zeros(count, np.int32), np.ones(count, np.int32),
                   np.ascontiguousarray(vs.reshape(-1)), np.arange(count) * n, rows=rows)
        srv.drain(timeout_s=600)
        recs = srv.poll()
        after = srv.stats()
        span = max(r["done_s"] for r in recs) - min(r["arrival_s"] for r in recs)
        out.append({"zipf": z, "distinct_rows": int(len(np.unique(rows))),
                    "refreshes": after["refreshes"] - before["refreshes"],
                    "batch_ms": span * 1e3, "failed": after["failed"] - before["failed"]})
    prog = srv.program(v)
    reeval = {}
    for mode in ("tc3", "bf16x9", "fp32"):
        prog.set_reeval_mode(mode)
        prog.reeval()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            prog.reeval()
        e1.record()
        torch.cuda.synchronize()
        reeval[mode] = e0.elapsed_time(e1) / 3
    srv.close()
    return {"n": n, "k": k, "batch": count, "r_cap": 8, "sweep": out,
            "reeval_ms_after_batch": reeval,
            "note": "batch_ms = arrival of the batch to completion of its last delta; "
                    "re-evaluation = the 4 squarings of A^16 after applying the batch to A"}


def _apply_to_a(aptr, ald, n, u, v):
    """A += u v^T through the library's stand-alone level pass (update only)."""
    import ctypes as C
    from paper_1403_6968_gb300 import _lib as L
    from paper_1403_6968_gb300.linview import _stream_ptr
    L.call("linview_level_pass", L.F32, n, C.c_void_p(aptr), ald, C.c_void_p(u.data_ptr()),
           C.c_void_p(v.data_ptr()), n, 1, None, None, 1, _stream_ptr())


def _drift_a(args, seed=0):
    import numpy as np
    import linview_inputs as li
    return li.power_matrix(args.n, seed=seed, dtype=np.float32)


def run_only(args):
    """One secondary section alone on GPU 0, its result as one JSON line."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__ as g
    g.build()
    fns = {"rank4_stream": lambda: rank_stream(args, 4),
           "k_sweep": lambda: k_sweep(args),
           "iteration_p_sweep": lambda: iteration_p_sweep(args),
           "gd_regression": lambda: gd_regression(),
           "small_fp64": lambda: small_fp64(),
           "ols_row_blocks": lambda: ols_sweep(),
           "iteration_adjoint": lambda: iteration_adjoint(),
           "serving": lambda: serving_sweep(args),
           "serving_inflight": lambda: serving_inflight(args),
           "zipf_batches": lambda: zipf_batches(args),
           "gemm": lambda: gemm_section(args),
           "iteration_p_sweep_n30000": lambda: iteration_p_sweep(args, steps=3, n=30000),
           "gd_regression_n30000": lambda: gd_regression_device(),
           "drift": lambda: drift_report(drift_streams(args), _drift_a(args), args.k,
                                         not args.no_cpu_baseline),
           "ols_drift": lambda: ols_drift_report(ols_drift_streams(), not args.no_cpu_baseline)}
    print(json.dumps({"section": args.only, args.only: fns[args.only]()}), flush=True)
    return 0


def main():
    args = _args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        return run_only(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
