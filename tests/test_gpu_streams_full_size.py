"""GPU parity over whole update streams at the workloads' own sizes.

* Powers + sums of powers (A^16 and S' = sum_{i<=16} A^i, n = 8192, FP32): the
  200-update rank-1 row stream in the bench's program configuration (r_max 1),
  and the 200-update rank-4 stream (r_max 4); every 10th update (and after the
  first) sampled rows of all 9 views -- 16 fixed rows plus every row updated
  since the previous check -- against the FP64 oracle on the current A,
  computed row by row from the plain definition.  Drift that builds up over
  the stream shows here: the bound is the FP32 one, 1e-4 relative Frobenius,
  after every checked update.
* The general form T_i = A T_{i-1} + B at n = 8192, p = 64, k = 16 with rank-2
  updates (linear and exponential models): every view T_1 .. T_16 in full
  against the oracle's re-evaluation after updates 1, 3 and 6.

The oracle holds A in FP64 (the FP32-rounded inputs promoted, so the metric
measures the method's error, not input rounding).
"""
import numpy as np
import pytest

import linview_inputs as li
from oracle import iteration as oi
from oracle import powers as op
from oracle.metrics import rel_frob

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4
N, K, L = 8192, 16, 4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _prog(*a, **kw):
    from paper_1403_6968_gb300 import Program
    return Program(*a, **kw)


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _view_rows(prog, vid, rows):
    out = np.empty((len(rows), N), dtype=np.float32)
    for j, i in enumerate(rows):
        prog.read_view_rows(vid, int(i), 1, out=out[j:j + 1])
    return out


def _check_rows(prog, rows, pr, sr, where):
    errs = {}
    for j in range(L + 1):
        errs[f"P{1 << j}"] = rel_frob(_view_rows(prog, j, rows), pr[1 << j])
    for j in range(1, L + 1):
        errs[f"S{1 << j}"] = rel_frob(_view_rows(prog, L + j, rows), sr[1 << j])
    assert max(errs.values()) <= TOL, (where, errs)
    return max(errs.values())


def _fixed_rows(seed):
    g = np.random.default_rng(seed)
    return sorted({0, N - 1} | set(int(i) for i in g.choice(N, 14, replace=False)))


def test_config1_rank1_row_stream_200_updates():
    a = li.power_matrix(N, seed=0, dtype=np.float32)
    prog = _prog("power_sum", [_dev(a)], k=K, r_max=1)
    a64 = a.astype(np.float64)
    fixed = _fixed_rows(100)
    recent = set()
    checks = {1} | set(range(10, 201, 10))
    worst = 0.0
    for t, (i, v) in enumerate(li.row_update_stream(N, 200, seed=0, dtype=np.float32), 1):
        prog.apply_row_delta(int(i), _dev(v))
        a64[i] += v.astype(np.float64)
        recent.add(int(i))
        if t in checks:
            prog.sync()
            rows = sorted(set(fixed) | recent)
            assert len(rows) >= 16
            pr, sr = op.power_rows(a64, rows, K)
            worst = max(worst, _check_rows(prog, rows, pr, sr, t))
            recent = set()
    prog.close()
    print(f"rank-1 stream: worst sampled-row error over 21 checks {worst:.2e}")


def test_config1_rank4_stream_200_updates():
    a = li.power_matrix(N, seed=0, dtype=np.float32)
    prog = _prog("power_sum", [_dev(a)], k=K, r_max=4)
    a0 = a.astype(np.float64)
    ups = li.lowrank_update_stream(N, 4, 200, seed=0, dtype=np.float32)
    uall = np.zeros((N, 4 * len(ups)))
    vall = np.zeros((N, 4 * len(ups)))
    fixed = _fixed_rows(101)
    g = np.random.default_rng(102)
    checks = {1} | set(range(10, 201, 10))
    worst = 0.0
    for t, (u, v) in enumerate(ups, 1):
        prog.apply_delta(_dev(u), _dev(v))
        uall[:, 4 * (t - 1):4 * t] = u
        vall[:, 4 * (t - 1):4 * t] = v
        if t in checks:
            prog.sync()
            # every row changes under a dense rank-4 update: fresh rows each check
            rows = sorted(set(fixed) | set(int(i) for i in g.choice(N, 8, replace=False)))
            pr, sr = op.power_rows_factored(a0, uall[:, :4 * t], vall[:, :4 * t], rows, K)
            worst = max(worst, _check_rows(prog, rows, pr, sr, t))
    prog.close()
    print(f"rank-4 stream: worst sampled-row error over 21 checks {worst:.2e}")


@pytest.mark.parametrize("model", ["linear", "exp"])
def test_config3_iteration_n8192_p64_rank2(model):
    n, p, k = N, 64, 16
    a, b, t0 = li.iteration_inputs(n, p, seed=0, dtype=np.float32)
    prog = _prog("iteration", [_dev(a), _dev(b), _dev(t0)], k=k, r_max=2, p=p, model=model)
    a64 = a.astype(np.float64)
    b64, t064 = b.astype(np.float64), t0.astype(np.float64)
    # view ids of T_1 .. T_k (linear) or T_1, T_2, T_4, .., T_k (exponential)
    if model == "linear":
        tviews = {i: i for i in range(1, k + 1)}
    else:
        tviews = {1 << j: 1 + j for j in range(k.bit_length())}
    for t, (u, v) in enumerate(li.lowrank_update_stream(n, 2, 6, seed=3, dtype=np.float32), 1):
        prog.apply_delta(_dev(u), _dev(v))
        a64 += u.astype(np.float64) @ v.astype(np.float64).T
        if t in (1, 3, 6):
            prog.sync()
            ts = oi.reeval(a64, b64, t064, k)
            errs = {i: rel_frob(prog.read_view_host(vid), ts[i]) for i, vid in tviews.items()}
            assert max(errs.values()) <= TOL, (model, t, errs)
    prog.close()
