"""GPU parity: matrix powers and sums of powers through the C ABI vs the FP64 oracle.

Tolerances: FP64 programs 1e-10 relative Frobenius (the benchmark spec's bound);
FP32 programs 1e-4 (spec bound for reduced-precision forms; a missing or
mis-signed delta term gives errors of the size of the delta, >= 1e-3 here).
"""
import numpy as np
import pytest

import linview_inputs as li
from oracle import powers as op
from oracle.metrics import rel_frob

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-10, "f32": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _prog(*a, **kw):
    from paper_1403_6968_gb300 import Program
    return Program(*a, **kw)


def _np(prec):
    return np.float64 if prec == "f64" else np.float32


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _check_all(prog, acur, k, sums, tol):
    pw = op.reeval_powers(acur, k)
    sm = op.reeval_sums(acur, k, pw) if sums else None
    L = len(op.levels(k)) - 1
    errs = []
    for j in range(L + 1):
        errs.append(rel_frob(prog.read_view_host(j), pw[1 << j]))
    if sums:
        for j in range(1, L + 1):
            errs.append(rel_frob(prog.read_view_host(L + j), sm[1 << j]))
    assert max(errs) <= tol, errs
    return max(errs)


def test_config0_fp64_a8_row_updates():
    """A^8 by 3 squarings, n=256, FP64, 10 row updates e_i v^T (i uniform,
    v ~ N(0, 0.01^2)); every view vs FP64 re-evaluation after every update."""
    n, k = 256, 8
    a = li.power_matrix(n, seed=0)
    prog = _prog("power", [_dev(a)], k=k, r_max=1, precision="f64")
    acur = a.copy()
    _check_all(prog, acur, k, False, 1e-12)
    for i, v in li.row_update_stream(n, 10, seed=0):
        prog.apply_row_delta(i, _dev(v))
        acur[i] += v
        prog.sync()
        _check_all(prog, acur, k, False, TOL["f64"])


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n,k,r,sums", [
    (1, 1, 1, False), (7, 2, 1, True), (100, 16, 1, True), (513, 4, 3, True),
    (1000, 8, 2, False), (1500, 16, 8, True), (777, 16, 4, True), (2049, 2, 5, True)])
def test_ragged_sizes_and_ranks(prec, n, k, r, sums):
    dt = _np(prec)
    a = li.power_matrix(n, seed=n, dtype=dt)
    prog = _prog("power_sum" if sums else "power", [_dev(a)], k=k, r_max=r, precision=prec)
    acur = a.astype(np.float64)
    for t, (u, v) in enumerate(li.lowrank_update_stream(n, r, 3, seed=n + 1, dtype=dt)):
        prog.apply_delta(_dev(u), _dev(v))
        acur += u.astype(np.float64) @ v.astype(np.float64).T
    # plus a row update at the last row
    (_, v), = li.row_update_stream(n, 1, seed=n + 2, dtype=dt)
    prog.apply_row_delta(n - 1, _dev(v))
    acur[n - 1] += v.astype(np.float64)
    prog.sync()
    _check_all(prog, acur, k, sums, TOL[prec])


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_matches_oracle_incremental(prec):
    n, k, r = 600, 16, 2
    dt = _np(prec)
    a = li.power_matrix(n, seed=3, dtype=dt)
    prog = _prog("power_sum", [_dev(a)], k=k, r_max=r, precision=prec)
    inc = op.IncrementalPowers(a.astype(np.float64), k, sums=True)
    for u, v in li.lowrank_update_stream(n, r, 4, seed=4, dtype=dt):
        prog.apply_delta(_dev(u), _dev(v))
        inc.apply(u.astype(np.float64), v.astype(np.float64))
    prog.sync()
    L = 4
    for j in range(L + 1):
        assert rel_frob(prog.read_view_host(j), inc.p[1 << j]) <= TOL[prec]
    for j in range(1, L + 1):
        assert rel_frob(prog.read_view_host(L + j), inc.s[1 << j]) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n,r,upd", [(1, 1, True), (5, 3, True), (300, 8, True), (1000, 8, False),
                                     (1031, 16, True), (2048, 64, True), (640, 24, False),
                                     (777, 1, True), (1029, 2, True), (1030, 4, True),
                                     (1032, 16, True), (1036, 2, True), (300, 40, True),
                                     (301, 48, True)])
def test_level_pass_kernel(prec, n, r, upd):
    """One Appendix-A level pass (P U, P^T V, P += U V^T) on caller memory."""
    from paper_1403_6968_gb300 import level_pass
    if prec == "f64" and r > 32:
        pytest.skip("FP64 level pass takes r <= 32")
    dt = _np(prec)
    g = np.random.default_rng(n * 100 + r)
    p = g.standard_normal((n, n)).astype(dt)
    u = g.standard_normal((n, r)).astype(dt)
    v = g.standard_normal((n, r)).astype(dt)
    ld = ((n + 3) // 4) * 4
    # a sentinel in the caller's padding: row ends that fall inside a 16-byte
    # unit (n % 4 != 0 in FP32) must not be written past
    P = torch.full((n, ld), 3.0, dtype=torch.float64 if prec == "f64" else torch.float32,
                   device="cuda")
    P[:, :n] = _dev(p)
    Pv = P[:, :n]
    Ut, Vt = _dev(u.T.copy()), _dev(v.T.copy())
    Xt, Yt = torch.empty_like(Ut), torch.empty_like(Ut)
    level_pass(Pv, Ut, Vt, Xt, Yt, do_update=upd)
    torch.cuda.synchronize()
    x_ref, y_ref, p_ref = op.level_products(p, u, v)
    tol = 1e-13 if prec == "f64" else 1e-5
    assert rel_frob(Xt.cpu().numpy().T, x_ref) <= tol
    assert rel_frob(Yt.cpu().numpy().T, y_ref) <= tol
    got_p = Pv.cpu().numpy()
    assert rel_frob(got_p, p_ref if upd else p) <= tol
    assert bool((P[:, n:] == 3.0).all())  # padding untouched


@pytest.mark.parametrize("n,r,upd", [(200, 17, True), (1000, 32, False), (1031, 33, True),
                                     (2048, 48, True), (129, 64, True), (4100, 64, False),
                                     (20, 24, True), (33, 40, False)])
def test_tensor_core_products_pass(n, r, upd):
    """Level passes wider than 16 columns in FP32 with a factor stride that is
    a multiple of 64: X = P U and Y = P^T V run on the tensor cores (split
    TF32, K cut into parts whose partial sums are added afterwards), then
    P += U V^T.  Against the oracle's FP64 products: ragged n (not a multiple
    of 32 or of 128), one and two factor-column blocks (r <= 32, r > 32).
    Bound 2e-6: each product carries ~2^-21 relative error (TF32 split with a
    truncated low part), and the 32-deep tensor-pipe segments are summed in
    FP32 registers, so the error does not grow with n."""
    from paper_1403_6968_gb300 import level_pass
    g = np.random.default_rng(n * 7 + r)
    p = g.standard_normal((n, n)).astype(np.float32)
    u = g.standard_normal((n, r)).astype(np.float32)
    v = g.standard_normal((n, r)).astype(np.float32)
    ld = ((n + 3) // 4) * 4
    ldf = ((n + 63) // 64) * 64
    P = torch.full((n, ld), 3.0, dtype=torch.float32, device="cuda")
    P[:, :n] = _dev(p)
    Pv = P[:, :n]

    def fac(x):
        buf = torch.zeros((r, ldf), dtype=torch.float32, device="cuda")
        if x is not None:
            buf[:, :n] = _dev(x.T.copy())
        return buf[:, :n]

    Ut, Vt, Xt, Yt = fac(u), fac(v), fac(None), fac(None)
    level_pass(Pv, Ut, Vt, Xt, Yt, do_update=upd)
    torch.cuda.synchronize()
    x_ref, y_ref, p_ref = op.level_products(p, u, v)
    assert rel_frob(Xt.cpu().numpy().T, x_ref) <= 2e-6
    assert rel_frob(Yt.cpu().numpy().T, y_ref) <= 2e-6
    assert rel_frob(Pv.cpu().numpy(), p_ref if upd else p) <= 1e-5
    assert bool((P[:, n:] == 3.0).all())


def test_reeval_modes_against_oracle():
    n, k = 1024, 16
    a = li.power_matrix(n, seed=5, dtype=np.float32)
    prog = _prog("power_sum", [_dev(a)], k=k, r_max=1)
    ref_p = op.reeval_powers(a.astype(np.float64), k)
    errs = {}
    # the library's own split-TF32 GEMM first (the default), then the cuBLAS
    # comparison arithmetics.  Own GEMM: <= 4e-7 relative error per product
    # (round-to-nearest split TF32, 32-deep round-toward-zero accumulation
    # segments summed in FP32 registers, independent of K); each of the 4
    # squarings about doubles the relative error it inherits, so A^16 ends
    # below (1 + 2 + 4 + 8) x 4e-7 = 6e-6: bound 1e-5, and at least 20x better
    # than one TF32 product per step
    for mode, tol in (("default", 1e-5), ("tc3", 1e-5), ("fp32", 1e-5), ("bf16x9", 1e-5),
                      ("tf32", 5e-2)):
        prog.set_reeval_mode(mode)
        prog.reeval()
        prog.sync()
        errs[mode] = rel_frob(prog.read_view_host(4), ref_p[16])
        assert errs[mode] <= tol, errs
    assert errs["tc3"] < 5e-2 * errs["tf32"], errs
    ref_s = op.reeval_sums(a.astype(np.float64), k, ref_p)
    prog.set_reeval_mode("default")
    prog.reeval()
    for j in range(1, 5):
        assert rel_frob(prog.read_view_host(4 + j), ref_s[1 << j]) <= 1e-5, j


def test_bitwise_deterministic():
    n, k = 1200, 16
    a = li.power_matrix(n, seed=6, dtype=np.float32)
    ups = li.lowrank_update_stream(n, 2, 3, seed=7, dtype=np.float32)
    outs = []
    for _ in range(2):
        prog = _prog("power_sum", [_dev(a)], k=k, r_max=2)
        for u, v in ups:
            prog.apply_delta(_dev(u), _dev(v))
        prog.sync()
        outs.append([prog.read_view_host(j) for j in range(prog.num_views())])
        prog.close()
    for x, y in zip(*outs):
        assert np.array_equal(x, y)


def test_correction_period_resets_to_reeval():
    n, k = 512, 8
    a = li.power_matrix(n, seed=8, dtype=np.float32)
    prog = _prog("power", [_dev(a)], k=k, r_max=1, correction_period=3)
    acur = a.astype(np.float64)
    for i, v in li.row_update_stream(n, 3, seed=9, dtype=np.float32):
        prog.apply_row_delta(i, _dev(v))
        acur[i] += v
    prog.sync()
    got = [prog.read_view_host(j) for j in range(4)]
    prog.reeval()
    prog.sync()
    for j in range(4):
        assert np.array_equal(got[j], prog.read_view_host(j))  # last update ran re-evaluation
    _check_all(prog, acur, k, False, 1e-5)


def test_host_side_factors_and_errors():
    from paper_1403_6968_gb300 import LinviewError
    n, k = 64, 4
    a = li.power_matrix(n, seed=10, dtype=np.float32)
    prog = _prog("power", [a], k=k, r_max=2)          # host input
    (u, v), = li.lowrank_update_stream(n, 2, 1, seed=11, dtype=np.float32)
    prog.apply_delta(u, v)                             # host factors
    prog.sync()
    acur = a.astype(np.float64) + u.astype(np.float64) @ v.astype(np.float64).T
    _check_all(prog, acur, k, False, 1e-5)
    (u3, v3), = li.lowrank_update_stream(n, 3, 1, seed=12, dtype=np.float32)
    with pytest.raises(LinviewError) as e:
        prog.apply_delta(u3, v3)
    assert e.value.name == "ERANK"
    with pytest.raises(LinviewError) as e:
        prog.apply_row_delta(n, np.zeros(n, np.float32))
    assert e.value.name == "EINVAL"
    with pytest.raises(LinviewError) as e:
        _prog("power", [a], k=3, r_max=1)
    assert e.value.name == "EINVAL"
    _check_all(prog, acur, k, False, 1e-5)             # failed calls changed nothing


@pytest.mark.parametrize("prec,r", [("f32", 1), ("f64", 1), ("f32", 4)])
def test_nonfinite_delta_is_reported(prec, r):
    """A NaN in an update makes a factor core non-finite (at the first level
    whose core involves it: C_2 = V_2^T U_2 carries P^T v); linview_sync
    reports ENONFINITE once, and a program created afterwards is unaffected.
    Rank 1 reaches the cores summed by the assembly (levels of <= 8 columns),
    rank 4 also the stand-alone core reductions (16 and 32 columns)."""
    from paper_1403_6968_gb300 import LinviewError
    n, k = 256, 16
    dt = _np(prec)
    a = li.power_matrix(n, seed=41, dtype=dt)
    prog = _prog("power", [_dev(a)], k=k, r_max=r, precision=prec)
    if r == 1:
        v = np.zeros(n, dt)
        v[7] = np.nan
        prog.apply_row_delta(3, _dev(v))
    else:
        (u, v), = li.lowrank_update_stream(n, r, 1, seed=42, dtype=dt)
        v = v.copy()
        v[5, 2] = np.inf
        prog.apply_delta(_dev(u), _dev(v))
    with pytest.raises(LinviewError) as e:
        prog.sync()
    assert e.value.name == "ENONFINITE"
    prog.sync()  # reported once
    prog.close()
    fresh = _prog("power", [_dev(a)], k=k, r_max=r, precision=prec)
    (i, v), = li.row_update_stream(n, 1, seed=43, dtype=dt)
    fresh.apply_row_delta(i, _dev(v))
    fresh.sync()
    acur = a.astype(np.float64)
    acur[i] += v.astype(np.float64)
    _check_all(fresh, acur, k, False, TOL[prec])
    fresh.close()


@pytest.mark.parametrize("kind,model", [("power_sum", "exp"), ("power", "linear")])
def test_prepare_updates_then_every_rank(kind, model):
    """linview_prepare_updates captures the propagation graphs of ranks
    1..r_max without running anything (the views are unchanged); updates of
    every rank afterwards replay them and match the oracle.  max_rank past
    r_max is ERANK."""
    from paper_1403_6968_gb300 import LinviewError
    n, k, r_max = 300, 8, 4
    a = li.power_matrix(n, seed=81, dtype=np.float32)
    prog = _prog(kind, [_dev(a)], k=k, r_max=r_max, model=model)
    before = prog.read_view_host(1)
    prog.prepare_updates()
    prog.sync()
    assert np.array_equal(prog.read_view_host(1), before)
    with pytest.raises(LinviewError) as e:
        prog.prepare_updates(r_max + 1)
    assert e.value.name == "ERANK"
    acur = a.astype(np.float64)
    for r in range(1, r_max + 1):
        (u, v), = li.lowrank_update_stream(n, r, 1, seed=82 + r, dtype=np.float32)
        prog.apply_delta(_dev(u), _dev(v))
        acur += u.astype(np.float64) @ v.astype(np.float64).T
    prog.sync()
    if model == "exp":
        _check_all(prog, acur, k, kind == "power_sum", TOL["f32"])
    else:
        pw = op.reeval_powers(acur, k)
        assert rel_frob(prog.read_view_host(k - 1), pw[k]) <= TOL["f32"]
    prog.close()


def test_device_pointer_flags_are_checked():
    """Entry points that take device pointers refuse host memory flagged as
    device memory with EINVAL before any launch.  The host memory here is
    page-locked, which kernels could read through unified addressing, so the
    test cannot fault the GPU even if a check were missing; the views are
    unchanged afterwards."""
    import ctypes as C
    from paper_1403_6968_gb300 import _lib as L
    lib = L.load()
    n, k = 64, 4
    a = li.power_matrix(n, seed=71, dtype=np.float32)
    prog = _prog("power", [_dev(a)], k=k, r_max=2)
    before = prog.read_view_host(2)
    host = torch.zeros((n, n), dtype=torch.float32).pin_memory()
    hp = C.c_void_p(host.data_ptr())
    dev = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    dp = C.c_void_p(dev.data_ptr())
    assert lib.linview_apply_delta(prog.h, 0, 2, hp, n, hp, n, 1, None) == L.EINVAL
    assert lib.linview_apply_row_delta(prog.h, 0, 3, hp, 1, None) == L.EINVAL
    assert lib.linview_read_view(prog.h, 0, hp, n, L.DST_DEVICE, None) == L.EINVAL
    assert lib.linview_level_pass(L.F32, n, hp, n, dp, dp, n, 2, None, None, 1, None) == L.EINVAL
    assert lib.linview_level_pass(L.F32, n, dp, n, hp, dp, n, 2, None, None, 1, None) == L.EINVAL
    assert lib.linview_gemm(L.F32, 0, 0, n, n, n, 1.0, dp, n, hp, n, 0.0, dp, n, None) == L.EINVAL
    prog.sync()
    assert np.array_equal(prog.read_view_host(2), before)
    prog.close()


def test_read_rows_async_host_destination():
    """LINVIEW_DST_HOST_ASYNC: the rows reach a pinned host buffer once the
    stream is synchronised, equal to a synchronous read; an unknown
    destination is EINVAL.  Two steps in flight, as the bench's e2e loop."""
    import ctypes as C
    from paper_1403_6968_gb300 import _lib as L
    n, k = 640, 8
    a = li.power_matrix(n, seed=31, dtype=np.float32)
    prog = _prog("power", [_dev(a)], k=k, r_max=1)
    acur = a.astype(np.float64)
    bufs = [torch.empty((3, n), dtype=torch.float32).pin_memory() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]
    cur = torch.cuda.current_stream()
    seen = []
    for t, (i, v) in enumerate(li.row_update_stream(n, 5, seed=32, dtype=np.float32)):
        b = t % 2
        prog.apply_row_delta(i, torch.from_numpy(v).pin_memory())
        acur[i] += v.astype(np.float64)
        prog.read_view_rows(3, 100 + t, 3, out=bufs[b], sync=False)
        done[b].record(cur)
        if t >= 1:
            done[1 - b].synchronize()
            seen.append((t - 1, bufs[1 - b].numpy().copy()))
    done[b].synchronize()
    seen.append((t, bufs[b].numpy().copy()))
    # the last read matches a synchronous read of the same rows, and the
    # A^8 rows agree with the oracle on the final A
    assert np.array_equal(seen[-1][1], prog.read_view_rows(3, 100 + t, 3))
    ref = op.reeval_powers(acur, k)[k]
    assert rel_frob(seen[-1][1], ref[100 + t:103 + t]) <= 1e-4
    lib = L.load()
    dst = np.zeros((1, n), np.float32)
    st = lib.linview_read_view_rows(prog.h, 3, 0, 1, C.c_void_p(dst.ctypes.data), n, 3, None)
    assert st == L.EINVAL
    with pytest.raises(ValueError):  # a strided out would receive nothing
        prog.read_view_rows(3, 0, 1, out=np.zeros((1, 2 * n), np.float32)[:, ::2])
    prog.close()


def test_full_size_sampled_rows():
    """configs: A^16 and S' = sum_{i<=16} A^i, n=8192, FP32, row and rank-4
    updates; sampled rows of every view vs the oracle computed row by row."""
    n, k = 8192, 16
    a = li.power_matrix(n, seed=0, dtype=np.float32)
    prog = _prog("power_sum", [_dev(a)], k=k, r_max=4)
    acur = a.astype(np.float64)
    rows = [0, 1234, 4097, n - 1]

    def check():
        pr, sr = op.power_rows(acur, rows, k)
        L = 4
        for j in range(L + 1):
            got = prog.read_view_host(j)[rows]
            assert rel_frob(got, pr[1 << j]) <= TOL["f32"], (j, rel_frob(got, pr[1 << j]))
        for j in range(1, L + 1):
            got = prog.read_view_host(L + j)[rows]
            assert rel_frob(got, sr[1 << j]) <= TOL["f32"]

    prog.sync()
    check()
    for i, v in li.row_update_stream(n, 3, seed=0, dtype=np.float32):
        prog.apply_row_delta(i, _dev(v))
        acur[i] += v
    for u, v in li.lowrank_update_stream(n, 4, 2, seed=0, dtype=np.float32):
        prog.apply_delta(_dev(u), _dev(v))
        acur += u.astype(np.float64) @ v.astype(np.float64).T
    prog.sync()
    check()


def test_full_size_bench_configuration():
    """The bench's own program and launch configuration (A^16 and S', n = 8192,
    FP32, r_max = 1: in-pass suffix sums, sums passes on the side stream, graph
    replays) after a stream of row updates; sampled rows, including the
    updated ones, vs the oracle computed row by row."""
    n, k = 8192, 16
    a = li.power_matrix(n, seed=0, dtype=np.float32)
    prog = _prog("power_sum", [_dev(a)], k=k, r_max=1)
    acur = a.astype(np.float64)
    ups = li.row_update_stream(n, 8, seed=5, dtype=np.float32)
    for i, v in ups:
        prog.apply_row_delta(i, _dev(v))
        acur[i] += v
    prog.sync()
    rows = sorted({0, 4097, n - 1} | {int(i) for i, _ in ups[:3]})
    pr, sr = op.power_rows(acur, rows, k)
    L = 4
    for j in range(L + 1):
        got = prog.read_view_host(j)[rows]
        assert rel_frob(got, pr[1 << j]) <= TOL["f32"], (j, rel_frob(got, pr[1 << j]))
    for j in range(1, L + 1):
        got = prog.read_view_host(L + j)[rows]
        assert rel_frob(got, sr[1 << j]) <= TOL["f32"], j


def test_profiling_inside_graph_replays():
    """Per-pass timing runs inside the replayed graphs (instrumented copies)
    and changes no result bit."""
    n, k = 1024, 16
    a = li.power_matrix(n, seed=41, dtype=np.float32)
    ups = li.row_update_stream(n, 28, seed=42, dtype=np.float32)
    plain = _prog("power_sum", [a], k=k, r_max=1)
    prof = _prog("power_sum", [a], k=k, r_max=1)
    prof.set_profiling(True)
    for i, v in ups[:3]:
        plain.apply_row_delta(i, _dev(v))
        prof.apply_row_delta(i, _dev(v))
    prof.reset_stats()
    for i, v in ups[3:8]:
        plain.apply_row_delta(i, _dev(v))
        prof.apply_row_delta(i, _dev(v))
    st = prof.pass_stats(0)
    passes = 9  # 4 fused level passes, 3 sums updates, final P_16 and S'_16 updates
    assert st["launches"] == 5 * passes
    assert st["ms"] > 0 and st["bytes"] == st["launches"] * 2.0 * n * n * 4
    assert prof.pass_stats(1)["launches"] + prof.pass_stats(2)["launches"] == st["launches"]
    for i, v in ups[8:]:
        plain.apply_row_delta(i, _dev(v))
        prof.apply_row_delta(i, _dev(v))
    assert prof.pass_stats(0)["launches"] == 16 * passes  # one sample per instrumented copy
    for vid in range(plain.num_views()):
        assert torch.equal(plain.read_view(vid), prof.read_view(vid))
    plain.close()
    prof.close()
