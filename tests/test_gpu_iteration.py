"""GPU parity: general form T_{i+1} = A T_i + B (Appendix B, linear model) and
the adjoints of L = ||T_k||_F^2 and of a loss of P_k, vs the FP64 oracle.

Tolerances: FP64 1e-10 for views, FP32 1e-4 (spec bounds); the FP64 GPU
adjoint meets central finite differences (h = 1e-3, FP64, n = 512) within
1e-6 ||dA||_F (truncation O(h^2) is far smaller; a wrong term is O(||dA||))."""
import numpy as np
import pytest

import linview_inputs as li
from oracle import iteration as oi
from oracle import powers as op
from oracle.metrics import rel_frob

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n,p,k,r", [(300, 5, 16, 2), (1, 1, 1, 1), (777, 64, 16, 2),
                                     (1030, 3, 4, 4), (64, 7, 2, 1)])
def test_iteration_incremental(prec, n, p, k, r):
    dt = np.float64 if prec == "f64" else np.float32
    a, b, t0 = li.iteration_inputs(n, p, seed=n, dtype=dt)
    prog = _prog("iteration", [_dev(a), _dev(b), _dev(t0)], k=k, r_max=r, precision=prec)
    acur = a.astype(np.float64)
    b64, t064 = b.astype(np.float64), t0.astype(np.float64)
    tol = 1e-10 if prec == "f64" else 1e-4
    ref = oi.reeval(acur, b64, t064, k)
    prog.sync()
    for i in range(1, k + 1):
        assert rel_frob(prog.read_view_host(i), ref[i]) <= tol
    for u, v in li.lowrank_update_stream(n, r, 3, seed=n + 1, dtype=dt):
        prog.apply_delta(_dev(u), _dev(v))
        acur += u.astype(np.float64) @ v.astype(np.float64).T
        prog.sync()
        ref = oi.reeval(acur, b64, t064, k)
        for i in range(1, k + 1):
            assert rel_frob(prog.read_view_host(i), ref[i]) <= tol, i
        assert rel_frob(prog.read_view_host(0), acur) <= tol


def test_iteration_matches_oracle_incremental_factors_path():
    n, p, k, r = 500, 8, 16, 2
    a, b, t0 = li.iteration_inputs(n, p, seed=1)
    prog = _prog("iteration", [_dev(a), _dev(b), _dev(t0)], k=k, r_max=r, precision="f64")
    inc = oi.IncrementalIteration(a, b, t0, k)
    for u, v in li.lowrank_update_stream(n, r, 3, seed=2):
        prog.apply_delta(_dev(u), _dev(v))
        inc.apply(u, v)
    prog.sync()
    for i in range(1, k + 1):
        assert rel_frob(prog.read_view_host(i), inc.t[i]) <= 1e-10


def _unit(x):
    return x / np.linalg.norm(x)


def test_iteration_adjoint_fp64_central_fd_n512():
    """Differentiation form at the FD size: n=512, p=64, k=16, FP64."""
    n, p, k = 512, 64, 16
    a, b, t0 = li.iteration_inputs(n, p, seed=21)
    prog = _prog("iteration", [_dev(a), _dev(b), _dev(t0)], k=k, r_max=2, precision="f64")
    (u, v), = li.lowrank_update_stream(n, 2, 1, seed=22)
    prog.apply_delta(_dev(u), _dev(v))
    acur = a + u @ v.T
    dA = torch.empty((n, n), dtype=torch.float64, device="cuda")
    dB = torch.empty((n, p), dtype=torch.float64, device="cuda")
    prog.adjoint_iteration(dA, dB)
    torch.cuda.synchronize()
    da, db = dA.cpu().numpy(), dB.cpu().numpy()
    ra, rb, _ = oi.adjoint(acur, b, t0, k)
    assert rel_frob(da, ra) <= 1e-10
    assert rel_frob(db, rb) <= 1e-10
    h = 1e-3
    g = np.random.default_rng(23)
    dirs = [_unit(li.normal((n, n), seed=30 + t)) for t in range(8)]
    for _ in range(8):
        e = np.zeros((n, n)); e[g.integers(n), g.integers(n)] = 1.0
        dirs.append(e)
    scale = float(np.linalg.norm(da))
    for e in dirs:
        fd = (oi.loss(acur + h * e, b, t0, k) - oi.loss(acur - h * e, b, t0, k)) / (2 * h)
        assert abs(fd - float(np.sum(da * e))) <= 1e-6 * scale
    for t in range(3):
        e = _unit(li.normal((n, p), seed=40 + t))
        fd = (oi.loss(acur, b + h * e, t0, k) - oi.loss(acur, b - h * e, t0, k)) / (2 * h)
        assert abs(fd - float(np.sum(db * e))) <= 1e-6 * float(np.linalg.norm(db))


@pytest.mark.parametrize("n,p", [(2048, 64), (1000, 3)])
def test_iteration_adjoint_fp32_vs_oracle(n, p):
    """p = 64: the products with A and A^T on the split-TF32 GEMM; p = 3: as
    products passes over A (a few columns)."""
    k = 16
    a, b, t0 = li.iteration_inputs(n, p, seed=31, dtype=np.float32)
    prog = _prog("iteration", [_dev(a), _dev(b), _dev(t0)], k=k, r_max=2)
    (u, v), = li.lowrank_update_stream(n, 2, 1, seed=32, dtype=np.float32)
    prog.apply_delta(_dev(u), _dev(v))
    acur = a.astype(np.float64) + u.astype(np.float64) @ v.astype(np.float64).T
    dA = torch.empty((n, n), dtype=torch.float32, device="cuda")
    dB = torch.empty((n, p), dtype=torch.float32, device="cuda")
    prog.adjoint_iteration(dA, dB)
    torch.cuda.synchronize()
    ra, rb, _ = oi.adjoint(acur, b.astype(np.float64), t0.astype(np.float64), k)
    assert rel_frob(dA.cpu().numpy(), ra) <= 1e-4
    assert rel_frob(dB.cpu().numpy(), rb) <= 1e-4
    # the seeded form at the seed 2 T_k is the same reverse pass, and adds
    # dT_0 = A^T G_1 (the oracle's third gradient)
    ra, rb, rt0 = oi.adjoint(acur, b.astype(np.float64), t0.astype(np.float64), k)
    gk = 2.0 * prog.read_view(k)
    dT0 = torch.empty((n, p), dtype=torch.float32, device="cuda")
    prog.adjoint_iteration_seed(gk, dA, dB, dT0)
    torch.cuda.synchronize()
    assert rel_frob(dT0.cpu().numpy(), rt0) <= 1e-4
    assert rel_frob(dB.cpu().numpy(), rb) <= 1e-4
    assert rel_frob(dA.cpu().numpy(), ra) <= 1e-4


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_power_adjoint_vs_oracle(prec):
    n, k = 384, 16
    dt = np.float64 if prec == "f64" else np.float32
    a = li.power_matrix(n, seed=41, dtype=dt)
    g = li.normal((n, n), seed=42, dtype=dt)
    prog = _prog("power", [_dev(a)], k=k, r_max=1, precision=prec)
    dA = torch.empty((n, n), dtype=torch.float64 if prec == "f64" else torch.float32,
                     device="cuda")
    prog.adjoint_power(_dev(g), dA)
    torch.cuda.synchronize()
    ref = op.adjoint_power_chain(a.astype(np.float64), k, g.astype(np.float64))
    assert rel_frob(dA.cpu().numpy(), ref) <= (1e-10 if prec == "f64" else 1e-4)


@pytest.mark.parametrize("prec,n,p,k,rb", [("f64", 300, 7, 8, 1), ("f64", 256, 16, 16, 2),
                                            ("f32", 1000, 64, 16, 2)])
def test_iteration_b_updates(prec, n, p, k, rb):
    """Updates to B (input 1) interleaved with updates to A, against the
    oracle's re-evaluation on the current A and B."""
    from paper_1403_6968_gb300 import Program
    from oracle import iteration as oi
    dt = np.float64 if prec == "f64" else np.float32
    a, b, t0 = li.iteration_inputs(n, p, seed=n + p, dtype=dt)
    prog = Program("iteration", [a, b, t0], k=k, r_max=max(rb, 2), precision=prec)
    acur, bcur = a.astype(np.float64), b.astype(np.float64)
    g = np.random.default_rng(n)
    for step in range(4):
        if step % 2:
            u = (g.standard_normal((n, 2)) * 0.01).astype(dt)
            v = (g.standard_normal((n, 2)) * 0.01).astype(dt)
            prog.apply_delta(u, v)
            acur += u.astype(np.float64) @ v.astype(np.float64).T
        else:
            ub = g.standard_normal((n, rb)).astype(dt)
            vb = g.standard_normal((p, rb)).astype(dt)
            prog.apply_delta(ub, vb, input_id=1)
            bcur += ub.astype(np.float64) @ vb.astype(np.float64).T
    ref = oi.reeval(acur, bcur, t0.astype(np.float64), k)
    tol = 1e-10 if prec == "f64" else 1e-4
    for i in range(1, k + 1):
        got = prog.read_view(i).cpu().numpy().astype(np.float64)
        assert rel_frob(got, ref[i]) <= tol, i
    got_b = prog.read_view(k + 1).cpu().numpy().astype(np.float64)
    assert rel_frob(got_b, bcur) <= tol
    prog.close()


@pytest.mark.parametrize("prec,k,r", [("f64", 16, 8), ("f32", 32, 8), ("f64", 48, 8),
                                      ("f32", 96, 8)])
def test_iteration_long_chains_wide_updates(prec, k, r):
    """Many views times a wide rank: the T-panel update stages (16 + 64) k r
    elements.  Past 48 KB (FP64 k r = 128, FP32 k r = 256) it opts in to more
    shared memory; past the device's limit (FP64 k r = 384, FP32 k r = 768)
    every view takes its own GEMM.  Updates to A and to B, against the
    oracle's re-evaluation."""
    n, p = 160, 3
    dt = np.float64 if prec == "f64" else np.float32
    a, b, t0 = li.iteration_inputs(n, p, seed=k + r, dtype=dt)
    prog = _prog("iteration", [_dev(a), _dev(b), _dev(t0)], k=k, r_max=r, precision=prec)
    acur, bcur = a.astype(np.float64), b.astype(np.float64)
    g = np.random.default_rng(k)
    for step in range(3):
        if step != 1:
            u = (g.standard_normal((n, r)) * 0.01).astype(dt)
            v = (g.standard_normal((n, r)) * 0.01).astype(dt)
            prog.apply_delta(_dev(u), _dev(v))
            acur += u.astype(np.float64) @ v.astype(np.float64).T
        else:
            ub = g.standard_normal((n, r)).astype(dt)
            vb = g.standard_normal((p, r)).astype(dt)
            prog.apply_delta(_dev(ub), _dev(vb), input_id=1)
            bcur += ub.astype(np.float64) @ vb.astype(np.float64).T
    prog.sync()
    ref = oi.reeval(acur, bcur, t0.astype(np.float64), k)
    tol = 1e-10 if prec == "f64" else 1e-4
    for i in range(1, k + 1):
        assert rel_frob(prog.read_view_host(i), ref[i]) <= tol, i
    prog.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n,p,k,r", [(300, 5, 16, 2), (1, 1, 1, 1), (777, 64, 16, 2),
                                     (1030, 3, 4, 4), (513, 1, 16, 1)])
def test_iteration_hybrid_strategy(prec, n, p, k, r):
    """Hybrid strategy (Sec. 4.3: dense dT_i, one n x n x p product per step)
    against the oracle's hybrid evaluation (the paper's three-term rule) and
    its re-evaluation, on updates to A (factored and row) and to B."""
    dt = np.float64 if prec == "f64" else np.float32
    a, b, t0 = li.iteration_inputs(n, p, seed=n + 7, dtype=dt)
    prog = _prog("iteration", [_dev(a), _dev(b), _dev(t0)], k=k, r_max=r, precision=prec,
                 strategy="hybrid")
    hyb = oi.HybridIteration(a, b, t0, k)
    acur, bcur = a.astype(np.float64), b.astype(np.float64)
    tol = 1e-10 if prec == "f64" else 1e-4
    g = np.random.default_rng(n)
    for step, (u, v) in enumerate(li.lowrank_update_stream(n, r, 3, seed=n + 8, dtype=dt)):
        prog.apply_delta(_dev(u), _dev(v))
        hyb.apply(u, v)
        acur += u.astype(np.float64) @ v.astype(np.float64).T
        if step == 1:  # a row update e_i v^T of A and a rank-1 update of B
            i = int(g.integers(n))
            w = (g.standard_normal(n) * 0.01).astype(dt)
            prog.apply_row_delta(i, _dev(w))
            e = np.zeros((n, 1))
            e[i, 0] = 1.0
            hyb.apply(e, w.astype(np.float64).reshape(n, 1))
            acur[i] += w.astype(np.float64)
            ub = g.standard_normal((n, 1)).astype(dt)
            vb = g.standard_normal((p, 1)).astype(dt)
            prog.apply_delta(_dev(ub), _dev(vb), input_id=1)
            bcur += ub.astype(np.float64) @ vb.astype(np.float64).T
            hyb = oi.HybridIteration(acur, bcur, t0, k)  # B changed: restart the oracle
    prog.sync()
    ref = oi.reeval(acur, bcur, t0.astype(np.float64), k)
    for i in range(1, k + 1):
        got = prog.read_view_host(i)
        assert rel_frob(got, ref[i]) <= tol, i
        assert rel_frob(got, hyb.t[i]) <= tol, i
    assert rel_frob(prog.read_view_host(0), acur) <= tol
    assert rel_frob(prog.read_view_host(k + 1), bcur) <= tol


def test_iteration_hybrid_equals_factored_fp64():
    """Both strategies maintain the same views (FP64, to rounding)."""
    n, p, k, r = 400, 9, 8, 2
    a, b, t0 = li.iteration_inputs(n, p, seed=31)
    progs = [_prog("iteration", [_dev(a), _dev(b), _dev(t0)], k=k, r_max=r, precision="f64",
                   strategy=s) for s in ("factored", "hybrid")]
    for u, v in li.lowrank_update_stream(n, r, 4, seed=32):
        for pr in progs:
            pr.apply_delta(_dev(u), _dev(v))
    for pr in progs:
        pr.sync()
    for i in range(1, k + 1):
        assert rel_frob(progs[1].read_view_host(i), progs[0].read_view_host(i)) <= 1e-11, i


def test_strategy_validation():
    from paper_1403_6968_gb300 import LinviewError
    a = li.power_matrix(64, seed=1)
    with pytest.raises(LinviewError):
        _prog("power", [_dev(a)], k=4, precision="f64", strategy="hybrid")


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n,p,k,r,model,s", [(300, 5, 16, 2, "exp", 8), (1030, 3, 4, 1, "exp", 2),
                                             (513, 64, 8, 2, "exp", 4), (64, 1, 2, 1, "exp", 1),
                                             (777, 16, 16, 1, "skip", 4), (300, 7, 8, 2, "skip", 2),
                                             (129, 3, 5, 1, "skip", 1), (1030, 9, 12, 1, "skip", 4)])
def test_iteration_exp_and_skip_models(prec, n, p, k, r, model, s):
    """Exponential and skip-s models of the general form (App. B): the views
    T_1, T_2, .., T_s, T_2s, .., T_k (and the auxiliary P_h, S'_h) after factored
    and row updates of A and an update to B, against the oracle's
    re-evaluation."""
    dt = np.float64 if prec == "f64" else np.float32
    a, b, t0 = li.iteration_inputs(n, p, seed=n + 11, dtype=dt)
    kw = {"model": model} if model == "exp" else {"model": "skip", "skip": s}
    prog = _prog("iteration", [_dev(a), _dev(b), _dev(t0)], k=k, r_max=r, precision=prec, **kw)
    Ls = s.bit_length() - 1
    tidx = [1 << j for j in range(Ls + 1)] + list(range(2 * s, k + 1, s))
    NT = len(tidx)
    assert prog.num_views() == 1 + NT + 2 + 2 * Ls
    acur = a.astype(np.float64)
    b64, t064 = b.astype(np.float64), t0.astype(np.float64)
    tol = 1e-10 if prec == "f64" else 1e-4

    def check():
        prog.sync()
        T, P, S = oi.skip_reeval(acur, b64, t064, k, s)
        for j, i in enumerate(tidx):
            assert rel_frob(prog.read_view_host(1 + j), T[i]) <= tol, i
        assert rel_frob(prog.read_view_host(0), acur) <= tol
        assert rel_frob(prog.read_view_host(NT + 1), b64) <= tol
        for l in range(1, Ls + 1):
            h = 1 << l
            assert rel_frob(prog.read_view_host(NT + 2 + l), P[h]) <= tol, h
            sprime = S[h] - np.eye(n) + P[h]   # S'_h = A + .. + A^h
            assert rel_frob(prog.read_view_host(NT + 2 + Ls + l), sprime) <= tol, h

    check()
    g = np.random.default_rng(n)
    for step, (u, v) in enumerate(li.lowrank_update_stream(n, r, 3, seed=n + 12, dtype=dt)):
        prog.apply_delta(_dev(u), _dev(v))
        acur += u.astype(np.float64) @ v.astype(np.float64).T
        if step == 1:
            i = int(g.integers(n))
            w = (g.standard_normal(n) * 0.01).astype(dt)
            prog.apply_row_delta(i, _dev(w))
            acur[i] += w.astype(np.float64)
            ub = g.standard_normal((n, r)).astype(dt)
            vb = g.standard_normal((p, r)).astype(dt)
            prog.apply_delta(_dev(ub), _dev(vb), input_id=1)
            b64 += ub.astype(np.float64) @ vb.astype(np.float64).T
    check()


def test_iteration_exp_model_errors():
    from paper_1403_6968_gb300 import LinviewError, _lib
    n, p = 64, 3
    a, b, t0 = li.iteration_inputs(n, p, seed=5)
    with pytest.raises(LinviewError) as e:
        _prog("iteration", [_dev(a), _dev(b), _dev(t0)], k=6, precision="f64", model="exp")
    assert e.value.status == _lib.EINVAL
    with pytest.raises(LinviewError) as e:  # k must be a multiple of s and >= 2s
        _prog("iteration", [_dev(a), _dev(b), _dev(t0)], k=6, precision="f64", model="skip",
              skip=4)
    assert e.value.status == _lib.EINVAL
    with pytest.raises(LinviewError):
        _prog("iteration", [_dev(a), _dev(b), _dev(t0)], k=4, precision="f64", model="exp",
              strategy="hybrid")


@pytest.mark.parametrize("prec,model,s", [("f64", "exp", 4), ("f64", "skip", 2), ("f32", "skip", 4)])
def test_iteration_adjoint_exp_and_skip_models(prec, model, s):
    """The adjoint of L = ||T_k||_F^2 does not depend on the iterative model:
    exponential and skip programs (which keep only some T_i) give the oracle's
    gradients after updates."""
    n, p, k = 256, 8, 8
    dt = np.float64 if prec == "f64" else np.float32
    a, b, t0 = li.iteration_inputs(n, p, seed=77, dtype=dt)
    kw = {"model": "exp"} if model == "exp" else {"model": "skip", "skip": s}
    prog = _prog("iteration", [_dev(a), _dev(b), _dev(t0)], k=k, r_max=2, precision=prec, **kw)
    acur = a.astype(np.float64)
    for u, v in li.lowrank_update_stream(n, 2, 2, seed=78, dtype=dt):
        prog.apply_delta(_dev(u), _dev(v))
        acur += u.astype(np.float64) @ v.astype(np.float64).T
    tdt = torch.float64 if prec == "f64" else torch.float32
    dA = torch.zeros((n, n), dtype=tdt, device="cuda")
    dB = torch.zeros((n, p), dtype=tdt, device="cuda")
    prog.adjoint_iteration(dA, dB)
    torch.cuda.synchronize()
    ra, rb, _ = oi.adjoint(acur, b.astype(np.float64), t0.astype(np.float64), k)
    tol = 1e-10 if prec == "f64" else 1e-4
    assert rel_frob(dA.cpu().numpy(), ra) <= tol
    assert rel_frob(dB.cpu().numpy(), rb) <= tol
