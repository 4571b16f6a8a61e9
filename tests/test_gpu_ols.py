"""GPU parity: OLS with W = (X^T X)^{-1} maintained by block Woodbury under
row-block replacements, vs the FP64 oracle (Section 4.1, Example 3.3).

Tolerances: FP64 programs 1e-9 (kappa(X^T X) ~ 1e4 times FP64 rounding);
FP32 programs 1e-4 relative Frobenius per update (the reduced-precision bound)."""
import numpy as np
import pytest

import linview_inputs as li
from oracle import ols as oo
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
@pytest.mark.parametrize("m,n,p,k", [(2000, 200, 4, 1), (3000, 257, 3, 4), (4096, 512, 16, 16),
                                     (100, 30, 1, 5), (1500, 100, 2, 32)])
def test_row_block_updates(prec, m, n, p, k):
    """Every update against the oracle's fresh solve."""
    dt = np.float64 if prec == "f64" else np.float32
    x, y, _ = li.ols_inputs(m, n, p, seed=m + n, dtype=dt)
    prog = _prog("ols", [_dev(x), _dev(y)], k=k, precision=prec)
    ref = oo.IncrementalOLS(x.astype(np.float64), y.astype(np.float64))
    tol = 1e-9 if prec == "f64" else 1e-4
    prog.sync()
    assert rel_frob(prog.read_view_host(0), ref.w) <= tol
    assert rel_frob(prog.read_view_host(1), ref.beta) <= tol
    for rows, new in li.ols_row_replacements(m, n, k, 5, seed=m, dtype=dt, cols_seed=m + n):
        prog.apply_row_block(rows, _dev(new))
        ref.replace_rows(rows, new.astype(np.float64))
        prog.sync()
        fresh = oo.reeval(ref.x, ref.y)
        assert rel_frob(prog.read_view_host(0), fresh["W"]) <= tol
        assert rel_frob(prog.read_view_host(1), fresh["beta"]) <= tol
        assert rel_frob(prog.read_view_host(2), fresh["XtY"]) <= (1e-12 if prec == "f64" else 1e-6)
    assert np.array_equal(prog.read_view_host(3), ref.x.astype(dt))


def test_host_rows_and_errors():
    from paper_1403_6968_gb300 import LinviewError
    m, n, p, k = 500, 40, 2, 3
    x, y, _ = li.ols_inputs(m, n, p, seed=1)
    prog = _prog("ols", [x, y], k=k, precision="f64")
    ref = oo.IncrementalOLS(x, y)
    (rows, new), = li.ols_row_replacements(m, n, k, 1, seed=2, cols_seed=1)
    prog.apply_row_block(rows, new)          # host new rows
    ref.replace_rows(rows, new)
    prog.sync()
    assert rel_frob(prog.read_view_host(0), ref.w) <= 1e-10
    for bad_rows in ([0, 0, 1], [m, 1, 2], [-1, 1, 2]):
        with pytest.raises(LinviewError) as e:
            prog.apply_row_block(bad_rows, new)
        assert e.value.name == "EINVAL"
    with pytest.raises(LinviewError) as e:
        prog.apply_row_block(list(range(k + 1)), np.zeros((k + 1, n)))
    assert e.value.name == "ESHAPE"
    assert rel_frob(prog.read_view_host(0), ref.w) <= 1e-10


def test_high_leverage_core_f32():
    """FP32 programs invert the Woodbury core by a Newton-Schulz iteration from
    C = diag(I, -I), which converges when the replaced rows' leverages are
    small (m >> n) and hands over to Gauss-Jordan otherwise.  m = 40, n = 32
    without scaled columns: leverages near 0.8, kappa(X^T X) about 1e2, so
    FP32 still meets 1e-4 after every update."""
    m, n, p, k = 40, 32, 2, 3
    x, y, _ = li.ols_inputs(m, n, p, seed=77, frac=0.0, dtype=np.float32)
    prog = _prog("ols", [_dev(x), _dev(y)], k=k, precision="f32")
    ref = oo.IncrementalOLS(x.astype(np.float64), y.astype(np.float64))
    for rows, new in li.ols_row_replacements(m, n, k, 6, seed=78, frac=0.0, dtype=np.float32):
        prog.apply_row_block(rows, _dev(new))
        ref.replace_rows(rows, new.astype(np.float64))
        prog.sync()
        fresh = oo.reeval(ref.x, ref.y)
        assert rel_frob(prog.read_view_host(0), fresh["W"]) <= 1e-4
        assert rel_frob(prog.read_view_host(1), fresh["beta"]) <= 1e-4


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_singular_core_is_reported(prec):
    """X = I (16 x 16): replacing row 0 by zeros makes X'^T X' singular, so the
    Woodbury core M = diag(1, -1) + U^T W U = [[1, 0], [0, 0]] is exactly
    singular; the device latches ESINGULAR and W is left as it was (FP32: the
    Newton-Schulz residual starts at 1, so Gauss-Jordan decides)."""
    from paper_1403_6968_gb300 import LinviewError
    n = 16
    dt = np.float64 if prec == "f64" else np.float32
    x = np.eye(n, dtype=dt)
    y = np.arange(2 * n, dtype=dt).reshape(n, 2)
    prog = _prog("ols", [x, y], k=1, precision=prec)
    prog.sync()
    prog.apply_row_block([0], np.zeros((1, n), dtype=dt))
    with pytest.raises(LinviewError) as e:
        prog.sync()
    assert e.value.name == "ESINGULAR"
    assert np.array_equal(prog.read_view_host(0), np.eye(n))


def test_reeval_resets_to_fresh_inverse():
    m, n, p, k = 3000, 256, 4, 4
    x, y, _ = li.ols_inputs(m, n, p, seed=3, dtype=np.float32)
    prog = _prog("ols", [_dev(x), _dev(y)], k=k)
    xs = x.astype(np.float64)
    for rows, new in li.ols_row_replacements(m, n, k, 4, seed=4, dtype=np.float32, cols_seed=3):
        prog.apply_row_block(rows, _dev(new))
        xs[rows] = new
    prog.reeval()
    prog.sync()
    fresh = oo.reeval(xs, y.astype(np.float64))
    assert rel_frob(prog.read_view_host(0), fresh["W"]) <= 1e-5
    assert rel_frob(prog.read_view_host(1), fresh["beta"]) <= 1e-5


@pytest.mark.parametrize("k", [1, 16])
def test_full_size_precision_form(k):
    """X 65536 x 4096 (10% columns x1e-2), Y 65536 x 16, FP32 views, FP64 core;
    three row-block updates, W (sampled rows) and beta vs the FP64 oracle."""
    m, n, p = 65536, 4096, 16
    x, y, _ = li.ols_inputs(m, n, p, seed=0, dtype=np.float32)
    prog = _prog("ols", [_dev(x), _dev(y)], k=k)
    ref = oo.IncrementalOLS(x.astype(np.float64), y.astype(np.float64))
    rows_s = [0, 1000, 2047, n - 1]
    for rows, new in li.ols_row_replacements(m, n, k, 3, seed=k, dtype=np.float32,
                                             cols_seed=0):
        prog.apply_row_block(rows, _dev(new))
        ref.replace_rows(rows, new.astype(np.float64))
        prog.sync()
        w = prog.read_view_rows(0, 0, n)[rows_s]
        assert rel_frob(w, ref.w[rows_s]) <= 1e-4
        assert rel_frob(prog.read_view_host(1), ref.beta) <= 1e-4


@pytest.mark.parametrize("k,count", [(8, 12), (32, 20)])
def test_newton_correction_step(k, count):
    """correction="newton" (FP32 OLS): the program keeps Z = X^T X as
    double-float pairs through the row-block updates, and correct() applies one
    Newton-Schulz step W <- W + W (I - Z W), then refines beta by
    beta + W (X^T Y - Z beta).  The corrected W equals that step taken in FP64
    from the program's own W before the correction and the oracle's exact Z (to
    FP32 rounding: 2e-7); W and beta are no farther from the exact solution
    than before.  k = 32, 20 updates: the 640 replaced rows overflow the
    program's 512-row history once, so Z is also brought up to date in the
    middle of the stream."""
    m, n, p = 3000, 256, 4
    x, y, _ = li.ols_inputs(m, n, p, seed=21, dtype=np.float32)
    prog = _prog("ols", [_dev(x), _dev(y)], k=k, correction="newton")
    ref = oo.IncrementalOLS(x.astype(np.float64), y.astype(np.float64))
    for rows, new in li.ols_row_replacements(m, n, k, count, seed=22, dtype=np.float32,
                                             cols_seed=21):
        prog.apply_row_block(rows, _dev(new))
        ref.replace_rows(rows, new.astype(np.float64))
    prog.sync()
    w0 = prog.read_view_host(0).astype(np.float64)
    b0 = prog.read_view_host(1).astype(np.float64)
    z = ref.x.T @ ref.x
    fresh = oo.reeval(ref.x, ref.y)
    step = oo.newton_schulz_step(w0, z)
    prog.correct()
    prog.sync()
    w1 = prog.read_view_host(0).astype(np.float64)
    b1 = prog.read_view_host(1).astype(np.float64)
    assert rel_frob(w1, step) <= 2e-7
    # beta: one refinement step with the corrected W (the program's own)
    assert rel_frob(b1, oo.refine_beta(w1, b0, ref.xty, z)) <= 2e-7
    assert rel_frob(w1, fresh["W"]) <= 1.05 * rel_frob(w0, fresh["W"]) + 1e-7
    assert rel_frob(b1, fresh["beta"]) <= 1.05 * rel_frob(b0, fresh["beta"]) + 1e-7


def test_newton_correction_period_and_reeval():
    """Every correction_period-th update runs the step; a re-evaluation resets Z
    from the FP64 X^T X (a step right after it keeps W at its rounding)."""
    m, n, p, k = 2000, 200, 3, 4
    x, y, _ = li.ols_inputs(m, n, p, seed=31, dtype=np.float32)
    prog = _prog("ols", [_dev(x), _dev(y)], k=k, correction="newton", correction_period=3)
    ref = oo.IncrementalOLS(x.astype(np.float64), y.astype(np.float64))
    for rows, new in li.ols_row_replacements(m, n, k, 7, seed=32, dtype=np.float32,
                                             cols_seed=31):
        prog.apply_row_block(rows, _dev(new))
        ref.replace_rows(rows, new.astype(np.float64))
        prog.sync()
        fresh = oo.reeval(ref.x, ref.y)
        assert rel_frob(prog.read_view_host(0), fresh["W"]) <= 1e-4
        assert rel_frob(prog.read_view_host(1), fresh["beta"]) <= 1e-4
    prog.reeval()
    prog.sync()
    w0 = prog.read_view_host(0)
    e0 = rel_frob(w0, fresh["W"])
    prog.correct()
    prog.sync()
    assert rel_frob(prog.read_view_host(0), fresh["W"]) <= 2 * e0 + 1e-7


def test_newton_correction_is_fp32_ols_only():
    from paper_1403_6968_gb300 import LinviewError
    x, y, _ = li.ols_inputs(300, 20, 2, seed=41)
    with pytest.raises(LinviewError) as e:
        _prog("ols", [x, y], k=2, precision="f64", correction="newton")
    assert e.value.name == "EUNSUPPORTED"
    a = li.power_matrix(64, seed=1, dtype=np.float32)
    with pytest.raises(LinviewError) as e:
        _prog("power", [_dev(a)], k=4, correction="newton")
    assert e.value.name == "EUNSUPPORTED"
