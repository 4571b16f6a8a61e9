"""GPU parity: the linear iterative model of matrix powers (Appendix A,
P_i = A P_{i-1}, views A, A^2, ..., A^k) and its sums view S'_k, through the
C ABI, against the FP64 oracle's re-evaluation on the updated A.

Tolerances as for the exponential model: FP64 1e-10, FP32 1e-4 relative
Frobenius error."""
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


def _np(prec):
    return np.float64 if prec == "f64" else np.float32


def _check(prog, a, k, sums, prec):
    pw = op.linear_powers(a, k)
    for i in range(1, k + 1):
        got = prog.read_view(i - 1).cpu().numpy().astype(np.float64)
        assert rel_frob(got, pw[i - 1]) <= TOL[prec], (i, rel_frob(got, pw[i - 1]))
    if sums:
        got = prog.read_view(k).cpu().numpy().astype(np.float64)
        ref = np.sum(pw, axis=0)
        assert rel_frob(got, ref) <= TOL[prec]


@pytest.mark.parametrize("prec,n,k,r,sums", [
    ("f64", 256, 2, 1, False), ("f64", 256, 3, 1, True), ("f64", 200, 5, 2, True),
    ("f64", 256, 8, 1, True), ("f64", 300, 8, 4, False), ("f32", 1000, 16, 1, True),
    ("f32", 777, 16, 4, True), ("f32", 512, 32, 2, False)])
def test_linear_model_matches_reevaluation(prec, n, k, r, sums):
    from paper_1403_6968_gb300 import Program
    dt = _np(prec)
    a = li.power_matrix(n, seed=n + k, dtype=dt)
    prog = Program("power_sum" if sums else "power", [a], k=k, r_max=r, precision=prec,
                   model="linear")
    assert prog.num_views() == k + (1 if sums else 0)
    acur = a.astype(np.float64)
    if r == 1:
        for i, v in li.row_update_stream(n, 6, seed=k, dtype=dt):
            prog.apply_row_delta(i, v)
            acur[i] += v.astype(np.float64)
    else:
        for u, v in li.lowrank_update_stream(n, r, 6, seed=k, dtype=dt):
            prog.apply_delta(u, v)
            acur += u.astype(np.float64) @ v.astype(np.float64).T
    _check(prog, acur, k, sums, prec)
    # the incremental oracle of the same model agrees with its re-evaluation
    prog.close()


def test_linear_model_matches_exponential_model():
    """Both models maintain A^k: after the same updates their A^k views agree."""
    from paper_1403_6968_gb300 import Program
    n, k = 512, 16
    a = li.power_matrix(n, seed=3, dtype=np.float32)
    lin = Program("power", [a], k=k, r_max=2, model="linear")
    exp = Program("power", [a], k=k, r_max=2)
    for u, v in li.lowrank_update_stream(n, 2, 5, seed=4, dtype=np.float32):
        lin.apply_delta(u, v)
        exp.apply_delta(u, v)
    x = lin.read_view(k - 1).cpu().numpy().astype(np.float64)
    y = exp.read_view(4).cpu().numpy().astype(np.float64)
    assert rel_frob(x, y) <= 1e-4
    lin.close()
    exp.close()


def test_linear_model_errors():
    from paper_1403_6968_gb300 import LinviewError, Program
    a = li.power_matrix(64, seed=1, dtype=np.float32)
    with pytest.raises(LinviewError) as e:
        Program("power", [a], k=16, r_max=8, model="linear")  # r_max * k > 64
    assert e.value.name == "EUNSUPPORTED"
    with pytest.raises(LinviewError):
        Program("power", [a], k=1, r_max=1, model="linear")
    it = li.iteration_inputs(64, 2, seed=1, dtype=np.float32)
    with pytest.raises(LinviewError):  # the skip step must be a power of two
        Program("iteration", list(it), k=6, r_max=1, model="skip", skip=3)
    prog = Program("power", [a], k=4, r_max=1, model="linear")
    g = torch.zeros((64, 64), device="cuda")
    with pytest.raises(LinviewError):
        prog.adjoint_power(g, torch.zeros_like(g))
    prog.close()


@pytest.mark.parametrize("prec,n,k,s,r,sums", [
    ("f64", 256, 8, 2, 1, True), ("f64", 200, 12, 4, 2, False), ("f64", 256, 16, 4, 1, True),
    ("f64", 128, 8, 1, 2, True), ("f32", 1000, 16, 4, 1, True), ("f32", 777, 16, 2, 4, True),
    ("f32", 512, 32, 8, 2, False)])
def test_skip_model_matches_reevaluation(prec, n, k, s, r, sums):
    """Skip-s model (Appendix A): views A^(2^j) up to A^s, then A^2s .. A^k,
    and the sums S'_h of the same h (Section 4.2.3)."""
    from paper_1403_6968_gb300 import Program
    dt = _np(prec)
    a = li.power_matrix(n, seed=n + k + s, dtype=dt)
    prog = Program("power_sum" if sums else "power", [a], k=k, r_max=r, precision=prec,
                   model="skip", skip=s)
    hs = op.skip_levels(k, s)
    assert prog.num_views() == (2 * len(hs) - 1 if sums else len(hs))
    acur = a.astype(np.float64)
    if r == 1:
        for i, v in li.row_update_stream(n, 6, seed=k + s, dtype=dt):
            prog.apply_row_delta(i, v)
            acur[i] += v.astype(np.float64)
    else:
        for u, v in li.lowrank_update_stream(n, r, 6, seed=k + s, dtype=dt):
            prog.apply_delta(u, v)
            acur += u.astype(np.float64) @ v.astype(np.float64).T
    ref = op.skip_powers(acur, k, s)
    for vid, h in enumerate(hs):
        got = prog.read_view(vid).cpu().numpy().astype(np.float64)
        assert rel_frob(got, ref[h]) <= TOL[prec], (h, rel_frob(got, ref[h]))
    if sums:
        sref = op.skip_sums(acur, k, s)
        for j, h in enumerate(hs[1:], start=1):
            got = prog.read_view(len(hs) + j - 1).cpu().numpy().astype(np.float64)
            assert rel_frob(got, sref[h]) <= TOL[prec], ("S", h, rel_frob(got, sref[h]))
    prog.close()


def test_skip_model_errors():
    from paper_1403_6968_gb300 import LinviewError, Program
    a = li.power_matrix(64, seed=1, dtype=np.float32)
    for k, s in ((16, 3), (12, 8), (8, 8)):
        with pytest.raises(LinviewError):
            Program("power", [a], k=k, r_max=1, model="skip", skip=s)
    with pytest.raises(LinviewError):
        Program("power", [a], k=8, r_max=1, model="exp", skip=2)
