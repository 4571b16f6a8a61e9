"""GPU: reverse mode through torch.autograd.Function (paper_1403_6968_gb300.autograd).

The backward passes are the library's adjoint kernels on the program's
resident views.  Checked against central finite differences
(torch.autograd.gradcheck, FP64, small n) and against the FP64 oracle's
adjoints (oracle.powers.adjoint_power_chain, oracle.iteration.adjoint).
"""
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


def _ag():
    from paper_1403_6968_gb300 import autograd
    return autograd


def test_matrix_power_gradcheck_fp64():
    ag = _ag()
    a = torch.from_numpy(li.power_matrix(12, seed=3)).cuda().requires_grad_()
    assert torch.autograd.gradcheck(lambda x: ag.matrix_power(x, 8), (a,), eps=1e-6, atol=1e-7,
                                    rtol=1e-5)


def test_general_iteration_gradcheck_fp64():
    ag = _ag()
    a, b, t0 = li.iteration_inputs(10, 3, seed=4)
    args = tuple(torch.from_numpy(x).cuda().requires_grad_() for x in (a, b, t0))
    assert torch.autograd.gradcheck(lambda x, y, z: ag.general_iteration(x, y, z, 5), args,
                                    eps=1e-6, atol=1e-7, rtol=1e-5)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-4)])
def test_matrix_power_grad_vs_oracle(prec, tol):
    ag = _ag()
    dt = np.float64 if prec == "f64" else np.float32
    n, k = 300, 16
    a = li.power_matrix(n, seed=5, dtype=dt)
    g = li.normal((n, n), seed=6, dtype=dt)
    at = torch.from_numpy(a).cuda().requires_grad_()
    out = ag.matrix_power(at, k)
    assert rel_frob(out.detach().cpu().numpy(), op.reeval_powers(a, k)[k]) <= tol
    out.backward(torch.from_numpy(g).cuda())
    ref = op.adjoint_power_chain(a.astype(np.float64), k, g.astype(np.float64))
    assert rel_frob(at.grad.cpu().numpy(), ref) <= tol


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-4)])
def test_general_iteration_loss_grad_vs_oracle(prec, tol):
    ag = _ag()
    dt = np.float64 if prec == "f64" else np.float32
    n, p, k = 256, 8, 16
    a, b, t0 = li.iteration_inputs(n, p, seed=7, dtype=dt)
    ts = [torch.from_numpy(x).cuda().requires_grad_() for x in (a, b, t0)]
    tk = ag.general_iteration(*ts, k)
    (tk * tk).sum().backward()
    da, db, dt0 = oi.adjoint(a.astype(np.float64), b.astype(np.float64), t0.astype(np.float64), k)
    for got, ref in zip(ts, (da, db, dt0)):
        assert rel_frob(got.grad.cpu().numpy(), ref) <= tol
