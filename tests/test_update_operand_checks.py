"""Host-side checks of the update calls of the Python binding (no GPU).

``Program.apply_delta``, ``apply_row_delta`` and ``apply_row_block`` hand
pointers to the library, which reads n rows of every factor (p rows of V for
an update to B).  A factor with too few rows must be refused on the host with
ValueError, before any call into the library.  A program shell (no device
program) drives the checks: arguments that pass them reach the library, which
rejects the null handle with EINVAL.
"""
import numpy as np
import pytest

pytest.importorskip("torch")

from paper_1403_6968_gb300 import _lib as L  # noqa: E402
from paper_1403_6968_gb300.linview import LinviewError, Program  # noqa: E402


def shell(kind=L.POWER, n=32, p=0):
    prog = object.__new__(Program)
    d = L.ProgramDesc()
    d.kind, d.n, d.p = kind, n, p
    prog.desc = d
    prog.n = n
    prog.h = None
    prog.device_index = 0
    prog.precision = L.F32
    prog.np_dtype = np.float32
    return prog


class NullStream:
    """Stands in for a CUDA stream (the legacy stream's handle, 0)."""
    cuda_stream = 0


def reaches_library(fn, *a, **kw):
    with pytest.raises(LinviewError) as e:
        fn(*a, stream=NullStream(), **kw)
    return e.value.name == "EINVAL"


def z(*shape):
    return np.zeros(shape, np.float32)


def test_apply_delta_shapes():
    prog = shell(n=32)
    assert reaches_library(prog.apply_delta, z(32, 3), z(32, 3))
    for u, v in [(z(31, 3), z(32, 3)), (z(32, 3), z(16, 3)), (z(32, 3), z(32, 2)),
                 (z(32, 3, 1), z(32, 3))]:
        with pytest.raises(ValueError):
            prog.apply_delta(u, v)


def test_apply_delta_to_b_takes_p_rows():
    prog = shell(kind=L.ITERATION, n=32, p=5)
    assert reaches_library(prog.apply_delta, z(32, 2), z(5, 2), input_id=1)
    with pytest.raises(ValueError):
        prog.apply_delta(z(32, 2), z(32, 2), input_id=1)   # V of an update to B is p x rank
    with pytest.raises(ValueError):
        prog.apply_delta(z(32, 2), z(5, 2), input_id=0)    # V of an update to A is n x rank


def test_row_delta_and_row_block_shapes():
    prog = shell(n=32)
    assert reaches_library(prog.apply_row_delta, 3, z(32))
    with pytest.raises(ValueError):
        prog.apply_row_delta(3, z(31))
    ols = shell(kind=L.OLS, n=32, p=4)
    assert reaches_library(ols.apply_row_block, [1, 5], z(2, 32))
    for rows, new in [([1, 5], z(2, 31)), ([1, 5, 7], z(2, 32)), ([1], z(32))]:
        with pytest.raises(ValueError):
            ols.apply_row_block(rows, new)


def test_wrong_dtype_is_refused():
    prog = shell(n=8)
    with pytest.raises(TypeError):
        prog.apply_delta(np.zeros((8, 1)), np.zeros((8, 1)))   # FP64 factors, FP32 program


def test_read_and_adjoint_operands():
    """read_view / read_view_rows destinations and the adjoints' tensors:
    exact shape, the program's dtype, unit inner stride; the adjoints take
    CUDA tensors only (a host tensor here is refused before any call)."""
    import torch
    prog = shell(kind=L.ITERATION, n=8, p=3)
    prog.view_shape = lambda vid: (8, 3)   # the shell has no device program to ask
    for bad in (torch.zeros((8, 2)), torch.zeros((8, 3), dtype=torch.float64),
                torch.zeros((3, 8)).t()):
        with pytest.raises(ValueError):
            prog.read_view(1, out=bad, stream=NullStream())
    with pytest.raises(ValueError):
        prog.read_view_rows(1, 0, 2, out=np.zeros((3, 3), np.float32), stream=NullStream())
    assert reaches_library(prog.read_view_rows, 1, 0, 2, out=np.zeros((2, 3), np.float32))
    g = torch.zeros((8, 3))
    with pytest.raises(ValueError):        # host tensors: the adjoints write device memory
        prog.adjoint_iteration_seed(g, dA=torch.zeros((8, 8)), stream=NullStream())
    with pytest.raises(ValueError):
        prog.adjoint_power(torch.zeros((8, 8)), torch.zeros((8, 8)), stream=NullStream())
    with pytest.raises(ValueError):
        prog.adjoint_iteration(dA=torch.zeros((8, 7)), stream=NullStream())


def test_program_inputs_and_replay_factors_are_checked():
    """Program inputs must have the kind's shapes (the library reads them in
    place); a replay trace whose factors reach past its array is refused."""
    from paper_1403_6968_gb300.linview import Server
    with pytest.raises(ValueError):
        Program("power", [z(8, 9)], k=4)
    with pytest.raises(ValueError):
        Program("iteration", [z(8, 8), z(8, 3), z(7, 3)], k=4)
    with pytest.raises(ValueError):
        Program("ols", [z(20, 8), z(19, 2)], k=2)
    srv = object.__new__(Server)
    srv.h, srv._n, srv._keep = None, {0: (16, 16)}, []
    f = np.zeros(2 * 16 * 3, np.float32)
    with pytest.raises(ValueError):   # rank 3 at offset 1 needs 96 floats from there
        srv.replay([0.0], [0], [3], f, [1])
    with pytest.raises(ValueError):
        srv.replay([0.0, 0.1], [0], [3], f, [0])
