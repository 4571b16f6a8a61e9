"""GPU: a program's device memory through the caller's allocator callbacks.

The descriptor's alloc/free callbacks let PyTorch's caching allocator own the
views, factor arenas and scratch of a program: the bytes PyTorch was asked for
(its requested_bytes counter) grow by exactly linview_program_device_bytes at
creation (and by the lazily made work space of later calls), memory_allocated()
by at least that much (PyTorch may hand out a whole cached segment, up to 1 MB
more, for a large request), the estimate used for admission is the same
figure, and everything goes back to the allocator at linview_destroy.  With
allocator=None the library uses cudaMalloc and PyTorch sees nothing.
"""
import numpy as np
import pytest

import linview_inputs as li
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


def _pkg():
    import paper_1403_6968_gb300 as P
    return P


def _requested():
    return torch.cuda.memory_stats()["requested_bytes.all.current"]


@pytest.mark.parametrize("kind,n,k,r_max", [("power", 1000, 16, 4), ("power_sum", 2048, 16, 1),
                                            ("power_sum", 513, 8, 8)])
def test_power_program_memory_is_torchs(kind, n, k, r_max):
    import gc
    P = _pkg()
    a = li.power_matrix(n, seed=3, dtype=np.float32)
    ad = torch.from_numpy(a).cuda()
    # programs left unreferenced by earlier tests return their memory when
    # collected: collect them now, not in the middle of the measurement
    gc.collect()
    torch.cuda.synchronize()
    before, req0 = torch.cuda.memory_allocated(), _requested()
    prog = P.Program(kind, [ad], k=k, r_max=r_max)
    held = P.program_device_bytes(prog)
    assert held == P.estimate_device_bytes(n, k, r_max=r_max, kind=kind)
    assert _requested() - req0 == held
    assert torch.cuda.memory_allocated() - before >= held
    # the program works on that memory
    (i, v), = li.row_update_stream(n, 1, seed=4, dtype=np.float32)
    prog.apply_row_delta(i, torch.from_numpy(v).cuda())
    prog.sync()
    a64 = a.astype(np.float64)
    a64[i] += v
    assert rel_frob(prog.read_view_host(op.levels(k).index(k)), op.reeval_powers(a64, k)[k]) <= 1e-4
    prog.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before and _requested() == req0


def test_cudamalloc_default_is_invisible_to_torch():
    P = _pkg()
    n = 1024
    a = li.power_matrix(n, seed=5, dtype=np.float32)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    prog = P.Program("power", [a], k=16, r_max=2, allocator=None)
    assert P.program_device_bytes(prog) > 0
    assert torch.cuda.memory_allocated() == before
    prog.close()


def test_lazy_work_space_and_ols_through_the_allocator():
    import gc
    P = _pkg()
    n, p, k = 300, 8, 4
    a, b, t0 = li.iteration_inputs(n, p, seed=6)
    gc.collect()  # earlier tests' unreferenced programs free their memory now
    torch.cuda.synchronize()
    req0 = _requested()
    prog = P.Program("iteration", [a, b, t0], k=k, r_max=2, p=p, precision="f64")
    held0 = P.program_device_bytes(prog)
    assert _requested() - req0 == held0
    dA = torch.empty((n, n), dtype=torch.float64, device="cuda")
    dB = torch.empty((n, p), dtype=torch.float64, device="cuda")
    base = _requested()
    prog.adjoint_iteration(dA, dB)   # allocates its gradient panel on first use
    torch.cuda.synchronize()
    held1 = P.program_device_bytes(prog)
    assert held1 > held0
    assert _requested() - base == held1 - held0
    prog.close()
    del dA, dB
    torch.cuda.synchronize()
    assert _requested() == req0
    x, y, _ = li.ols_inputs(4096, 256, 4, seed=7)
    ols = P.Program("ols", [x, y], k=4, precision="f64")
    assert _requested() - req0 == P.program_device_bytes(ols)
    ols.close()
    torch.cuda.synchronize()
    assert _requested() == req0


def test_temporary_work_space_goes_back():
    """Re-evaluation (FP32, own tensor-core GEMM) takes its split operands as
    temporary blocks from the allocator and returns them in the same call."""
    P = _pkg()
    n = 1024
    a = li.power_matrix(n, seed=9, dtype=np.float32)
    prog = P.Program("power_sum", [a], k=8, r_max=1)
    torch.cuda.synchronize()
    req0 = _requested()
    peak0 = torch.cuda.max_memory_allocated()
    torch.cuda.reset_peak_memory_stats()
    prog.reeval()
    torch.cuda.synchronize()
    assert _requested() == req0
    # the split operands (2 x n x 2n floats) were live during the call
    assert torch.cuda.max_memory_allocated() - torch.cuda.memory_allocated() >= 2 * n * 2 * n * 4
    prog.close()
    del peak0


def test_allocator_failure_is_enomem():
    """An allocator that refuses makes creation fail with ENOMEM and leaks
    nothing it handed out before."""
    import ctypes as C
    from paper_1403_6968_gb300 import _lib as L
    lib = L.load()
    handed = []

    def alloc(nbytes, stream, ctx):
        if len(handed) >= 3:
            return None
        ptr = torch.cuda.caching_allocator_alloc(int(nbytes))
        handed.append(ptr)
        return ptr

    def free(ptr, nbytes, stream, ctx):
        handed.remove(int(ptr))
        torch.cuda.caching_allocator_delete(int(ptr))

    fa, ff = L.ALLOC_FN(alloc), L.FREE_FN(free)
    n = 256
    a = li.power_matrix(n, seed=8, dtype=np.float32)
    d = L.ProgramDesc()
    d.kind, d.precision, d.n, d.k, d.r_max = L.POWER, L.F32, n, 8, 1
    d.alloc = C.cast(fa, C.c_void_p).value
    d.free = C.cast(ff, C.c_void_p).value
    h = C.c_void_p()
    ptrs = (C.c_void_p * 1)(a.ctypes.data)
    lds = (C.c_int64 * 1)(n)
    st = lib.linview_create_program(C.byref(d), ptrs, lds, 0, None, C.byref(h))
    assert st == L.ENOMEM and not h.value
    assert handed == []      # the blocks obtained before the refusal went back
    d.free = None            # alloc without free is rejected up front
    assert lib.linview_create_program(C.byref(d), ptrs, lds, 0, None, C.byref(h)) == L.EINVAL
