"""GPU: the library's own dense product (linview_gemm) against FP64 products
of the same inputs.

FP32 products that fill tensor-core tiles run on tcgen05 in split TF32 and
must reach near-FP32 accuracy: relative Frobenius error <= 1e-6 (measured
1.7e-7 at K = 1024 and 3.2e-7 at K = 8192; one TF32 product alone gives ~5e-4
and whole-K accumulation in tensor memory ~8e-6 at K = 1000, so a dropped lo
term or a lost segment fails); the rest, and every FP64 product, run on the
CUDA cores.  Shapes span several tiles with
ragged edges in M, N and K, all four transpose combinations, accumulation
into C (beta = 1, in place) and the degenerate sizes.
"""
import numpy as np
import pytest

from oracle.metrics import rel_frob

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _run(M, N, K, ta, tb, alpha, beta, dtype, seed=0):
    from paper_1403_6968_gb300 import gemm
    g = np.random.default_rng(seed)
    npdt = np.float64 if dtype == torch.float64 else np.float32
    a = g.standard_normal((K, M) if ta else (M, K)).astype(npdt)
    b = g.standard_normal((N, K) if tb else (K, N)).astype(npdt)
    c0 = g.standard_normal((M, N)).astype(npdt)
    c = torch.from_numpy(c0.copy()).cuda()
    gemm(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), c, alpha=alpha, beta=beta,
         ta=ta, tb=tb)
    torch.cuda.synchronize()
    A = a.astype(np.float64).T if ta else a.astype(np.float64)
    B = b.astype(np.float64).T if tb else b.astype(np.float64)
    ref = alpha * (A @ B) + beta * c0.astype(np.float64)
    return rel_frob(c.cpu().numpy(), ref)


@pytest.mark.parametrize("M,N,K", [(1000, 1000, 1000), (300, 200, 700), (8192, 64, 8192),
                                   (2048, 256, 2048), (129, 33, 129), (640, 384, 1024),
                                   (1000, 8, 1000), (2048, 16, 4096)])
@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
def test_fp32_tensor_core_products(M, N, K, ta, tb):
    if M * N * K > 2e10 and (ta, tb) != (False, False):
        pytest.skip("one transpose combination at the largest size is enough")
    assert _run(M, N, K, ta, tb, 1.0, 0.0, torch.float32) <= 1e-6


@pytest.mark.parametrize("M,N,K,beta,alpha", [(512, 512, 512, 1.0, 1.0), (1000, 96, 333, 1.0, -0.5),
                                              (256, 256, 4096, 0.5, 2.0)])
def test_fp32_accumulate(M, N, K, beta, alpha):
    assert _run(M, N, K, False, False, alpha, beta, torch.float32, seed=1) <= 1e-6


@pytest.mark.parametrize("M,N,K", [(64, 2, 8192), (100, 7, 50), (127, 31, 127), (1, 1, 1)])
def test_fp32_cuda_core_products(M, N, K):
    # plain FP32 accumulation in 64-deep split-K blocks, summed in order
    assert _run(M, N, K, False, True, 1.0, 0.0, torch.float32, seed=2) <= 2e-6


@pytest.mark.parametrize("M,N,K", [(256, 256, 256), (300, 77, 1030), (64, 2, 4096), (513, 129, 9)])
@pytest.mark.parametrize("ta,tb", [(False, False), (True, True)])
def test_fp64_products(M, N, K, ta, tb):
    assert _run(M, N, K, ta, tb, 1.0, 1.0, torch.float64, seed=3) <= 1e-13


def test_empty_and_errors():
    from paper_1403_6968_gb300 import LinviewError, gemm
    z = torch.zeros((0, 5), device="cuda")
    gemm(z, torch.zeros((5, 4), device="cuda"), torch.zeros((0, 4), device="cuda"))  # no work
    with pytest.raises(ValueError):
        gemm(torch.zeros((3, 5), device="cuda"), torch.zeros((4, 4), device="cuda"),
             torch.zeros((3, 4), device="cuda"))
    with pytest.raises(LinviewError):
        from paper_1403_6968_gb300 import _lib as L
        import ctypes as C
        L.call("linview_gemm", L.F32, 0, 0, 4, 4, 0, 1.0, C.c_void_p(1), 4, C.c_void_p(1), 4, 0.0,
               C.c_void_p(1), 4, None)
