"""Host-side operand checks of the stand-alone level passes (no launch, no GPU).

``level_pass`` and ``level_pass_noalloc`` hand raw device pointers to the
library, which trusts the sizes it is given; every mismatch the kernels could
turn into an out-of-bounds access must be caught on the host first.  Stand-in
tensors (shape, strides, dtype, device) drive the shared checker directly.
"""
import pytest

torch = pytest.importorskip("torch")

from paper_1403_6968_gb300.linview import _check_pass_operands  # noqa: E402

CUDA0 = torch.device("cuda", 0)


class FakeT:
    """The attributes the checker reads, for a row-major 2-D tensor."""

    def __init__(self, rows, cols, dtype=torch.float32, ld=None, inner=1, device=CUDA0, ndim=2):
        self.shape = (rows, cols)
        self.dtype = dtype
        self.device = device
        self.is_cuda = device.type == "cuda"
        self._strides = (cols if ld is None else ld, inner)
        self._ndim = ndim

    def stride(self, i):
        return self._strides[i]

    def dim(self):
        return self._ndim


def ok_args(n=64, r=4, dtype=torch.float32):
    return dict(P=FakeT(n, n, dtype), U=FakeT(r, n, dtype), V=FakeT(r, n, dtype),
                X=FakeT(r, n, dtype), Y=FakeT(r, n, dtype))


def check(**kw):
    return _check_pass_operands(kw["P"], kw["U"], kw["V"], kw.get("X"), kw.get("Y"))


def test_valid_operands_pass():
    assert check(**ok_args()) == (64, 4, 64)
    a = ok_args(dtype=torch.float64)
    a["X"] = None
    a["Y"] = None
    assert check(**a) == (64, 4, 64)
    # factors may be wider than n (padded rows), P may have a padded row stride
    a = ok_args()
    a["P"] = FakeT(64, 64, ld=80)
    for k in ("U", "V", "X", "Y"):
        a[k] = FakeT(4, 72)
    assert check(**a) == (64, 4, 72)


@pytest.mark.parametrize("name,bad", [
    ("U", FakeT(4, 64, torch.float64)),                 # dtype differs from P
    ("V", FakeT(4, 64, torch.float64)),
    ("X", FakeT(4, 64, torch.float64)),
    ("Y", FakeT(4, 64, torch.float64)),
    ("U", FakeT(4, 64, device=torch.device("cpu"))),     # host tensor
    ("V", FakeT(4, 64, device=torch.device("cuda", 1))),  # another device
    ("X", FakeT(4, 64, device=torch.device("cpu"))),
    ("U", FakeT(4, 64, inner=2)),                        # non-unit inner stride
    ("Y", FakeT(4, 64, inner=4)),
    ("U", FakeT(4, 63)),                                 # short factor rows (< n)
    ("V", FakeT(4, 32)),
    ("X", FakeT(4, 63)),
    ("V", FakeT(3, 64)),                                 # rank differs from U
    ("X", FakeT(4, 64, ld=96)),                          # row stride differs from U
    ("U", FakeT(4, 64, ndim=1)),
])
def test_each_bad_factor_raises(name, bad):
    a = ok_args()
    a[name] = bad
    with pytest.raises(ValueError):
        check(**a)


@pytest.mark.parametrize("bad", [
    FakeT(64, 63),                                       # fewer columns than rows
    FakeT(64, 64, inner=2),
    FakeT(64, 64, device=torch.device("cpu")),
    FakeT(64, 64, dtype=torch.float16),
    FakeT(64, 64, ndim=3),
])
def test_bad_view_raises(bad):
    a = ok_args()
    a["P"] = bad
    with pytest.raises(ValueError):
        check(**a)


def test_missing_factor_raises():
    a = ok_args()
    a["V"] = None
    with pytest.raises(ValueError):
        check(**a)
