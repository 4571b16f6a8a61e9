"""Thin Python binding of the LINVIEW C ABI (argument marshalling only).

Every computation runs in the CUDA library (``liblinview.so``); this module
turns torch tensors / numpy arrays into pointers, leading dimensions and the
current CUDA stream, and raises ``LinviewError`` on a non-OK status.
PyTorch provides device memory and streams.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L
from ._lib import LinviewError  # noqa: F401

KINDS = {"power": L.POWER, "power_sum": L.POWER_SUM, "iteration": L.ITERATION, "ols": L.OLS}
MODELS = {"exp": L.MODEL_EXP, "linear": L.MODEL_LINEAR, "skip": L.MODEL_SKIP}
STRATEGIES = {"factored": L.STRATEGY_FACTORED, "hybrid": L.STRATEGY_HYBRID}
CORRECTIONS = {"reeval": L.CORRECT_REEVAL, "newton": L.CORRECT_NEWTON}
REEVAL = {"default": L.REEVAL_DEFAULT, "fp32": L.REEVAL_FP32, "tf32": L.REEVAL_TF32,
          "bf16x9": L.REEVAL_BF16X9, "fp64": L.REEVAL_FP64, "tc3": L.REEVAL_TC3}


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


_TORCH_CB = None
_LIVE = None


def _torch_allocator():
    """The (alloc, free) callbacks that hand a program's device memory to
    PyTorch's caching allocator (module-level, so they outlive every program).
    ``alloc_ctx`` carries the device index + 1."""
    global _TORCH_CB
    if _TORCH_CB is None:
        torch = _torch()

        def alloc(nbytes, stream, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), device=int(ctx or 1) - 1,
                                                          stream=int(stream or 0))
            except Exception:  # out of memory: the library reports ENOMEM
                return None

        def free(ptr, nbytes, stream, ctx):
            try:
                torch.cuda.caching_allocator_delete(int(ptr))
            except Exception:
                pass

        _TORCH_CB = (L.ALLOC_FN(alloc), L.FREE_FN(free))
    return _TORCH_CB


def _track(prog):
    """Programs whose memory belongs to PyTorch are destroyed at exit, while
    PyTorch can still take the memory back."""
    global _LIVE
    import atexit
    import weakref
    if _LIVE is None:
        _LIVE = weakref.WeakSet()

        def close_all():
            for pr in list(_LIVE):
                try:
                    pr.close()
                except Exception:
                    pass
        atexit.register(close_all)
    _LIVE.add(prog)


def _dtype_of(precision):
    return np.float64 if precision == L.F64 else np.float32


class _Operand:
    """A 2-D row-major operand: (pointer, ld, on_device, keepalive)."""

    def __init__(self, x, np_dtype):
        torch = _torch()
        if isinstance(x, torch.Tensor):
            want = torch.float64 if np_dtype == np.float64 else torch.float32
            if x.dtype != want:
                raise TypeError(f"expected {want}, got {x.dtype}")
            if x.dim() == 1:
                x = x.reshape(-1, 1)
            if x.stride(1) != 1:
                x = x.contiguous()
            self.keep = x
            self.ptr = C.c_void_p(x.data_ptr())
            self.ld = x.stride(0) if x.shape[0] > 1 else x.shape[1]
            self.on_device = 1 if x.is_cuda else 0
            self.shape = tuple(x.shape)
        else:
            a = np.asarray(x)
            if a.dtype != np_dtype:
                raise TypeError(f"expected {np_dtype}, got {a.dtype}")
            if a.ndim == 1:
                a = a.reshape(-1, 1)
            a = np.ascontiguousarray(a)
            self.keep = a
            self.ptr = C.c_void_p(a.ctypes.data)
            self.ld = a.shape[1]
            self.on_device = 0
            self.shape = a.shape


class Program:
    """A maintained program (powers, sums of powers, iteration, OLS).

    ``inputs`` are torch tensors (CUDA or CPU) or numpy arrays, all of the
    program's element type (float32 or float64).  ``allocator="torch"`` (the
    default) gives the program's device memory to PyTorch's caching allocator
    through the descriptor's alloc/free callbacks (so ``torch.cuda.
    memory_allocated()`` counts it); ``allocator=None`` lets the library call
    cudaMalloc itself.
    """

    def __init__(self, kind, inputs, k, r_max=1, precision="f32", p=0, m=0,
                 correction_period=0, reeval_mode="default", model=None, skip=0,
                 strategy="factored", stream=None, allocator="torch", correction="reeval"):
        self.lib = L.load()
        self.precision = L.F64 if precision in ("f64", "fp64", L.F64) else L.F32
        self.np_dtype = _dtype_of(self.precision)
        ops = [_Operand(x, self.np_dtype) for x in inputs]
        d = L.ProgramDesc()
        d.kind = KINDS[kind] if isinstance(kind, str) else int(kind)
        d.precision = self.precision
        d.n = ops[0].shape[1] if d.kind != L.OLS else ops[0].shape[1]
        d.m = m if m else (ops[0].shape[0] if d.kind == L.OLS else 0)
        d.p = p if p else (ops[1].shape[1] if d.kind in (L.ITERATION, L.OLS) else 0)
        d.k = int(k)
        d.r_max = int(r_max)
        d.correction_period = int(correction_period)
        d.reeval_mode = REEVAL[reeval_mode] if isinstance(reeval_mode, str) else int(reeval_mode)
        if model is None:  # iteration programs default to the linear model (views T_1..T_k)
            model = "linear" if d.kind == L.ITERATION else "exp"
        d.model = MODELS[model] if isinstance(model, str) else int(model)
        d.skip = int(skip)
        d.strategy = STRATEGIES[strategy] if isinstance(strategy, str) else int(strategy)
        d.correction = CORRECTIONS[correction] if isinstance(correction, str) else int(correction)
        # the library reads each input in place with these shapes
        want = {L.POWER: [(d.n, d.n)], L.POWER_SUM: [(d.n, d.n)],
                L.ITERATION: [(d.n, d.n), (d.n, d.p), (d.n, d.p)],
                L.OLS: [(d.m, d.n), (d.m, d.p)]}.get(d.kind)
        if want is not None and (len(ops) != len(want) or
                                 any(tuple(o.shape) != w for o, w in zip(ops, want))):
            raise ValueError(f"{kind} inputs must have shapes {want}, got "
                             f"{[tuple(o.shape) for o in ops]}")
        if allocator == "torch":
            torch = _torch()
            fa, ff = _torch_allocator()
            d.alloc = C.cast(fa, C.c_void_p).value
            d.free = C.cast(ff, C.c_void_p).value
            d.alloc_ctx = torch.cuda.current_device() + 1
        elif allocator is not None:
            raise ValueError("allocator must be 'torch' or None")
        on_dev = {o.on_device for o in ops}
        if len(on_dev) != 1:
            raise ValueError("inputs must all be on the device or all on the host")
        ptrs = (C.c_void_p * len(ops))(*[o.ptr for o in ops])
        lds = (C.c_int64 * len(ops))(*[o.ld for o in ops])
        h = C.c_void_p()
        L.call("linview_create_program", C.byref(d), ptrs, lds, on_dev.pop(), _stream_ptr(stream),
               C.byref(h))
        self.h = h
        self.desc = d
        self.device_index = _torch().cuda.current_device() if _torch().cuda.is_available() else 0
        if allocator == "torch":
            _track(self)
        self.n = d.n
        self.k = d.k

    # -- updates -----------------------------------------------------------
    def _check_tensor(self, t, shape, name, device_only=True):
        """A tensor the library reads or writes through a raw pointer: the
        program's dtype, unit inner stride, exactly ``shape``, and a CUDA
        tensor on the program's device (or host memory where allowed)."""
        torch = _torch()
        want = torch.float64 if self.precision == L.F64 else torch.float32
        if not isinstance(t, torch.Tensor) or t.dim() != 2:
            raise ValueError(f"{name} must be a 2-D tensor")
        if t.dtype != want:
            raise ValueError(f"{name} has dtype {t.dtype}, the program computes in {want}")
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} must be {tuple(shape)}, got {tuple(t.shape)}")
        if t.shape[0] > 0 and t.shape[1] > 0 and t.stride(1) != 1:
            raise ValueError(f"{name} must have unit inner stride")
        if t.is_cuda:
            if t.device.index != self.device_index:
                raise ValueError(f"{name} is on {t.device}, the program on cuda:{self.device_index}")
        elif device_only:
            raise ValueError(f"{name} must be a CUDA tensor")

    def _check_side(self, *ops):
        """Operands the library reads on the device: CUDA tensors on this
        program's device (a wrong shape or device would become an
        out-of-bounds access there instead of an error here)."""
        for o in ops:
            if o.on_device and o.keep.device.index != self.device_index:
                raise ValueError(f"operand on {o.keep.device}, program on cuda:{self.device_index}")

    def apply_delta(self, U, V, input_id=0, stream=None):
        """dX = U V^T for input ``input_id``: U is n x rank; V is n x rank for
        A (input 0) and p x rank for B (input 1 of an iteration program)."""
        u = _Operand(U, self.np_dtype)
        v = _Operand(V, self.np_dtype)
        if u.on_device != v.on_device:
            raise ValueError("U and V must be on the same side")
        if len(u.shape) != 2 or len(v.shape) != 2 or u.shape[1] != v.shape[1]:
            raise ValueError(f"U and V must be 2-D with the same rank, got {u.shape}, {v.shape}")
        v_rows = self.desc.p if (int(input_id) == 1 and self.desc.kind == L.ITERATION) else self.n
        if u.shape[0] != self.n or v.shape[0] != v_rows:
            raise ValueError(f"U must be {self.n} x rank and V {v_rows} x rank, "
                             f"got {u.shape}, {v.shape}")
        self._check_side(u, v)
        L.call("linview_apply_delta", self.h, input_id, u.shape[1], u.ptr, u.ld, v.ptr, v.ld,
               u.on_device, _stream_ptr(stream))

    def apply_row_delta(self, row, v, input_id=0, stream=None):
        o = _Operand(v, self.np_dtype)
        if o.shape[0] * o.shape[1] != self.n:
            raise ValueError(f"v must have n = {self.n} entries, got shape {o.shape}")
        self._check_side(o)
        L.call("linview_apply_row_delta", self.h, input_id, int(row), o.ptr, o.on_device,
               _stream_ptr(stream))

    def apply_row_block(self, rows, new_rows, stream=None):
        rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
        o = _Operand(new_rows, self.np_dtype)
        if o.shape != (len(rows), self.n):
            raise ValueError(f"new_rows must be {len(rows)} x {self.n}, got {o.shape}")
        self._check_side(o)
        L.call("linview_apply_row_block", self.h, len(rows),
               rows.ctypes.data_as(C.POINTER(C.c_int64)), o.ptr, o.ld, o.on_device,
               _stream_ptr(stream))

    # -- views -------------------------------------------------------------
    def num_views(self):
        return self.lib.linview_num_views(self.h)

    def view_shape(self, vid):
        r, c = C.c_int64(), C.c_int64()
        L.call("linview_view_shape", self.h, int(vid), C.byref(r), C.byref(c))
        return r.value, c.value

    def read_view(self, vid, out=None, stream=None):
        """Copy view ``vid`` into a new (or given) CUDA tensor."""
        torch = _torch()
        rows, cols = self.view_shape(vid)
        if out is None:
            dt = torch.float64 if self.precision == L.F64 else torch.float32
            out = torch.empty((rows, cols), dtype=dt, device="cuda")
        self._check_tensor(out, (rows, cols), "out", device_only=False)
        L.call("linview_read_view", self.h, int(vid), C.c_void_p(out.data_ptr()), out.stride(0),
               1 if out.is_cuda else 0, _stream_ptr(stream))
        return out

    def read_view_rows(self, vid, row0, nrows, out=None, stream=None, sync=True):
        """Rows [row0, row0+nrows) of a view into ``out`` (numpy or torch; host
        or device); returns ``out``.  A host ``out`` is ready on return unless
        ``sync`` is False: then the copy is queued on the stream and the caller
        synchronises the stream (or an event recorded after the call) before
        reading ``out``, which must stay alive until then (a pinned tensor lets
        the copy overlap later work)."""
        rows, cols = self.view_shape(vid)
        if out is None:
            out = np.empty((nrows, cols), dtype=self.np_dtype)
        o = _Operand(out, self.np_dtype)
        if o.keep is not out and not (hasattr(out, "data_ptr") and
                                      o.keep.data_ptr() == out.data_ptr()):
            raise ValueError("out must be a contiguous row-major array")
        if tuple(o.shape) != (int(nrows), cols):
            raise ValueError(f"out must be {(int(nrows), cols)}, got {tuple(o.shape)}")
        self._check_side(o)
        dst = o.on_device if (o.on_device or sync) else L.DST_HOST_ASYNC
        L.call("linview_read_view_rows", self.h, int(vid), int(row0), int(nrows), o.ptr, o.ld,
               dst, _stream_ptr(stream))
        return out

    def read_view_host(self, vid, stream=None):
        rows, cols = self.view_shape(vid)
        out = np.empty((rows, cols), dtype=self.np_dtype)
        L.call("linview_read_view", self.h, int(vid), C.c_void_p(out.ctypes.data), cols, 0,
               _stream_ptr(stream))
        return out

    # -- strategies and status --------------------------------------------
    def reeval(self, stream=None):
        L.call("linview_reeval", self.h, _stream_ptr(stream))

    def correct(self, stream=None):
        """The program's residual correction now (``correction``): re-evaluation,
        or for an FP32 OLS program created with correction="newton" one
        Newton-Schulz step W <- W + W (I - Z W) from the maintained Z = X^T X."""
        L.call("linview_correct", self.h, _stream_ptr(stream))

    def set_reeval_mode(self, mode):
        L.call("linview_set_reeval_mode", self.h, REEVAL[mode] if isinstance(mode, str) else mode)

    def prepare_updates(self, max_rank=None, stream=None):
        """Capture the propagation graphs of update ranks 1..max_rank (default
        r_max) now, so that no first update of a rank pays for the capture."""
        r = self.desc.r_max if max_rank is None else int(max_rank)
        L.call("linview_prepare_updates", self.h, r, _stream_ptr(stream))

    def sync(self, stream=None):
        L.call("linview_sync", self.h, _stream_ptr(stream))

    # -- adjoints ----------------------------------------------------------
    def adjoint_iteration(self, dA=None, dB=None, stream=None):
        n, p = self.n, self.desc.p
        if dA is not None:
            self._check_tensor(dA, (n, n), "dA")
        if dB is not None:
            self._check_tensor(dB, (n, p), "dB")
        pa = C.c_void_p(dA.data_ptr()) if dA is not None else None
        pb = C.c_void_p(dB.data_ptr()) if dB is not None else None
        L.call("linview_adjoint_iteration", self.h, pa, dA.stride(0) if dA is not None else 0,
               pb, dB.stride(0) if dB is not None else 0, _stream_ptr(stream))

    def adjoint_iteration_seed(self, Gk, dA=None, dB=None, dT0=None, stream=None):
        """Vector-Jacobian product of (A, B, T_0) -> T_k at dL/dT_k = Gk (CUDA tensors)."""
        n, p = self.n, self.desc.p
        self._check_tensor(Gk, (n, p), "Gk")
        for t, shape, name in ((dA, (n, n), "dA"), (dB, (n, p), "dB"), (dT0, (n, p), "dT0")):
            if t is not None:
                self._check_tensor(t, shape, name)

        def ptr(t):
            return (C.c_void_p(t.data_ptr()), t.stride(0)) if t is not None else (None, 0)
        (pa, la), (pb, lb), (pt, lt) = ptr(dA), ptr(dB), ptr(dT0)
        L.call("linview_adjoint_iteration_seed", self.h, C.c_void_p(Gk.data_ptr()), Gk.stride(0),
               pa, la, pb, lb, pt, lt, _stream_ptr(stream))

    def adjoint_power(self, G, dA, stream=None):
        self._check_tensor(G, (self.n, self.n), "G")
        self._check_tensor(dA, (self.n, self.n), "dA")
        L.call("linview_adjoint_power", self.h, C.c_void_p(G.data_ptr()), G.stride(0),
               C.c_void_p(dA.data_ptr()), dA.stride(0), _stream_ptr(stream))

    # -- measurement -------------------------------------------------------
    def set_profiling(self, on=True):
        L.call("linview_set_profiling", self.h, 1 if on else 0)

    def reset_stats(self):
        L.call("linview_reset_stats", self.h)

    def pass_stats(self, kernel=0):
        """kernel: 0 all view passes, 1 fused products+update pass, 2 update-only pass."""
        n, ms, b, al = C.c_int64(), C.c_double(), C.c_double(), C.c_int64()
        L.call("linview_pass_stats", self.h, int(kernel), C.byref(n), C.byref(ms), C.byref(b),
               C.byref(al))
        return {"launches": n.value, "ms": ms.value, "bytes": b.value, "all_launches": al.value}

    def view_device_ptr(self, vid):
        ptr, ld = C.c_void_p(), C.c_int64()
        L.call("linview_view_device_ptr", self.h, int(vid), C.byref(ptr), C.byref(ld))
        return ptr.value, ld.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.linview_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check_pass_operands(P, U, V, X, Y):
    """Host-side checks of a level pass's operands, before any launch: P is a
    2-D CUDA float32/float64 tensor with unit inner stride and at least
    P.shape[0] columns; U, V (and X, Y when given) are r x n row-major CUDA
    tensors (each row one factor column) on P's device, of P's dtype, with
    unit inner stride, n = P.shape[0] columns at least and one common row
    stride.  Raises ValueError, so that a wrong call never becomes an
    out-of-bounds device access.  Returns (n, r, ldf)."""
    if getattr(P, "dim", lambda: 0)() != 2:
        raise ValueError("P must be a 2-D tensor")
    if not P.is_cuda:
        raise ValueError("P must be a CUDA tensor")
    if str(P.dtype) not in ("torch.float32", "torch.float64"):
        raise ValueError(f"P must be float32 or float64, got {P.dtype}")
    n = P.shape[0]
    if n < 1 or P.shape[1] < n:
        raise ValueError(f"P must be n x n (n >= 1), got {tuple(P.shape)}")
    if P.stride(1) != 1:
        raise ValueError("P must have unit inner stride (row-major)")
    if getattr(U, "dim", lambda: 0)() != 2:
        raise ValueError("U must be a 2-D (r, n) tensor")
    r = U.shape[0]
    ldf = U.stride(0)
    for name, t in (("U", U), ("V", V), ("X", X), ("Y", Y)):
        if t is None:
            if name in ("U", "V"):
                raise ValueError(f"{name} is required")
            continue
        if t.dim() != 2:
            raise ValueError(f"{name} must be a 2-D (r, n) tensor")
        if not t.is_cuda or t.device != P.device:
            raise ValueError(f"{name} must be a CUDA tensor on P's device ({P.device})")
        if t.dtype != P.dtype:
            raise ValueError(f"{name} has dtype {t.dtype}, P has {P.dtype}")
        if t.stride(1) != 1:
            raise ValueError(f"{name} must have unit inner stride")
        if t.shape[0] != r or t.stride(0) != ldf:
            raise ValueError("U, V, X, Y must share shape (r, n) and row stride")
        if t.shape[1] < n:
            raise ValueError(f"{name} has {t.shape[1]} columns, fewer than n = {n}")
    return n, r, ldf


def level_pass(P, U, V, X=None, Y=None, do_update=True, stream=None):
    """One exponential-model level pass on caller tensors (all CUDA).

    P: n x n (row-major); U, V, X, Y: column-major n x r given as r x n
    row-major tensors (each row one factor column, i.e. U_cm = U.T)."""
    torch = _torch()
    n, r, ldf = _check_pass_operands(P, U, V, X, Y)
    prec = L.F64 if P.dtype == torch.float64 else L.F32
    L.call("linview_level_pass", prec, n, C.c_void_p(P.data_ptr()), P.stride(0),
           C.c_void_p(U.data_ptr()), C.c_void_p(V.data_ptr()), ldf, r,
           C.c_void_p(X.data_ptr()) if X is not None else None,
           C.c_void_p(Y.data_ptr()) if Y is not None else None,
           1 if do_update else 0, _stream_ptr(stream))


def gemm(a, b, c, alpha=1.0, beta=0.0, ta=False, tb=False, stream=None):
    """c = alpha op(a) op(b) + beta c with the library's own GEMM (CUDA
    tensors, row-major, float32 or float64, unit inner stride)."""
    torch = _torch()
    for name, t in (("a", a), ("b", b), ("c", c)):
        if t.dim() != 2 or not t.is_cuda or t.stride(1) != 1 or t.dtype != c.dtype:
            raise ValueError(f"{name} must be a 2-D CUDA tensor of c's dtype with unit inner stride")
        if t.device != c.device:
            raise ValueError(f"{name} is not on c's device")
    M, N = c.shape
    K = a.shape[0] if ta else a.shape[1]
    if (a.shape[1] if ta else a.shape[0]) != M or (b.shape[1] if tb else b.shape[0]) != K or \
            (b.shape[0] if tb else b.shape[1]) != N:
        raise ValueError("shapes of op(a), op(b) and c do not match")
    prec = L.F64 if c.dtype == torch.float64 else L.F32
    L.call("linview_gemm", prec, int(ta), int(tb), M, N, K, float(alpha),
           C.c_void_p(a.data_ptr()), a.stride(0), C.c_void_p(b.data_ptr()), b.stride(0),
           float(beta), C.c_void_p(c.data_ptr()), c.stride(0), _stream_ptr(stream))


def check_bounded_wait(limit_ns=20_000_000, stream=None):
    """Run the library's bounded-wait diagnostic (a device wait on a barrier
    that never completes, limit ``limit_ns``).  Returns the time the wait took
    in ns once it gave up and latched its timeout, the expected outcome;
    raises LinviewError on anything else."""
    w = C.c_int64()
    st = L.load().linview_check_bounded_wait(int(limit_ns), _stream_ptr(stream), C.byref(w))
    if st != L.ETIMEOUT:
        L.check(st, "linview_check_bounded_wait")
        raise LinviewError(st, "linview_check_bounded_wait", "the wait did not expire")
    return w.value


def level_pass_noalloc(P, U, V, X=None, Y=None, do_update=True, stream=None):
    """``level_pass`` for callers that may not allocate device memory: the
    partial sums use the library's built-in 16 MiB device array instead of
    stream-ordered allocations (see linview_level_pass_noalloc in
    include/linview.h for the size limit and the rule that overlapping calls
    must be serialised)."""
    torch = _torch()
    n, r, ldf = _check_pass_operands(P, U, V, X, Y)
    prec = L.F64 if P.dtype == torch.float64 else L.F32
    L.call("linview_level_pass_noalloc", prec, n, C.c_void_p(P.data_ptr()), P.stride(0),
           C.c_void_p(U.data_ptr()), C.c_void_p(V.data_ptr()), ldf, r,
           C.c_void_p(X.data_ptr()) if X is not None else None,
           C.c_void_p(Y.data_ptr()) if Y is not None else None,
           1 if do_update else 0, _stream_ptr(stream))


def estimate_device_bytes(n, k, r_max=1, kind="power", precision="f32", model="exp", skip=0):
    """Device bytes a power (or power-sum) program of this shape would hold."""
    d = L.ProgramDesc()
    d.kind = KINDS[kind]
    d.model = MODELS[model]
    d.skip = int(skip)
    d.precision = L.F64 if precision in ("f64", "fp64") else L.F32
    d.n, d.k, d.r_max = int(n), int(k), int(r_max)
    b = C.c_int64()
    L.call("linview_estimate_device_bytes", C.byref(d), C.byref(b))
    return b.value


def program_device_bytes(prog):
    b = C.c_int64()
    L.call("linview_program_device_bytes", prog.h, C.byref(b))
    return b.value


class _ServedProgram(Program):
    """A server-owned program: views can be read, the server frees it."""

    def __init__(self, handle, n, k):
        self.lib = L.load()
        self.h = C.c_void_p(handle)
        self.precision = L.F32
        self.np_dtype = np.float32
        self.n, self.k = n, k
        self.device_index = _torch().cuda.current_device()

    def _refuse(self, *a, **kw):
        raise RuntimeError("a served view is updated through Server.submit / submit_row "
                           "(the server's scheduler thread issues its work)")

    apply_delta = apply_row_delta = apply_row_block = _refuse

    def close(self):
        self.h = None


class Server:
    """Continuous-batching server of maintained A^k views (linview_server_*).

    Views and their factors stay resident on the GPU; requests dA = U V^T
    are queued per view, coalesced while the view is busy, and refreshed on
    per-view streams by the library's scheduler thread."""

    def __init__(self, max_inflight=4, r_cap=8, hbm_budget_bytes=0):
        L.load()
        h = C.c_void_p()
        L.call("linview_server_create", int(hbm_budget_bytes), int(max_inflight), int(r_cap),
               C.byref(h))
        self.h = h
        self.r_cap = r_cap
        self._n = {}
        self._keep = []

    def add_view(self, A, k):
        a = _Operand(A, np.float32)
        if len(a.shape) != 2 or a.shape[0] != a.shape[1]:
            raise ValueError(f"A must be square, got {a.shape}")
        if a.on_device:  # the server reads A on its own stream
            _torch().cuda.current_stream().synchronize()
        v = C.c_int32()
        L.call("linview_server_add_view", self.h, a.shape[0], int(k), a.ptr, a.ld, a.on_device,
               C.byref(v))
        self._n[v.value] = (a.shape[0], int(k))
        return v.value

    def submit(self, view, U, V, arrival_s=-1.0):
        """Request dA = U V^T (U, V: n x rank).  Up to r_cap columns it
        coalesces with the view's queued requests; a wider request is served
        by re-evaluation together with everything queued for the view."""
        u = np.ascontiguousarray(np.asarray(U, dtype=np.float32))
        w = np.ascontiguousarray(np.asarray(V, dtype=np.float32))
        if u.ndim == 1:
            u, w = u.reshape(-1, 1), w.reshape(-1, 1)
        n = self._n.get(int(view), (None,))[0]
        if u.ndim != 2 or u.shape != w.shape or (n is not None and u.shape[0] != n):
            raise ValueError(f"U and V must both be n x rank (n = {n}), got {u.shape}, {w.shape}")
        t = C.c_uint64()
        L.call("linview_server_submit", self.h, int(view), u.shape[1], C.c_void_p(u.ctypes.data),
               u.shape[1], C.c_void_p(w.ctypes.data), w.shape[1], float(arrival_s), C.byref(t))
        return t.value

    def submit_row(self, view, row, v, arrival_s=-1.0):
        """Row update dA = e_row v^T (coalesced by row with other queued ones)."""
        w = np.ascontiguousarray(np.asarray(v, dtype=np.float32).reshape(-1))
        n = self._n.get(int(view), (None,))[0]
        if n is not None and w.shape[0] != n:
            raise ValueError(f"v must have n = {n} entries, got {w.shape[0]}")
        t = C.c_uint64()
        L.call("linview_server_submit_row", self.h, int(view), int(row),
               C.c_void_p(w.ctypes.data), float(arrival_s), C.byref(t))
        return t.value

    def replay(self, t_s, views, ranks, factors, offsets, rows=None):
        """Open-loop load: request i at t_s[i] seconds after the call; its U
        (n x rank, row-major) at factors[offsets[i]:], V right after it; with
        ``rows`` given and rows[i] >= 0, the row update e_rows[i] v^T with v
        at factors[offsets[i]:].  ``factors`` must stay alive until ``drain``
        returns."""
        t_s = np.ascontiguousarray(t_s, dtype=np.float64)
        views = np.ascontiguousarray(views, dtype=np.int32)
        ranks = np.ascontiguousarray(ranks, dtype=np.int32)
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        rows_a = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
        if factors.dtype != np.float32 or not factors.flags.c_contiguous:
            raise TypeError("factors must be a contiguous float32 array")
        m = len(t_s)
        if not (len(views) == len(ranks) == len(offsets) == m) or \
                (rows_a is not None and len(rows_a) != m):
            raise ValueError("t_s, views, ranks, offsets (and rows) must have one entry per request")
        # every request's factors lie inside ``factors`` (the library reads
        # them in place): n floats for a row update, 2 n rank otherwise
        nv = np.array([self._n.get(int(v), (0,))[0] for v in views], dtype=np.int64)
        is_row = np.zeros(m, bool) if rows_a is None else rows_a >= 0
        need = np.where(is_row, nv, 2 * nv * ranks.astype(np.int64))
        if m and (np.any(offsets < 0) or np.any(offsets + need > factors.size)):
            raise ValueError("a request's factors reach past the end of ``factors``")
        self._keep.append(factors)
        L.call("linview_server_replay", self.h, len(t_s), C.c_void_p(t_s.ctypes.data),
               C.c_void_p(views.ctypes.data), C.c_void_p(ranks.ctypes.data),
               C.c_void_p(factors.ctypes.data), C.c_void_p(offsets.ctypes.data),
               None if rows_a is None else C.c_void_p(rows_a.ctypes.data))

    def drain(self, timeout_s=0.0):
        L.call("linview_server_drain", self.h, float(timeout_s))
        self._keep.clear()

    def poll(self, max_records=4096):
        """Completion records as a list of dicts (oldest first)."""
        buf = (L.Completion * max_records)()
        cnt = C.c_int32()
        out = []
        while True:
            L.call("linview_server_poll", self.h, C.cast(buf, C.c_void_p), max_records, C.byref(cnt))
            for i in range(cnt.value):
                c = buf[i]
                out.append({f: getattr(c, f) for f, _ in L.Completion._fields_ if f != "reserved"})
            if cnt.value < max_records:
                return out

    def view_state(self, view):
        st = C.c_int32()
        L.call("linview_server_view_state", self.h, int(view), C.byref(st))
        return ("waiting", "resident", "removed")[st.value]

    def program(self, view):
        """The resident view's program (read its views after ``drain``)."""
        h = C.c_void_p()
        L.call("linview_server_view_program", self.h, int(view), C.byref(h))
        n, k = self._n[view]
        return _ServedProgram(h.value, n, k)

    def remove_view(self, view):
        L.call("linview_server_remove_view", self.h, int(view))

    def stats(self):
        s = L.ServerStats()
        L.call("linview_server_stats_get", self.h, C.byref(s))
        return {f: getattr(s, f) for f, _ in L.ServerStats._fields_ if f != "reserved"}

    def clock(self):
        return L.load().linview_server_clock(self.h)

    def close(self):
        if getattr(self, "h", None):
            L.load().linview_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
