"""GB300-native LINVIEW: incremental maintenance of iterative linear-algebra
programs under factored low-rank updates (arXiv 1403.6968).

The computation lives in ``liblinview.so`` (hand-written sm_103a CUDA behind
the C ABI in ``include/linview.h``); ``linview`` is a thin ctypes binding that
marshals torch tensors and streams.  Build with ``python -m
paper_1403_6968_gb300.build``.
"""
from .linview import (Program, LinviewError, Server, level_pass, level_pass_noalloc,  # noqa: F401
                      estimate_device_bytes, program_device_bytes, check_bounded_wait, gemm)
from . import _lib  # noqa: F401
