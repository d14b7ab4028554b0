"""FP64 CPU oracle of the 3-D Laplace FMM (Yokota & Barba, arXiv:1106.2176).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import this package. It shares no code
with the GPU library in ``paper_1106_2176_gb300``; both sides take their inputs
from the seeded generators in ``paper_1106_2176_gb300.inputs`` only.

The arithmetic lives in ``oracle.c`` (plain C, FP64, no FMA contraction); this
module compiles it with gcc and wraps it with ctypes and numpy.
"""
from .oracle import (  # noqa: F401
    build,
    lib,
    direct,
    regular,
    irregular,
    p2m,
    m2m,
    m2l,
    l2l,
    l2p,
    Tree,
    fmm,
    nm,
    set_threads,
    get_threads,
)
