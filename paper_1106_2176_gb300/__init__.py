"""GB300-native fast multipole method for the 3-D Laplace kernel.

A from-scratch single-GPU implementation of the FMM of Yokota & Barba,
"A Tuned and Scalable Fast Multipole Method as a Preeminent Algorithm for
Exascale Systems" (arXiv:1106.2176): Morton octree, P2M/M2M/M2L/L2L/L2P over
spherical-harmonic expansions and the P2P near field, as hand-written CUDA for
sm_103a behind the C ABI of include/fmm.h.

    import torch
    from paper_1106_2176_gb300 import FMM
    f = FMM(n, p=8, theta=0.5, ncrit=128, precision="mixed")
    f.build(x, q)                # x (n, 3), q (n,): CUDA tensors (or numpy arrays)
    phi, grad = f.evaluate()     # potential and gradient, input order

Also: ``FMM(..., m2l_engine="tensor" | "cudacore" | "rotation")``,
``batch.FMMBatch`` (many systems in one CUDA graph), ``autograd.fmm_energy``
(weighted energy with gradients for x, q and w), ``tune.tune_ncrit`` (leaf
size) and ``fmm.m2l_rotation_host`` (one rotation M2L on the host).
"""
from .fmm import FMM, FMMError  # noqa: F401
