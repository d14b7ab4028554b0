"""GB300-native fast multipole method for the 3-D Laplace kernel.

A from-scratch single-GPU implementation of the FMM of Yokota & Barba,
"A Tuned and Scalable Fast Multipole Method as a Preeminent Algorithm for
Exascale Systems" (arXiv:1106.2176): Morton octree, P2M/M2M/M2L/L2L/L2P over
spherical-harmonic expansions and the P2P near field, as hand-written CUDA for
sm_103a behind the C ABI of include/fmm.h.
"""
from .fmm import FMM, FMMError, unscale  # noqa: F401
