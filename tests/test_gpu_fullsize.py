"""GPU FMM at the full sizes of the precision and scale workloads, in the launch
configuration the bench times, against the oracle's FP64 direct sum on seeded
sampled targets (the oracle computes each sampled output alone):

- N = 10^6 uniform cube, charges U[-1,1], p = 10, theta = 0.4, ncrit = 64:
  FP64 GPU FMM and mixed precision;
- N = 10^7 uniform cube, FP32 positions and charges, p = 8, theta = 0.5,
  ncrit = 128, mixed precision;
- N = 10^8 uniform cube, the same parameters (the largest scale size).

Tolerance: the mixed path stays within the FP64 FMM's own truncation error
plus 2e-6 of the direct sum; every result within the 1e-4 error budget."""
import numpy as np
import pytest

import oracle
from paper_1106_2176_gb300 import inputs

from gpu_common import rel, run_fmm

pytestmark = pytest.mark.gpu

MIXED_SLACK = 2e-6


def test_precision_workload_1e6():
    n = 1_000_000
    x, q = inputs.uniform_cube(n, 1)
    t = inputs.sample_targets(n, 1024, seed=2)
    pd, gd = oracle.direct(x, q, targets=t)
    p64, g64, f64 = run_fmm(x, q, 10, 0.4, 64, precision="fp64", dtype=np.float64)
    pm, gm, fm = run_fmm(x, q, 10, 0.4, 64, precision="mixed", dtype=np.float64)
    e64 = rel(p64[t], pd), rel(g64[t], gd)
    em = rel(pm[t], pd), rel(gm[t], gd)
    assert fm.stats()["async_error"] == 0
    assert e64[0] < 1e-4 and e64[1] < 1e-4
    assert em[0] <= e64[0] + MIXED_SLACK and em[1] <= e64[1] + MIXED_SLACK


def test_scale_workload_1e7_launch_configuration():
    n = 10_000_000
    x, q = inputs.uniform_cube(n, 3, dtype=np.float32)
    t = inputs.sample_targets(n, 512, seed=3)
    pd, gd = oracle.direct(x.astype(np.float64), q.astype(np.float64), targets=t)
    pm, gm, fm = run_fmm(x, q, 8, 0.5, 128, precision="mixed", dtype=np.float32)
    st = fm.stats()
    assert st["async_error"] == 0 and st["depth"] == 6 and st["nleaves"] == 262144
    # p = 8, theta = 0.5 truncates at ~1e-7 (phi) and ~4e-7 (grad) on this
    # workload; the mixed path adds at most 2e-6
    assert rel(pm[t], pd) <= 1e-6 + MIXED_SLACK
    assert rel(gm[t], gd) <= 1e-6 + MIXED_SLACK


def test_scale_workload_1e8():
    # N = 10^8 uniform cube, FP32 positions and charges, p = 8, theta = 0.5,
    # ncrit = 128: a full octree of depth 7 (2,097,152 leaves of 47.7
    # particles), fast list path; 256 sampled targets against the oracle
    n = 100_000_000
    x, q = inputs.uniform_cube(n, 5, dtype=np.float32)
    t = inputs.sample_targets(n, 256, seed=6)
    pm, gm, fm = run_fmm(x, q, 8, 0.5, 128, precision="mixed", dtype=np.float32)
    st = fm.stats()
    fm.close()
    assert st["async_error"] == 0 and st["depth"] == 7 and st["nleaves"] == 8 ** 7 and st["uniform_path"] == 1
    pd, gd = oracle.direct(x.astype(np.float64), q.astype(np.float64), targets=t)
    assert rel(pm[t], pd) <= 1e-6 + MIXED_SLACK
    assert rel(gm[t], gd) <= 1e-6 + MIXED_SLACK
