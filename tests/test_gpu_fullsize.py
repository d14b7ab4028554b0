"""GPU FMM at the full sizes of the precision and scale workloads, in the launch
configuration the bench times, against the oracle's FP64 direct sum on seeded
sampled targets (the oracle computes each sampled output alone):

- N = 10^6 uniform cube, charges U[-1,1], p = 10, theta = 0.4, ncrit = 64:
  FP64 GPU FMM and mixed precision, 4,096 targets;
- N = 10^7 uniform cube, FP32 positions and charges, p = 8, theta = 0.5,
  ncrit = 128, FP64 and mixed precision, 4,096 targets;
- N = 10^8 uniform cube, the same parameters (the largest scale size), FP64
  and mixed precision, 1,024 targets (the oracle's sampled direct sum over
  10^8 sources is the cost here).

Tolerance (the bound the method states for a mixed-precision path): the mixed
result stays within the FP64 FMM's own truncation error on the same targets
plus 2e-6 of the direct sum; every result is inside the 1e-4 error budget."""
import numpy as np
import pytest

import oracle
from paper_1106_2176_gb300 import inputs

from gpu_common import rel, run_fmm

pytestmark = pytest.mark.gpu

MIXED_SLACK = 2e-6


def _check_pair(x, q, t, P, theta, ncrit, dtype):
    """FP64 and mixed GPU FMM on the same input; both against the oracle's
    direct sum on targets t. Returns the two error pairs and the mixed stats."""
    pd, gd = oracle.direct(np.asarray(x, np.float64), np.asarray(q, np.float64), targets=t)
    p64, g64, f64 = run_fmm(x, q, P, theta, ncrit, precision="fp64", dtype=np.float64)
    assert f64.stats()["async_error"] == 0
    f64.close()
    e64 = rel(p64[t], pd), rel(g64[t], gd)
    del p64, g64
    pm, gm, fm = run_fmm(x, q, P, theta, ncrit, precision="mixed", dtype=dtype)
    st = fm.stats()
    fm.close()
    em = rel(pm[t], pd), rel(gm[t], gd)
    assert st["async_error"] == 0
    assert e64[0] < 1e-4 and e64[1] < 1e-4
    assert em[0] <= e64[0] + MIXED_SLACK and em[1] <= e64[1] + MIXED_SLACK, (em, e64)
    return e64, em, st


def test_precision_workload_1e6():
    n = 1_000_000
    x, q = inputs.uniform_cube(n, 1)
    t = inputs.sample_targets(n, 4096, seed=2)
    _check_pair(x, q, t, 10, 0.4, 64, np.float64)


def test_scale_workload_1e7_launch_configuration():
    n = 10_000_000
    x, q = inputs.uniform_cube(n, 3, dtype=np.float32)
    t = inputs.sample_targets(n, 4096, seed=3)
    _, _, st = _check_pair(x, q, t, 8, 0.5, 128, np.float32)
    assert st["depth"] == 6 and st["nleaves"] == 262144


def test_scale_workload_1e8():
    # N = 10^8 uniform cube, FP32 positions and charges, p = 8, theta = 0.5,
    # ncrit = 128: a full octree of depth 7 (2,097,152 leaves of 47.7
    # particles), fast list path
    n = 100_000_000
    x, q = inputs.uniform_cube(n, 5, dtype=np.float32)
    t = inputs.sample_targets(n, 1024, seed=6)
    _, _, st = _check_pair(x, q, t, 8, 0.5, 128, np.float32)
    assert st["depth"] == 7 and st["nleaves"] == 8 ** 7 and st["uniform_path"] == 1
