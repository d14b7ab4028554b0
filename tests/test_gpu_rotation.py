"""Rotation-based M2L engine (rotate each translation onto the z axis,
translate along z, rotate back; Sec. 2.2): the FP64 FMM with it against the
oracle FMM (dense M2L, the definition), against the dense CUDA-core engine at
p = 16, where the tensor cores do not apply, and in mixed precision within the
FP64 truncation error plus the mixed slack, on uniform and adaptive trees."""
import numpy as np
import pytest

import oracle
from paper_1106_2176_gb300 import inputs

from gpu_common import rel, run_fmm

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12   # FP64 parity bound; the closed-form rotation maps are exact to ~1e-15
MIXED_SLACK = 2e-6


@pytest.mark.parametrize("P,theta,ncrit,gen", [(4, 0.5, 64, "uniform"), (8, 0.5, 32, "uniform"), (12, 0.4, 64, "uniform"),
                                               (10, 0.3, 64, "uniform"), (8, 0.6, 16, "plummer"), (6, 0.4, 8, "plummer"),
                                               (12, 0.5, 32, "plummer"), (16, 0.4, 64, "uniform")])
def test_rotation_fp64_matches_oracle(P, theta, ncrit, gen):
    x, q = getattr(inputs, "uniform_cube" if gen == "uniform" else "plummer")(6000, 13)
    po, go = oracle.fmm(x, q, P, theta, ncrit)
    phi, grad, f = run_fmm(x, q, P, theta, ncrit, precision="fp64", engine="rotation")
    assert f.stats()["m2l_engine"] == 3 and f.stats()["async_error"] == 0
    assert rel(phi, po) <= FP64_TOL and rel(grad, go) <= FP64_TOL


def test_rotation_matches_dense_engine_p16():
    x, q = inputs.uniform_cube(20000, 14)
    pr, gr, _ = run_fmm(x, q, 16, 0.5, 64, precision="fp64", engine="rotation")
    pd, gd, _ = run_fmm(x, q, 16, 0.5, 64, precision="fp64", engine="cudacore")
    assert rel(pr, pd) <= FP64_TOL and rel(gr, gd) <= FP64_TOL


@pytest.mark.parametrize("P,gen", [(8, "uniform"), (10, "plummer"), (16, "uniform")])
def test_rotation_mixed_within_truncation_error(P, gen):
    n = 20000
    x, q = getattr(inputs, "uniform_cube" if gen == "uniform" else "plummer")(n, 15)
    t = inputs.sample_targets(n, 512, seed=4)
    pd, gd = oracle.direct(x, q, targets=t)
    p64, g64, _ = run_fmm(x, q, P, 0.5, 64, precision="fp64", engine="rotation")
    pm, gm, f = run_fmm(x, q, P, 0.5, 64, precision="mixed", engine="rotation")
    assert f.stats()["m2l_engine"] == 3
    assert rel(pm[t], pd) <= rel(p64[t], pd) + MIXED_SLACK
    assert rel(gm[t], gd) <= rel(g64[t], gd) + MIXED_SLACK


def test_rotation_engine_rejects_high_p():
    from paper_1106_2176_gb300 import FMM
    from paper_1106_2176_gb300.fmm import FMMError
    with pytest.raises(FMMError):
        FMM(1000, p=18, theta=0.5, ncrit=64, precision="fp64", m2l_engine="rotation")
