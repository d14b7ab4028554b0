"""Tensor-core M2L sources by TMA tile loads on complete levels (Sec. 2.2:
boxes indexed by lattice position; on a level where every box exists, the
sources of a block of targets under one translation are the same block
shifted). The kernel then receives, row by row, the values the per-row
lookups and gathers deliver (zeros where the shifted position leaves the
level), so every result is bitwise that of the gather path."""
import numpy as np
import pytest

import oracle
from paper_1106_2176_gb300 import inputs

from gpu_common import ensure_built, rel, run_fmm, torch_cuda

pytestmark = pytest.mark.gpu

MIXED_SLACK = 2e-6


def clustered(n_uniform, n_cluster, seed):
    """A uniform cube (complete upper levels) plus a dense Plummer cluster in
    one corner (adaptive deeper levels)."""
    xu, qu = inputs.uniform_cube(n_uniform, seed)
    xc, qc = inputs.plummer(n_cluster, seed + 1)
    xc = 0.6 + 0.02 * xc / np.max(np.abs(xc))
    return np.concatenate([xu, xc]), np.concatenate([qu, qc])


# (order, input, leaf size, expected lattice levels as a bit mask)
CASES = [
    (8, "uniform", 200000, 64, 1 << 4),
    (8, "uniform", 1000000, 64, (1 << 4) | (1 << 5)),
    (6, "uniform", 500000, 32, (1 << 4) | (1 << 5)),
    (4, "uniform", 300000, 64, 1 << 4),
    (10, "uniform", 200000, 64, 1 << 4),
    (8, "clustered", 300000, 32, 1 << 4),
]


@pytest.mark.parametrize("P,gen,n,ncrit,levels", CASES)
def test_lattice_loads_give_the_gathered_results_bitwise(P, gen, n, ncrit, levels):
    if gen == "uniform":
        x, q = inputs.uniform_cube(n, 61 + P)
    else:
        x, q = clustered(n, n // 4, 61 + P)
    x, q = x.astype(np.float32), q.astype(np.float32)
    p1, g1, f1 = run_fmm(x, q, P, 0.5, ncrit, precision="mixed", dtype=np.float32, m2l_lattice=True)
    p0, g0, f0 = run_fmm(x, q, P, 0.5, ncrit, precision="mixed", dtype=np.float32, m2l_lattice=False)
    s1, s0 = f1.stats(), f0.stats()
    assert s1["m2l_engine"] == 1 and s1["async_error"] == 0 and s0["async_error"] == 0
    assert s1["lattice_levels"] == levels and s0["lattice_levels"] == 0
    assert np.array_equal(p1, p0) and np.array_equal(g1, g0)
    # the local expansions too, cell by cell
    _, L1 = f1.export_expansions()
    _, L0 = f0.export_expansions()
    assert np.array_equal(L1, L0)
    f1.close()
    f0.close()


def test_lattice_loads_with_float64_inputs():
    # FP64 positions and charges on the mixed path (FP32 expansions): the
    # lattice loads again give the gathered results bit for bit
    x, q = inputs.uniform_cube(200000, 75)
    p1, g1, f1 = run_fmm(x, q, 8, 0.5, 64, precision="mixed", dtype=np.float64, m2l_lattice=True)
    p0, g0, f0 = run_fmm(x, q, 8, 0.5, 64, precision="mixed", dtype=np.float64, m2l_lattice=False)
    assert f1.stats()["lattice_levels"] == 1 << 4 and f0.stats()["lattice_levels"] == 0
    assert f1.stats()["async_error"] == 0
    assert np.array_equal(p1, p0) and np.array_equal(g1, g0)
    f1.close()
    f0.close()


def test_lattice_path_within_the_error_bound():
    # N = 2e5 uniform, p = 8: level 4 by TMA; against the oracle's direct sum
    # on sampled targets, within the FP64 FMM's own error plus 2e-6
    # (FP32 inputs; the references take the same rounded positions and charges)
    x32, q32 = inputs.uniform_cube(200000, 71, dtype=np.float32)
    x, q = x32.astype(np.float64), q32.astype(np.float64)
    t = inputs.sample_targets(len(q), 1024, seed=71)
    pd, gd = oracle.direct(x, q, targets=t)
    p64, g64, _ = run_fmm(x, q, 8, 0.5, 64, precision="fp64")
    pm, gm, fm = run_fmm(x32, q32, 8, 0.5, 64, precision="mixed", dtype=np.float32)
    assert fm.stats()["lattice_levels"] == 1 << 4
    assert rel(p64[t], pd) < 1e-5
    assert rel(pm[t], pd) <= rel(p64[t], pd) + MIXED_SLACK and rel(gm[t], gd) <= rel(g64[t], gd) + MIXED_SLACK


def test_pool_threshold_and_switch_select_the_levels():
    # a pooling threshold above level 4's 4096 cells pools it: no lattice
    # level; the switch off: none either; rebuilding with it on again: level 4
    x, q = inputs.uniform_cube(200000, 72, dtype=np.float32)
    _, _, f = run_fmm(x, q, 8, 0.5, 64, precision="mixed", dtype=np.float32, m2l_pool=4096)
    assert f.stats()["lattice_levels"] == 0
    f.close()
    torch = torch_cuda()
    _, _, f = run_fmm(x, q, 8, 0.5, 64, precision="mixed", dtype=np.float32, m2l_lattice=False)
    assert f.stats()["lattice_levels"] == 0
    f.set_m2l_lattice(True)
    f.build(torch.tensor(x, device="cuda"), torch.tensor(q, device="cuda"))
    f.evaluate()
    torch.cuda.synchronize()
    assert f.stats()["lattice_levels"] == 1 << 4
    f.close()


def test_batch_of_lattice_systems_matches_their_own_evaluations():
    # the batch engine gathers on every level; each system's own evaluation
    # reads level 4 by TMA: bitwise the same results
    torch = torch_cuda()
    ensure_built()
    from paper_1106_2176_gb300.batch import FMMBatch
    systems = []
    for k, n in enumerate((200000, 5000, 250000, 20000)):
        x, q = inputs.uniform_cube(n, 80 + k, dtype=np.float32)
        systems.append((torch.tensor(x, device="cuda"), torch.tensor(q, device="cuda")))
    b = FMMBatch(systems, p=8, theta=0.5, ncrit=64, precision="mixed")
    assert b.handles[0].stats()["lattice_levels"] == 1 << 4
    ref = [(p.clone(), g.clone()) for p, g in b.evaluate_each()]
    for p, g in b.out:
        p.fill_(float("nan"))
        g.fill_(float("nan"))
    b.evaluate()
    torch.cuda.synchronize()
    for (p, g), (pr, gr) in zip(b.out, ref):
        assert bool((p == pr).all()) and bool((g == gr).all())
    assert b.status()[0] == 0
    b.close()
