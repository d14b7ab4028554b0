"""GPU FMM against the oracle: FP64 parity <= 1e-12 relative L2 at the same
p, theta, ncrit (Sec. 2.1 operators, Fig. flow_chart order); mixed precision
within the FP64 FMM's own truncation error plus 2e-6 of the FP64 direct sum."""
import numpy as np
import pytest

import oracle
from paper_1106_2176_gb300 import inputs

from gpu_common import ensure_built, rel, run_fmm, torch_cuda, unscale

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_SLACK = 2e-6


@pytest.fixture(scope="module")
def cube16k():
    x, q = inputs.uniform_cube(16384, 1)
    return x, q, oracle.fmm(x, q, 6, 0.5, 64), oracle.direct(x, q)


def test_fp64_matches_oracle_small_config(cube16k):
    # N = 16384, p = 6, theta = 0.5, ncrit = 64, FP64 throughout
    x, q, (po, go), _ = cube16k
    phi, grad, _ = run_fmm(x, q, 6, 0.5, 64)
    assert rel(phi, po) <= FP64_TOL and rel(grad, go) <= FP64_TOL


def test_fp64_expansions_match_oracle():
    x, q = inputs.uniform_cube(6000, 2)
    P = 5
    phi, grad, f = run_fmm(x, q, P, 0.5, 16)
    T = oracle.Tree(x, 16, 0.5)
    _, _, Mo, Lo = T.evaluate(q, P, expansions=True)
    Ms, Ls = f.export_expansions()
    t = f.export_tree()
    Mg, Lg = unscale(Ms, Ls, t["level"], t["box"][3], P)
    assert np.max(np.abs(Mg - Mo)) <= 1e-12 * np.max(np.abs(Mo))
    # local expansions per cell, relative to each cell's scale
    sc = np.max(np.abs(Lo), axis=1, keepdims=True) + 1e-300
    assert np.max(np.abs(Lg - Lo) / sc) <= 1e-11


@pytest.mark.parametrize("P,theta,ncrit,gen", [(1, 0.5, 32, "uniform"), (2, 0.5, 8, "uniform"), (10, 0.4, 64, "uniform"),
                                               (8, 0.7, 16, "plummer"), (4, 0.3, 4, "plummer"), (14, 0.5, 64, "uniform")])
def test_fp64_matches_oracle_variants(P, theta, ncrit, gen):
    x, q = getattr(inputs, "uniform_cube" if gen == "uniform" else "plummer")(8000, 11)
    po, go = oracle.fmm(x, q, P, theta, ncrit)
    phi, grad, _ = run_fmm(x, q, P, theta, ncrit)
    assert rel(phi, po) <= FP64_TOL and rel(grad, go) <= FP64_TOL


def test_fp64_float32_input():
    x, q = inputs.uniform_cube(10000, 12, dtype=np.float32)
    po, go = oracle.fmm(x.astype(np.float64), q.astype(np.float64), 6, 0.5, 32)
    phi, grad, _ = run_fmm(x, q, 6, 0.5, 32, precision="fp64", dtype=np.float32)
    # outputs are rounded to float32
    assert rel(phi, po) <= 1e-7 and rel(grad, go) <= 1e-7


def test_small_theta_is_direct_sum():
    x, q = inputs.uniform_cube(3000, 13)
    pd, gd = oracle.direct(x, q)
    phi, grad, f = run_fmm(x, q, 3, 0.001, 32)
    assert f.stats()["n_m2l_pairs"] == 0
    assert rel(phi, pd) <= 1e-13 and rel(grad, gd) <= 1e-13


@pytest.mark.parametrize("gen,ncrit", [("uniform", 32), ("uniform", 7), ("plummer", 13)])
def test_mixed_near_field_matches_direct_sum(gen, ncrit):
    # theta -> 0 leaves only P2P: the FP32 near-field kernel (packed pairs,
    # odd slice ends, several shared-memory chunks, the r = 0 test on
    # coincident particles of one leaf) against the FP64 direct sum of the
    # same FP32-rounded inputs
    n = 5000
    x, q = (inputs.uniform_cube(n, 23) if gen == "uniform" else inputs.plummer(n, 23))
    x = x.astype(np.float32)
    q = q.astype(np.float32)
    x[100:111] = x[100]  # eleven coincident particles
    x64, q64 = x.astype(np.float64), q.astype(np.float64)
    pd, gd = oracle.direct(x64, q64)
    phi, grad, f = run_fmm(x, q, 3, 0.001, ncrit, precision="mixed", dtype=np.float32)
    assert f.stats()["n_m2l_pairs"] == 0
    assert rel(phi, pd) <= MIXED_SLACK and rel(grad, gd) <= MIXED_SLACK


def test_serial_schedule_is_bitwise_identical():
    # fmm_set_overlap(0) runs the far and near field in turn on one stream;
    # every kernel's result is independent of the schedule
    x, q = inputs.uniform_cube(50000, 24, dtype=np.float32)
    p1, g1, f1 = run_fmm(x, q, 8, 0.5, 64, precision="mixed", dtype=np.float32)
    torch = torch_cuda()
    f1.set_overlap(False)
    xt, qt = torch.tensor(x, device="cuda"), torch.tensor(q, device="cuda")
    f1.build(xt, qt)
    p2, g2 = [t.cpu().numpy().astype(np.float64) for t in f1.evaluate()]
    st = f1.stats()
    assert np.array_equal(p1, p2) and np.array_equal(g1, g2)
    assert st["ms_p2p"] > 0 and st["ms_m2l"] > 0


def test_single_and_coincident_particles():
    for x in (np.array([[0.1, 0.2, 0.3]]), np.tile([[0.5, 0.5, 0.5]], (40, 1))):
        q = np.linspace(1, 2, len(x))
        phi, grad, _ = run_fmm(x, q, 4, 0.5, 8)
        assert np.all(phi == 0) and np.all(grad == 0)


def test_mixed_within_truncation_error(cube16k):
    x, q, (po, go), (pd, gd) = cube16k
    e64 = rel(po, pd), rel(go, gd)
    phi, grad, _ = run_fmm(x, q, 6, 0.5, 64, precision="mixed", dtype=np.float64)
    assert rel(phi, pd) <= e64[0] + MIXED_SLACK
    assert rel(grad, gd) <= e64[1] + MIXED_SLACK


def test_mixed_float32_inputs_precision_config():
    # N = 10^5 uniform, p = 10, theta = 0.4 (a reduced version of the 10^6 case)
    x, q = inputs.uniform_cube(100000, 1, dtype=np.float32)
    x64, q64 = x.astype(np.float64), q.astype(np.float64)
    t = inputs.sample_targets(100000, 1024, seed=2)
    pd, gd = oracle.direct(x64, q64, targets=t)
    p64, g64, _ = run_fmm(x, q, 10, 0.4, 64, precision="fp64", dtype=np.float64)
    pm, gm, _ = run_fmm(x, q, 10, 0.4, 64, precision="mixed", dtype=np.float32)
    assert rel(pm[t], pd) <= rel(p64[t], pd) + MIXED_SLACK
    assert rel(gm[t], gd) <= rel(g64[t], gd) + MIXED_SLACK


def test_direct_sum_kernel_matches_oracle():
    torch = torch_cuda()
    ensure_built()
    from paper_1106_2176_gb300 import FMM
    x, q = inputs.uniform_cube(20000, 14)
    t = inputs.sample_targets(20000, 700, seed=3)
    f = FMM(10, p=2)
    pg, gg = f.direct(torch.tensor(x, device="cuda"), torch.tensor(q, device="cuda"), torch.tensor(t, device="cuda"))
    pd, gd = oracle.direct(x, q, targets=t)
    assert rel(pg.cpu().numpy(), pd) <= 1e-14 and rel(gg.cpu().numpy(), gd) <= 1e-14


def test_host_memory_path_matches_device_path():
    ensure_built()
    from paper_1106_2176_gb300 import FMM
    x, q = inputs.uniform_cube(5000, 15)
    phi_d, grad_d, _ = run_fmm(x, q, 6, 0.5, 32)
    f = FMM(5000, p=6, theta=0.5, ncrit=32)
    f.build(x, q)
    phi_h, grad_h = f.evaluate()
    assert np.array_equal(phi_h, phi_d) and np.array_equal(grad_h, grad_d)


def test_errors_are_status_codes():
    torch = torch_cuda()
    ensure_built()
    from paper_1106_2176_gb300 import FMM, FMMError, fmm
    f = FMM(100, p=4)
    with pytest.raises(FMMError) as e:
        f.evaluate()
    assert e.value.code == fmm.FMM_ESTATE
    x = torch.zeros((200, 3), dtype=torch.float64, device="cuda")
    q = torch.ones(200, dtype=torch.float64, device="cuda")
    with pytest.raises(FMMError) as e:
        f.build(x, q)
    assert e.value.code == fmm.FMM_EINVAL
    x = torch.rand((50, 3), dtype=torch.float64, device="cuda")
    x[7, 1] = float("nan")
    with pytest.raises(FMMError) as e:
        f.build(x, q[:50])
    assert e.value.code == fmm.FMM_ENONFINITE
    # the handle stays usable after errors
    x = torch.rand((50, 3), dtype=torch.float64, device="cuda")
    f.build(x, q[:50])
    phi, grad = f.evaluate()
    assert torch.isfinite(phi).all()


def test_rebuild_same_handle_is_deterministic():
    x, q = inputs.uniform_cube(20000, 16)
    torch = torch_cuda()
    ensure_built()
    from paper_1106_2176_gb300 import FMM
    f = FMM(20000, p=6, precision="mixed")
    xt, qt = torch.tensor(x, device="cuda"), torch.tensor(q, device="cuda")
    outs = []
    for _ in range(3):
        f.build(xt, qt)
        outs.append([t.cpu().numpy() for t in f.evaluate()])
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0]) and np.array_equal(o[1], outs[0][1])


@pytest.mark.parametrize("P", [4, 6, 8])
def test_tensor_core_m2l_matches_fp64_expansions(P):
    # the local expansions of the mixed path (tcgen05 M2L in split TF32) against
    # the FP64 path's, cell by cell, relative to each cell's largest coefficient
    x, q = inputs.uniform_cube(60000, 21)
    _, _, f64 = run_fmm(x, q, P, 0.5, 32, precision="fp64")
    _, _, fmx = run_fmm(x, q, P, 0.5, 32, precision="mixed", engine="tensor")
    st = fmx.stats()
    assert st["m2l_engine"] == 1 and st["async_error"] == 0
    _, L64 = f64.export_expansions()
    _, Lmx = fmx.export_expansions()
    lev = f64.export_tree()["level"]
    sel = lev >= 2
    sc = np.max(np.abs(L64[sel]), axis=1, keepdims=True) + 1e-300
    assert np.max(np.abs(Lmx[sel] - L64[sel]) / sc) < 2e-5


def test_tensor_and_cudacore_engines_agree():
    x, q = inputs.uniform_cube(40000, 22, dtype=np.float32)
    pt, gt, ft = run_fmm(x, q, 8, 0.5, 64, precision="mixed", dtype=np.float32, engine="tensor")
    pc, gc, fc = run_fmm(x, q, 8, 0.5, 64, precision="mixed", dtype=np.float32, engine="cudacore")
    assert ft.stats()["m2l_engine"] == 1 and fc.stats()["m2l_engine"] == 2
    assert rel(pt, pc) < 1e-6 and rel(gt, gc) < 1e-6


@pytest.mark.parametrize("P", [2, 3, 5, 7, 8, 9, 10])
def test_mixed_irregular_m2l_matches_fp64_expansions(P):
    # adaptive tree (Plummer sphere, small leaves): the accepted pairs whose
    # cells sit on different levels run through the FP32 CUDA-core kernel (one
    # run of orders per lane, each p's own shared-memory layout); the local
    # expansions of every cell against the FP64 path's, relative to each
    # cell's largest coefficient
    x, q = inputs.plummer(40000, 31)
    _, _, f64 = run_fmm(x, q, P, 0.5, 8, precision="fp64")
    _, _, fmx = run_fmm(x, q, P, 0.5, 8, precision="mixed")
    st = fmx.stats()
    assert st["n_m2l_irregular"] > 1000 and st["async_error"] == 0
    _, L64 = f64.export_expansions()
    _, Lmx = fmx.export_expansions()
    lev = f64.export_tree()["level"]
    sel = lev >= 2
    sc = np.max(np.abs(L64[sel]), axis=1, keepdims=True) + 1e-300
    assert np.max(np.abs(Lmx[sel] - L64[sel]) / sc) < 2e-5


@pytest.mark.parametrize("pool,gen", [(0, "uniform"), (4096, "uniform"), (0, "plummer"), (100000, "plummer")])
def test_m2l_tile_pooling_keeps_the_error_bound(pool, gen):
    # per-octant tiles on every level (pool 0) or pooled tiles on every level
    # up to `pool` cells: the same pairs in other tiles, so each mixed run stays
    # within its FP64 FMM's error on the same targets plus 2e-6
    x, q = getattr(inputs, "uniform_cube" if gen == "uniform" else "plummer")(30000, 41)
    t = inputs.sample_targets(len(q), 512, seed=41)
    pd, gd = oracle.direct(x, q, targets=t)
    p64, g64, f64 = run_fmm(x, q, 6, 0.5, 32, precision="fp64", m2l_pool=pool)
    pm, gm, fm = run_fmm(x, q, 6, 0.5, 32, precision="mixed", m2l_pool=pool)
    assert fm.stats()["async_error"] == 0
    assert rel(p64[t], pd) < 1e-4 and rel(g64[t], gd) < 1e-4
    assert rel(pm[t], pd) <= rel(p64[t], pd) + MIXED_SLACK and rel(gm[t], gd) <= rel(g64[t], gd) + MIXED_SLACK


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_deep_adaptive_tree_against_oracle(precision):
    # a clustered input with small leaves reaches levels deeper than the dense
    # lattice maps (8): the M2L sources there come from the per-level hash
    # tables; FP64 to 1e-12 of the oracle FMM, mixed within the FP64 FMM's
    # error plus 2e-6 against the direct sum
    x, q = inputs.plummer(20000, 43)
    phi, grad, f = run_fmm(x, q, 6, 0.5, 4, precision=precision)
    assert f.stats()["depth"] >= 10 and f.stats()["async_error"] == 0
    if precision == "fp64":
        po, go = oracle.fmm(x, q, 6, 0.5, 4)
        assert rel(phi, po) <= FP64_TOL and rel(grad, go) <= FP64_TOL
    else:
        pd, gd = oracle.direct(x, q)
        p64, g64, _ = run_fmm(x, q, 6, 0.5, 4, precision="fp64")
        assert rel(phi, pd) <= rel(p64, pd) + MIXED_SLACK and rel(grad, gd) <= rel(g64, gd) + MIXED_SLACK
