"""GPU octree and interaction lists, bit for bit against the oracle (Sec. 2.1
near/far split, Sec. 2.2 Morton-indexed boxes, Sec. 5 sorted indices)."""
import numpy as np
import pytest

import oracle
from paper_1106_2176_gb300 import inputs

from gpu_common import ensure_built, torch_cuda

pytestmark = pytest.mark.gpu


def gpu_tree(x, q, ncrit, theta, dtype=np.float64, precision="fp64", uniform_path=True):
    torch = torch_cuda()
    ensure_built()
    from paper_1106_2176_gb300 import FMM
    f = FMM(len(q), p=4, theta=theta, ncrit=ncrit, precision=precision, uniform_path=uniform_path)
    f.build(torch.tensor(np.asarray(x, dtype), device="cuda"), torch.tensor(np.asarray(q, dtype), device="cuda"))
    return f.export_tree(), f


def compare(x, q, ncrit, theta, dtype=np.float64, uniform_path=True, T=None):
    g, f = gpu_tree(x, q, ncrit, theta, dtype, uniform_path=uniform_path)
    # the oracle sees exactly the values the GPU saw
    if T is None:
        T = oracle.Tree(np.asarray(x, dtype).astype(np.float64), ncrit, theta)
    ic, key, perm = T.particles()
    org, R0 = T.box()
    assert np.array_equal(g["box"][:3], org) and g["box"][3] == R0
    assert np.array_equal(g["keys"], key)
    assert np.array_equal(g["perm"].astype(np.int64), perm)
    c = T.cells()
    assert len(g["level"]) == T.ncells
    for k in ("level", "anchor", "begin", "end", "child", "nchild", "parent"):
        assert np.array_equal(g[k].astype(np.int64), c[k].astype(np.int64)), k
    (pp, pi), (mp, mi) = T.lists()
    assert np.array_equal(g["p2p_ptr"], pp) and np.array_equal(g["p2p_idx"].astype(np.int64), pi)
    assert np.array_equal(g["m2l_ptr"], mp) and np.array_equal(g["m2l_idx"].astype(np.int64), mi)
    s = f.stats()
    assert s["n_p2p_pairs"] == T.n_p2p and s["n_m2l_pairs"] == T.n_m2l
    assert s["n_interactions"] == T.interactions and s["depth"] == T.depth
    # the full-octree fast path is taken exactly when every leaf sits on the
    # deepest level and every level is full
    full = T.nleaves == 8 ** T.depth and T.ncells == (8 ** (T.depth + 1) - 1) // 7 and T.depth >= 1
    assert s["uniform_path"] == int(uniform_path and full)
    f.close()
    return T


@pytest.mark.parametrize("n,ncrit,theta,seed", [(1, 8, 0.5, 1), (2, 1, 0.5, 2), (7, 2, 0.5, 3), (1000, 16, 0.5, 4),
                                                (16384, 64, 0.5, 1), (50000, 32, 0.4, 5), (20000, 8, 0.7, 6)])
def test_uniform_tree_bit_exact(n, ncrit, theta, seed):
    x, q = inputs.uniform_cube(n, seed)
    compare(x, q, ncrit, theta)


@pytest.mark.parametrize("uniform_path", [True, False])
@pytest.mark.parametrize("n,ncrit,theta,seed", [(16384, 64, 0.5, 1), (50000, 32, 0.4, 5), (4096, 100, 0.3, 7)])
def test_full_octree_lists_with_and_without_fast_path(n, ncrit, theta, seed, uniform_path):
    # uniform cubes whose trees come out full: the lattice-stencil lists and
    # the traversal's both equal the oracle's
    x, q = inputs.uniform_cube(n, seed)
    T = compare(x, q, ncrit, theta, uniform_path=uniform_path)
    assert T.nleaves == 8 ** T.depth


@pytest.mark.parametrize("n,ncrit", [(20000, 16), (3000, 1)])
def test_plummer_tree_bit_exact(n, ncrit):
    x, q = inputs.plummer(n, 9)
    compare(x, q, ncrit, 0.5)


def test_float32_input_bit_exact():
    x, q = inputs.uniform_cube(30000, 10, dtype=np.float32)
    compare(x, q, 64, 0.5, dtype=np.float32)


def test_float32_subnormal_and_signed_zero_coordinates_bit_exact():
    # FP32 inputs whose coordinates are subnormal (below 2^-126), with +0 and
    # -0 among them: the box and the keys take every value exactly, as the
    # oracle does in FP64, although the library's FP32 arithmetic flushes
    # subnormals to zero
    rng = np.random.default_rng(12)
    m = rng.integers(-(2 ** 22), 2 ** 22, size=(3000, 3)).astype(np.float64)
    x = (m * 2.0 ** -149).astype(np.float32)
    x[:5] = 0.0
    x[5:10] = -0.0
    assert np.all(np.abs(x[x != 0]) < np.float32(2.0 ** -126))
    q = np.ones(3000, np.float32)
    compare(x, q, 16, 0.5, dtype=np.float32)


def test_ragged_sizes_span_several_sort_tiles():
    # 4096 keys per radix tile: sizes around tile edges
    for n in (4095, 4096, 4097, 12289):
        x, q = inputs.uniform_cube(n, n)
        compare(x, q, 16, 0.5)


def test_coincident_particles_reach_level_21():
    x = np.tile([[0.25, -0.5, 0.125]], (300, 1))
    x[:10] += np.linspace(0, 1, 10)[:, None]
    q = np.ones(300)
    T = compare(x, q, 8, 0.5)
    assert T.depth == 21


def test_duplicate_keys_sorted_stably():
    rng = np.random.default_rng(3)
    base = rng.uniform(-1, 1, (50, 3))
    x = base[rng.integers(0, 50, 5000)]
    q = rng.uniform(-1, 1, 5000)
    compare(x, q, 4, 0.5)


@pytest.fixture(scope="module")
def bench_size():
    """The scale workload the bench times: N = 10^7 uniform cube, FP32
    positions, ncrit = 128, theta = 0.5 (a full octree of depth 6, 262,144
    leaves, 4.4e7 P2P and 3.2e8 M2L pairs), with the oracle's tree of it."""
    n = 10_000_000
    x, q = inputs.uniform_cube(n, 3, dtype=np.float32)
    T = oracle.Tree(x.astype(np.float64), 128, 0.5)
    return x, q, T


@pytest.mark.parametrize("uniform_path", [True, False])
def test_bench_size_tree_and_lists_bit_exact(bench_size, uniform_path):
    # every array in full: keys, permutation, the seven cell arrays and both
    # CSR lists (the M2L list is expanded from the implicit lattice pairs)
    x, q, T = bench_size
    compare(x, q, 128, 0.5, dtype=np.float32, uniform_path=uniform_path, T=T)
    assert T.depth == 6 and T.nleaves == 8 ** 6


def test_differentiation_tree_bit_exact():
    # the adaptive tree of the differentiation workload: N = 10^6 Plummer
    # sphere, FP32 positions, ncrit = 64, theta = 0.5 (pairs of cells on
    # different levels in both lists)
    x, q = inputs.plummer(1_000_000, 7)
    T = compare(x.astype(np.float32), q.astype(np.float32), 64, 0.5, dtype=np.float32)
    assert T.nleaves < 8 ** T.depth
