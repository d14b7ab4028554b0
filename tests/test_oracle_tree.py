"""Pins of the oracle's Morton octree and dual-traversal lists (Sec. 2.1 near/far
split, Sec. 2.2 Morton-indexed boxes, Sec. 5 sorted indices with start/offset
ranges and Morton index at a prescribed maximum level)."""
import math

import numpy as np
import pytest

import oracle
from paper_1106_2176_gb300 import inputs


def _py_keys(x):
    """Quantisation and bit interleave with Python floats and ints."""
    lo = [min(p[k] for p in x) for k in range(3)]
    hi = [max(p[k] for p in x) for k in range(3)]
    c = [(lo[k] + hi[k]) * 0.5 for k in range(3)]
    R0 = max((hi[k] - lo[k]) * 0.5 for k in range(3)) or 1.0
    org = [c[k] - R0 for k in range(3)]
    s = 2097152.0 / (2.0 * R0)
    keys = []
    for p in x:
        ijk = [min(max(math.floor((p[k] - org[k]) * s), 0), 2097151) for k in range(3)]
        bits = "".join(str((ijk[2] >> b) & 1) + str((ijk[1] >> b) & 1) + str((ijk[0] >> b) & 1)
                       for b in reversed(range(21)))
        keys.append(int(bits, 2))
    return keys, org, R0


@pytest.mark.parametrize("n,seed", [(1, 1), (7, 2), (4096, 3)])
def test_keys_and_sort_bruteforce(n, seed):
    x, _ = inputs.uniform_cube(n, seed)
    T = oracle.Tree(x, 16, 0.5)
    ic, key, perm = T.particles()
    pk, org, R0 = _py_keys(x.tolist())
    o, r = T.box()
    assert list(o) == org and r == R0
    assert [int(k) for k in key] == [pk[i] for i in perm]
    # stable ascending sort by key, ties by input index
    ref = sorted(range(n), key=lambda i: (pk[i], i))
    assert list(perm) == ref


def test_sort_ties_stable():
    x = np.array([[0.0, 0, 0], [1, 1, 1], [0, 0, 0], [0.5, 0.5, 0.5], [0, 0, 0]])
    T = oracle.Tree(x, 1, 0.5)
    _, key, perm = T.particles()
    assert list(perm[:3]) == [0, 2, 4]


def _check_cells(T, ncrit):
    c = T.cells()
    n = T.n
    lev, b, e, ch, nc, par = c["level"], c["begin"], c["end"], c["child"], c["nchild"], c["parent"]
    _, key, _ = T.particles()
    assert b[0] == 0 and e[0] == n and lev[0] == 0
    # breadth-first: levels non-decreasing, anchors increasing within a level
    assert np.all(np.diff(lev) >= 0)
    for l in range(T.depth + 1):
        a = c["anchor"][lev == l]
        assert np.all(a[1:] > a[:-1])
    leaves = nc == 0
    # leaves partition [0, n)
    lb, le = np.sort(b[leaves]), np.sort(e[leaves])
    assert lb[0] == 0 and le[-1] == n and np.all(lb[1:] == le[:-1])
    for i in range(T.ncells):
        if nc[i] == 0:
            assert e[i] - b[i] <= ncrit or lev[i] == 21
            assert e[i] > b[i]
            continue
        assert e[i] - b[i] > ncrit and lev[i] < 21
        kids = range(ch[i], ch[i] + nc[i])
        assert sum(e[k] - b[k] for k in kids) == e[i] - b[i]
        assert b[ch[i]] == b[i] and e[ch[i] + nc[i] - 1] == e[i]
        for k in kids:
            assert par[k] == i and lev[k] == lev[i] + 1
            sh = 3 * (21 - int(lev[k]))
            pre = int(c["anchor"][k]) >> sh
            assert all((int(key[j]) >> sh) == pre for j in range(b[k], e[k]))


@pytest.mark.parametrize("gen,n,ncrit", [("uniform", 5000, 32), ("plummer", 5000, 16), ("uniform", 300, 1)])
def test_cell_invariants(gen, n, ncrit):
    x, _ = getattr(inputs, "uniform_cube" if gen == "uniform" else "plummer")(n, 9)
    _check_cells(oracle.Tree(x, ncrit, 0.5), ncrit)


def test_all_coincident_reaches_level_21():
    x = np.tile([[0.3, -0.1, 0.2]], (50, 1))
    T = oracle.Tree(x, 8, 0.5)
    c = T.cells()
    assert T.depth == 21 and T.ncells == 22 and T.nleaves == 1
    assert c["end"][-1] - c["begin"][-1] == 50
    (pp, pi), (mp, mi) = T.lists()
    assert T.n_p2p == 1 and T.n_m2l == 0


def _subtree_particles(c, i):
    return np.arange(c["begin"][i], c["end"][i])


@pytest.mark.parametrize("gen,n,ncrit,theta", [("uniform", 512, 4, 0.5), ("plummer", 400, 3, 0.5),
                                               ("uniform", 300, 2, 0.7), ("uniform", 256, 1, 0.3)])
def test_lists_cover_every_pair_exactly_once(gen, n, ncrit, theta):
    x, _ = getattr(inputs, "uniform_cube" if gen == "uniform" else "plummer")(n, 21)
    T = oracle.Tree(x, ncrit, theta)
    c = T.cells()
    (pp, pi), (mp, mi) = T.lists()
    cover = np.zeros((n, n), np.int32)
    for A in range(T.ncells):
        ta = _subtree_particles(c, A)
        for k in range(pp[A], pp[A + 1]):
            B = pi[k]
            assert c["nchild"][A] == 0 and c["nchild"][B] == 0
            cover[np.ix_(ta, _subtree_particles(c, B))] += 1
        for k in range(mp[A], mp[A + 1]):
            cover[np.ix_(ta, _subtree_particles(c, mi[k]))] += 1
    assert np.all(cover == 1)
    assert T.n_m2l > 0 and T.n_p2p > 0


def _geom_accept(c, box, A, B, theta):
    org, R0 = box
    cen = []
    rad = []
    for X in (A, B):
        l = c["level"][X]
        h = 2 * R0 / 2 ** l
        a = [0, 0, 0]
        k = int(c["anchor"][X])
        for b in range(21):
            for d in range(3):
                a[d] |= ((k >> (3 * b + d)) & 1) << b
        cen.append(np.array([org[d] + (a[d] / 2 ** 21) * 2 * R0 + h / 2 for d in range(3)]))
        rad.append(math.sqrt(3) * h / 2)
    return rad[0] + rad[1], theta * np.linalg.norm(cen[0] - cen[1])


def test_mac_matches_geometry():
    # accepted pairs satisfy r_A + r_B < theta |c_A - c_B| with r the half
    # diagonal; P2P pairs do not (checked in floating point, away from ties)
    x, _ = inputs.uniform_cube(2000, 4)
    theta = 0.5
    T = oracle.Tree(x, 16, theta)
    c = T.cells()
    (pp, pi), (mp, mi) = T.lists()
    box = T.box()
    for A in range(0, T.ncells, 7):
        for k in range(mp[A], mp[A + 1]):
            lhs, rhs = _geom_accept(c, box, A, mi[k], theta)
            assert lhs < rhs * (1 + 1e-12)
        for k in range(pp[A], pp[A + 1]):
            lhs, rhs = _geom_accept(c, box, A, pi[k], theta)
            assert lhs >= rhs * (1 - 1e-12)


def test_uniform_counts_match_lattice_reading():
    # uniform tree with every leaf at level 5 (32^3 cells, ~20 particles each):
    # interior leaves see 179 P2P leaves and interior cells 1253 M2L cells at
    # theta = 0.5 under the half-diagonal MAC
    x, _ = inputs.uniform_cube(655360, 8)
    T = oracle.Tree(x, 64, 0.5)
    c = T.cells()
    (pp, pi), (mp, mi) = T.lists()
    lev = c["level"]
    assert set(lev[c["nchild"] == 0]) == {5}
    assert np.diff(pp)[c["nchild"] == 0].max() == 179
    assert np.diff(mp)[lev == 5].max() == 1253
