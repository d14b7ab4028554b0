"""Pins of the oracle's direct sum (the quantity the FMM approximates, Sec. 2.1,
Laplace kernel Sec. 4) against closed forms and invariants."""
import json
import math
import os

import numpy as np

import oracle
from paper_1106_2176_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_two_charges_closed_form():
    g = json.load(open(os.path.join(GOLD, "two_charges.json")))
    phi, grad = oracle.direct(np.array(g["x"]), np.array(g["q"]))
    np.testing.assert_allclose(phi, g["phi"], rtol=1e-15, atol=1e-16)
    np.testing.assert_allclose(grad, g["grad"], rtol=1e-14, atol=1e-17)


def test_cube_corners_closed_form():
    g = json.load(open(os.path.join(GOLD, "cube_corners.json")))
    s = np.array([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)], float)
    x = g["half_side"] * s
    q = np.full(8, g["charge"])
    phi, grad = oracle.direct(x, q)
    np.testing.assert_allclose(phi, g["phi"], rtol=1e-14)
    np.testing.assert_allclose(grad, g["grad_along_sign"] * s, rtol=1e-13)


def test_newton_third_law():
    # sum_i q_i grad phi_i = 0 because the pair force is antisymmetric
    x, q = inputs.uniform_cube(2000, seed=11)
    phi, grad = oracle.direct(x, q)
    f = (q[:, None] * grad).sum(axis=0)
    scale = np.abs(q[:, None] * grad).sum(axis=0)
    assert np.all(np.abs(f) < 1e-12 * scale)


def test_symmetric_octahedron_equal_potentials():
    x = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    q = np.ones(6)
    phi, grad = oracle.direct(x, q)
    # 4 neighbours at sqrt(2), one opposite at 2
    np.testing.assert_allclose(phi, 4 / math.sqrt(2) + 0.5, rtol=1e-15)
    # field points outward along the vertex direction, same magnitude everywhere
    # the opposite vertex gives -(2,0,0)/8, the four neighbours -(1,.,.)/(2 sqrt 2) each
    mag = -(0.25 + math.sqrt(2.0))
    for i in range(6):
        np.testing.assert_allclose(grad[i], mag * x[i], rtol=1e-14, atol=1e-16)


def test_coincident_pairs_skipped():
    # particles 0 and 1 coincide: each sees only particle 2
    x = np.array([[0.1, 0.2, 0.3], [0.1, 0.2, 0.3], [0.1, 0.2, 1.3]])
    q = np.array([1.0, 2.0, 3.0])
    phi, grad = oracle.direct(x, q)
    np.testing.assert_allclose(phi[:2], [3.0, 3.0], rtol=1e-15)
    np.testing.assert_allclose(phi[2], 3.0, rtol=1e-15)
    np.testing.assert_allclose(grad[0], [0, 0, 3.0], rtol=1e-14, atol=1e-15)


def test_targets_subset_matches_full():
    x, q = inputs.uniform_cube(3000, seed=5)
    t = inputs.sample_targets(3000, 100, seed=6)
    pa, ga = oracle.direct(x, q)
    pt, gt = oracle.direct(x, q, targets=t)
    assert np.array_equal(pt, pa[t]) and np.array_equal(gt, ga[t])


def test_bruteforce_small():
    # an independent pure-Python double loop over a tiny input
    x, q = inputs.uniform_cube(37, seed=3)
    phi, grad = oracle.direct(x, q)
    for i in range(37):
        p, g = 0.0, [0.0, 0.0, 0.0]
        for j in range(37):
            if i == j:
                continue
            d = [x[i][k] - x[j][k] for k in range(3)]
            r = math.sqrt(sum(v * v for v in d))
            p += q[j] / r
            for k in range(3):
                g[k] += -q[j] * d[k] / r ** 3
        assert abs(p - phi[i]) <= 1e-13 * max(1.0, abs(p))
        for k in range(3):
            assert abs(g[k] - grad[i][k]) <= 1e-12 * max(1.0, abs(g[k]))
