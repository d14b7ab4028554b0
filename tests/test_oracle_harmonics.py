"""Pins of the oracle's solid harmonics (the basis of the series expansions of
Sec. 2.1) against closed forms, the binomial and addition theorems and
harmonicity."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import nm

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _closed(expr, x):
    X, Y, Z = x
    env = {"x": X, "y": Y, "z": Z, "r": np.sqrt(X * X + Y * Y + Z * Z), "w": complex(X, Y)}
    return complex(eval(expr, {}, env))


@pytest.mark.parametrize("pt", [(0.3, -0.7, 0.5), (-1.2, 0.4, -0.2), (0.0, 0.0, 0.8)])
def test_low_order_closed_forms(pt):
    g = json.load(open(os.path.join(GOLD, "harmonics_low_order.json")))
    R = oracle.regular(3, pt)
    Ih = oracle.irregular(3, pt)
    for key, expr in g["python"]["R"].items():
        n, m = map(int, key.split(","))
        assert abs(R[nm(n, m)] - _closed(expr, pt)) < 1e-14
    for key, expr in g["python"]["I"].items():
        n, m = map(int, key.split(","))
        assert abs(Ih[nm(n, m)] - _closed(expr, pt)) < 1e-13


def test_negative_order_symmetry():
    R = oracle.regular(9, (0.2, -0.5, 0.7))
    Ih = oracle.irregular(9, (0.2, -0.5, 0.7))
    for n in range(9):
        for m in range(1, n + 1):
            for X in (R, Ih):
                assert abs(X[nm(n, -m)] - (-1) ** m * np.conj(X[nm(n, m)])) < 1e-15 * (1 + abs(X[nm(n, m)]))


def test_binomial_theorem():
    # R_n^m(x + y) = sum_{k,l} R_k^l(x) R_{n-k}^{m-l}(y)
    P = 10
    x = np.array([0.31, -0.42, 0.27])
    y = np.array([-0.15, 0.22, 0.38])
    Rx, Ry, Rxy = oracle.regular(P, x), oracle.regular(P, y), oracle.regular(P, x + y)
    for n in range(P):
        for m in range(-n, n + 1):
            s = 0
            for k in range(n + 1):
                for l in range(-k, k + 1):
                    if abs(m - l) <= n - k:
                        s += Rx[nm(k, l)] * Ry[nm(n - k, m - l)]
            assert abs(s - Rxy[nm(n, m)]) < 1e-15


def test_addition_theorem_inverse_distance():
    # 1/|x - y| = sum_{n,m} conj(R_n^m(y)) I_n^m(x), |y| < |x|
    P = 30
    x = np.array([2.0, -1.5, 1.0])
    y = np.array([0.3, 0.2, -0.25])
    R, Ih = oracle.regular(P, y), oracle.irregular(P, x)
    s = np.sum(np.conj(R) * Ih)
    assert abs(s.imag) < 1e-15
    assert abs(s.real - 1.0 / np.linalg.norm(x - y)) < 1e-15


def test_harmonic_functions():
    # every R_n^m and I_n^m solves Laplace's equation (finite-difference Laplacian)
    # A wrong recurrence coefficient leaves a Laplacian of order |f| / |x|^2;
    # the central difference leaves truncation and rounding far below that.
    P = 7
    h = 1e-3
    for f, x0 in ((oracle.regular, np.array([0.6, -0.3, 0.45])),
                  (oracle.irregular, np.array([1.8, -1.1, 1.4]))):
        v0 = f(P, x0)
        lap = -6 * v0
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            lap = lap + f(P, x0 + e) + f(P, x0 - e)
        scale = np.abs(v0) / np.dot(x0, x0)
        assert np.all(np.abs(lap / h ** 2) <= 1e-3 * scale + 1e-7)


def test_ladder_relations():
    P = 8
    x0 = np.array([0.35, 0.2, -0.4])
    h = 1e-6
    R = oracle.regular(P, x0)
    d = []
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        d.append((oracle.regular(P, x0 + e) - oracle.regular(P, x0 - e)) / (2 * h))
    get = lambda n, m: R[nm(n, m)] if 0 <= n and abs(m) <= n else 0.0
    for n in range(1, P):
        for m in range(-n, n + 1):
            assert abs(d[2][nm(n, m)] - get(n - 1, m)) < 1e-8
            assert abs(d[0][nm(n, m)] + 1j * d[1][nm(n, m)] + get(n - 1, m + 1)) < 1e-8
            assert abs(d[0][nm(n, m)] - 1j * d[1][nm(n, m)] - get(n - 1, m - 1)) < 1e-8
