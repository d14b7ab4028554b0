"""Pins of the oracle's whole FMM against the direct sum (Sec. 2.1: O(N)
evaluation to a controllable accuracy; Sec. 3.1: p = 3 gives 3-4 significant
digits)."""
import numpy as np
import pytest

import oracle
from paper_1106_2176_gb300 import inputs


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def cube16k():
    x, q = inputs.uniform_cube(16384, 1)
    return x, q, oracle.direct(x, q)


def test_config_small_fp64(cube16k):
    # N = 16384, p = 6, theta = 0.5, ncrit = 64 against the full direct sum
    x, q, (pd, gd) = cube16k
    phi, grad = oracle.fmm(x, q, 6, 0.5, 64)
    assert rel(phi, pd) < 1e-5 and rel(grad, gd) < 5e-6


def test_small_theta_is_direct_sum():
    # theta -> 0: no pair passes the MAC, everything is P2P, the FMM is the
    # direct sum up to the order of summation
    x, q = inputs.uniform_cube(3000, 12)
    T = oracle.Tree(x, 32, 1e-3)
    assert T.n_m2l == 0
    phi, grad = T.evaluate(q, 3)
    pd, gd = oracle.direct(x, q)
    assert rel(phi, pd) < 1e-14 and rel(grad, gd) < 1e-14


def test_truncation_error_decays_with_p():
    x, q = inputs.uniform_cube(4096, 1)
    pd, gd = oracle.direct(x, q)
    T = oracle.Tree(x, 32, 0.5)
    errs = []
    for P in (2, 4, 6, 8, 10, 12):
        phi, grad = T.evaluate(q, P)
        errs.append(rel(phi, pd))
    errs = np.array(errs)
    assert np.all(np.diff(np.log(errs)) < 0)
    # geometric decay at least as fast as theta^p (slope of log err vs p)
    slope = np.polyfit([2, 4, 6, 8, 10, 12], np.log(errs), 1)[0]
    assert slope < np.log(0.5)


def test_p3_three_to_four_digits():
    # Sec. 3.1: p = 3 gives three to four correct digits
    x, q = inputs.uniform_cube(8192, 2)
    pd, _ = oracle.direct(x, q)
    phi, _ = oracle.fmm(x, q, 3, 0.5, 32)
    e = rel(phi, pd)
    # three significant digits: relative error of the order of 1e-3 at most
    assert 1e-5 < e < 2e-3


def test_plummer_converges():
    x, q = inputs.plummer(4000, 4)
    pd, gd = oracle.direct(x, q)
    e4 = rel(oracle.fmm(x, q, 4, 0.5, 16)[0], pd)
    e10 = rel(oracle.fmm(x, q, 10, 0.5, 16)[0], pd)
    assert e10 < 1e-2 * e4 and e10 < 1e-6


def test_expansions_monopole_and_linearity():
    x, q = inputs.uniform_cube(2000, 3)
    T = oracle.Tree(x, 32, 0.5)
    phi, grad, M, L = T.evaluate(q, 5, expansions=True)
    c = T.cells()
    _, _, perm = T.particles()
    qs = q[perm]
    for i in range(T.ncells):
        # total charge of a cell equals its monopole coefficient
        assert abs(M[i, 0] - qs[c["begin"][i]:c["end"][i]].sum()) < 1e-13
    phi2, grad2 = T.evaluate(2.0 * q, 5)
    assert np.array_equal(phi2, 2.0 * phi) and np.array_equal(grad2, 2.0 * grad)


def test_rejects_bad_arguments():
    x, q = inputs.uniform_cube(10, 1)
    for args in ((0, 0.5, 8), (41, 0.5, 8), (4, 0.0, 8), (4, 1.0, 8), (4, 0.5, 0)):
        with pytest.raises(ValueError):
            oracle.fmm(x, q, *args)
