"""Pins of the oracle's P2M, M2M, M2L, L2L and L2P (Sec. 2.1, Fig. flow_chart)
against the direct sum, exact translation identities and finite differences."""
import numpy as np
import pytest

import oracle
from oracle import nm


def _cluster(n, centre, radius, seed):
    rng = np.random.default_rng(seed)
    x = np.asarray(centre) + rng.uniform(-radius, radius, size=(n, 3))
    q = rng.uniform(-1, 1, n)
    return x, q


def _eval_multipole(P, M, c, y):
    # phi(y) = sum_{n,m} M_n^m I_n^m(y - c)
    return np.real(np.sum(M * oracle.irregular(P, np.asarray(y) - c)))


def test_p2m_low_moments():
    x, q = _cluster(20, [0.1, 0.2, 0.3], 0.2, 1)
    c = np.array([0.1, 0.2, 0.3])
    M = oracle.p2m(4, x, q, c)
    d = x - c
    assert abs(M[nm(0, 0)] - q.sum()) < 1e-14          # monopole = total charge
    assert abs(M[nm(1, 0)] - (q * d[:, 2]).sum()) < 1e-14  # conj(R_1^0) = z
    assert abs(M[nm(1, 1)] - (q * (d[:, 0] - 1j * d[:, 1]) / 2).sum()) < 1e-14


@pytest.mark.parametrize("P,tol", [(4, 2e-3), (8, 2e-5), (14, 1e-8)])
def test_p2m_far_field_converges(P, tol):
    x, q = _cluster(30, [0, 0, 0], 0.5, 2)
    ys = np.array([[2.5, 0.3, -0.2], [-1.0, 2.2, 1.1], [0.4, -0.6, -2.7]])
    M = oracle.p2m(P, x, q, np.zeros(3))
    ref, _ = oracle.direct(np.vstack([x, ys]), np.concatenate([q, np.zeros(3)]),
                           targets=np.arange(30, 33))
    got = np.array([_eval_multipole(P, M, np.zeros(3), y) for y in ys])
    assert np.max(np.abs(got - ref)) < tol * np.max(np.abs(ref))


def test_m2m_is_exact():
    # M2M(P2M about c) == P2M about c2, coefficient by coefficient
    P = 10
    x, q = _cluster(25, [0.25, -0.25, 0.25], 0.25, 3)
    c = np.array([0.25, -0.25, 0.25])
    c2 = np.array([0.5, -0.5, 0.0])
    M = oracle.p2m(P, x, q, c)
    M2 = oracle.m2m(P, M, c, c2)
    ref = oracle.p2m(P, x, q, c2)
    assert np.max(np.abs(M2 - ref)) < 1e-14 * np.max(np.abs(ref))


@pytest.mark.parametrize("P,tol,gtol", [(4, 5e-3, 5e-2), (8, 1e-5, 5e-4), (16, 5e-10, 2e-8),
                                        (24, 1e-13, 1e-12)])
def test_m2l_l2p_converges_to_direct(P, tol, gtol):
    xs, qs = _cluster(30, [0, 0, 0], 0.5, 4)
    cL = np.array([3.0, 1.0, -1.0])
    xt, _ = _cluster(12, cL, 0.5, 5)
    M = oracle.p2m(P, xs, qs, np.zeros(3))
    L = oracle.m2l(P, M, np.zeros(3), cL)
    phi, grad = oracle.l2p(P, L, cL, xt)
    allx = np.vstack([xs, xt])
    allq = np.concatenate([qs, np.zeros(12)])
    rp, rg = oracle.direct(allx, allq, targets=np.arange(30, 42))
    assert np.max(np.abs(phi - rp)) < tol * np.max(np.abs(rp))
    assert np.max(np.abs(grad - rg)) < gtol * np.max(np.abs(rg))


def test_m2l_sign_alternation_single_charge():
    # one unit charge at the multipole centre: L_n^m = (-1)^n I_n^m(D) exactly
    P = 6
    M = np.zeros(P * P, complex)
    M[0] = 1.0
    D = np.array([1.5, -2.0, 0.7])
    L = oracle.m2l(P, M, np.zeros(3), D)
    Ih = oracle.irregular(P, D)
    for n in range(P):
        for m in range(-n, n + 1):
            assert abs(L[nm(n, m)] - (-1) ** n * Ih[nm(n, m)]) < 1e-15 * (1 + abs(Ih[nm(n, m)]))


def test_l2l_is_exact():
    # L2P(L2L(L)) == L2P(L): a degree-(P-1) polynomial translated exactly
    P = 9
    rng = np.random.default_rng(6)
    L = np.zeros(P * P, complex)
    for n in range(P):
        L[nm(n, 0)] = rng.normal()
        for m in range(1, n + 1):
            v = complex(rng.normal(), rng.normal())
            L[nm(n, m)] = v
            L[nm(n, -m)] = (-1) ** m * np.conj(v)
    c = np.array([0.0, 0.0, 0.0])
    c2 = np.array([0.3, -0.2, 0.1])
    L2 = oracle.l2l(P, L, c, c2)
    pts = c2 + rng.uniform(-0.2, 0.2, (10, 3))
    p1, g1 = oracle.l2p(P, L, c, pts)
    p2, g2 = oracle.l2p(P, L2, c2, pts)
    assert np.max(np.abs(p1 - p2)) < 1e-13 * np.max(np.abs(p1))
    assert np.max(np.abs(g1 - g2)) < 1e-12 * np.max(np.abs(g1))


def test_l2p_gradient_matches_finite_difference():
    P = 8
    xs, qs = _cluster(20, [0, 0, 0], 0.5, 7)
    cL = np.array([2.5, -1.5, 1.0])
    L = oracle.m2l(P, oracle.p2m(P, xs, qs, np.zeros(3)), np.zeros(3), cL)
    x0 = cL + np.array([0.1, -0.2, 0.15])
    _, g = oracle.l2p(P, L, cL, x0[None])
    h = 1e-5
    fd = []
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        pp, _ = oracle.l2p(P, L, cL, (x0 + e)[None])
        pm, _ = oracle.l2p(P, L, cL, (x0 - e)[None])
        fd.append((pp[0] - pm[0]) / (2 * h))
    assert np.max(np.abs(g[0] - fd)) < 1e-8 * np.max(np.abs(fd))


def test_l2p_is_real_for_symmetric_coefficients():
    P = 5
    xs, qs = _cluster(10, [0, 0, 0], 0.4, 8)
    M = oracle.p2m(P, xs, qs, np.zeros(3))
    for n in range(P):
        assert abs(M[nm(n, 0)].imag) < 1e-15
        for m in range(1, n + 1):
            assert abs(M[nm(n, -m)] - (-1) ** m * np.conj(M[nm(n, m)])) < 1e-15


def test_m2l_reciprocity():
    # Green's reciprocity: the response of L_n^m to a unit M_j^k is
    # (-1)^n I_{j+n}^{k+m}(D); swapping the roles of (n, m) and (j, k) gives
    # (-1)^j of the same harmonic, so T[nm, jk] (-1)^j == T[jk, nm] (-1)^n for
    # every pair of degrees below P. A dropped degree on either side breaks it.
    P = 7
    D = np.array([1.7, -0.9, 2.2])
    T = np.zeros((P * P, P * P), complex)
    for col in range(P * P):
        e = np.zeros(P * P, complex)
        e[col] = 1.0
        T[:, col] = oracle.m2l(P, e, np.zeros(3), D)
    deg = np.repeat(np.arange(P), 2 * np.arange(P) + 1)
    sgn = (-1.0) ** deg
    lhs = T * sgn[None, :]
    rhs = T.T * sgn[:, None]
    assert np.max(np.abs(lhs - rhs)) <= 1e-14 * np.max(np.abs(T))
    assert np.all(np.abs(T[:, deg == P - 1]).max(axis=0) > 0)
