"""Rotation-based M2L (rotate the translation onto the z axis, translate
along z, rotate back; Sec. 2.2) on the host, FP64, against the oracle's dense
M2L L_n^m = (-1)^n sum M_j^k I_{j+n}^{k+m}(u) (the definition). Runs the
library's host code, no GPU."""
import numpy as np
import pytest

import oracle
from paper_1106_2176_gb300 import _build


def _packed(F, P):
    out = np.zeros(P * P)
    for n in range(P):
        for m in range(n + 1):
            v = F[oracle.nm(n, m)]
            if m == 0:
                out[n * n] = v.real
            else:
                out[n * n + 2 * m - 1] = v.real
                out[n * n + 2 * m] = v.imag
    return out


@pytest.fixture(scope="module")
def host():
    _build.build()
    from paper_1106_2176_gb300.fmm import m2l_rotation_host
    return m2l_rotation_host


# translations: generic, along +z and -z (no azimuth), in the xy plane, lattice
# vectors of a same-level stencil and a far one
U = [(3.0, 1.0, -2.0), (0.0, 0.0, 4.0), (0.0, 0.0, -5.0), (2.5, -3.5, 0.0), (-4.0, 2.0, 1.0), (1.0, 1.0, 1.0),
     (7.0, -9.0, 11.0)]


@pytest.mark.parametrize("P", [1, 2, 4, 8, 12, 16, 20])
def test_rotation_m2l_equals_dense_m2l(host, P):
    rng = np.random.default_rng(P)
    x = rng.uniform(-0.5, 0.5, (20, 3))
    q = rng.uniform(-1, 1, 20)
    M = oracle.p2m(P, x, q, np.zeros(3))
    Mp = _packed(M, P)
    for u in U:
        Lref = _packed(oracle.m2l(P, M, np.zeros(3), np.array(u)), P)
        L = host(P, u, Mp)
        # closed-form Wigner-d maps: the whole rotate-translate-rotate chain
        # stays within 1e-14 of the dense sum up to p = 20
        tol = 1e-13
        assert np.linalg.norm(L - Lref) <= tol * np.linalg.norm(Lref), (P, u)


def test_rotation_m2l_is_linear_and_rejects_bad_input(host):
    P = 6
    rng = np.random.default_rng(3)
    a, b = rng.standard_normal(P * P), rng.standard_normal(P * P)
    u = (2.0, -3.0, 1.5)
    assert np.allclose(host(P, u, a + 2 * b), host(P, u, a) + 2 * host(P, u, b), rtol=1e-13, atol=0)
    from paper_1106_2176_gb300.fmm import FMMError
    with pytest.raises(FMMError):
        host(P, (0.0, 0.0, 0.0), a)
