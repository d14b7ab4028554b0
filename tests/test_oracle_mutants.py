"""The pins catch plausible mistakes: each case plants one mistake (a dropped
term, a wrong sign, a wrong index or a transposed operand) in a private copy of
the oracle's C source, builds it on the CPU, and checks that a pin fails."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_1106_2176_gb300 import inputs

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    "m2l_sign_dropped": ("L[nm(n, m)] += ((n & 1) ? -1.0 : 1.0) * s;", "L[nm(n, m)] += s;"),
    "m2l_last_degree_dropped": ("for (int j = 0; j < P; j++)\n                for (int k = -j; k <= j; k++)\n                    s += M[nm(j, k)]",
                                "for (int j = 0; j < P - 1; j++)\n                for (int k = -j; k <= j; k++)\n                    s += M[nm(j, k)]"),
    "m2m_conj_dropped": ("s += conj(R[nm(k, l)]) * M[nm(n - k, m - l)];", "s += R[nm(k, l)] * M[nm(n - k, m - l)];"),
    "m2m_order_transposed": ("s += conj(R[nm(k, l)]) * M[nm(n - k, m - l)];", "s += conj(R[nm(k, l)]) * M[nm(n - k, l - m)];"),
    "l2l_direction_flipped": ("double t[3] = {c2[0] - c[0], c2[1] - c[1], c2[2] - c[2]};",
                              "double t[3] = {c[0] - c2[0], c[1] - c2[1], c[2] - c2[2]};"),
    "legendre_coefficient": ("- (double)(n + m - 1) * Pnm[(n - 2) * P + m]", "- (double)(n + m) * Pnm[(n - 2) * P + m]"),
    "l2p_dy_sign": ("cplx dy = 0.5 * I * (get(R, a - 1, b - 1) + get(R, a - 1, b + 1));",
                    "cplx dy = -0.5 * I * (get(R, a - 1, b - 1) + get(R, a - 1, b + 1));"),
    "p2p_grad_sign": ("                    gx -= qr3 * dx;\n                    gy -= qr3 * dy;\n                    gz -= qr3 * dz;\n                }\n                ps[i] += p;",
                      "                    gx += qr3 * dx;\n                    gy -= qr3 * dy;\n                    gz -= qr3 * dz;\n                }\n                ps[i] += p;"),
    "mac_radius_inscribed": ("double lhs = 3.0 * (double)((WA + WB) * (WA + WB));", "double lhs = 1.0 * (double)((WA + WB) * (WA + WB));"),
    "tie_splits_one_side": ("if (!la && (lb || t->level[A] < t->level[B])) {", "if (!la && (lb || t->level[A] <= t->level[B])) {"),
}


def _build(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / (name + ".c")
    path.write_text(src.replace(old, new))
    so = tmp_path / (name + ".so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                           "-o", str(so), str(path), "-lm"])
    L = ctypes.CDLL(str(so))
    d = ctypes.POINTER(ctypes.c_double)
    L.orc_fmm.argtypes = [ctypes.c_int64, d, d, ctypes.c_int, ctypes.c_double, ctypes.c_int, d, d]
    L.orc_tree_build.argtypes = [ctypes.c_int64, d, ctypes.c_int, ctypes.c_double]
    L.orc_tree_build.restype = ctypes.c_void_p
    L.orc_tree_sizes.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]
    L.orc_tree_free.argtypes = [ctypes.c_void_p]
    L.orc_m2l.argtypes = [ctypes.c_int, ctypes.c_void_p, d, d, ctypes.c_void_p]
    return L


def _m2l_reciprocal(L):
    """The M2L reciprocity pin of the operator tests, on the given library."""
    P = 6
    d = ctypes.POINTER(ctypes.c_double)
    z = np.zeros(3)
    D = np.array([1.7, -0.9, 2.2])
    T = np.zeros((P * P, P * P), complex)
    for col in range(P * P):
        e = np.zeros(P * P, complex)
        e[col] = 1.0
        out = np.zeros(P * P, complex)
        L.orc_m2l(P, e.ctypes.data, z.ctypes.data_as(d), D.ctypes.data_as(d), out.ctypes.data)
        T[:, col] = out
    sgn = (-1.0) ** np.repeat(np.arange(P), 2 * np.arange(P) + 1)
    return np.max(np.abs(T * sgn[None, :] - T.T * sgn[:, None])) <= 1e-14 * np.max(np.abs(T))


def _pins_pass(L):
    """The whole-FMM accuracy pin and the list-size pin, on small inputs."""
    d = ctypes.POINTER(ctypes.c_double)
    x, q = inputs.uniform_cube(3000, 31)
    pd, gd = oracle.direct(x, q)
    phi = np.zeros(3000)
    grad = np.zeros((3000, 3))
    L.orc_fmm(3000, x.ctypes.data_as(d), q.ctypes.data_as(d), 8, 0.5, 16, phi.ctypes.data_as(d),
              grad.ctypes.data_as(d))
    ok = (np.linalg.norm(phi - pd) / np.linalg.norm(pd) < 1e-6
          and np.linalg.norm(grad - gd) / np.linalg.norm(gd) < 1e-6)
    # every ordered pair covered once: P2P interactions + M2L-covered pairs = n^2 - n
    ref = oracle.Tree(x, 16, 0.5)
    h = L.orc_tree_build(3000, x.ctypes.data_as(d), 16, 0.5)
    s = np.zeros(7, np.int64)
    L.orc_tree_sizes(h, s.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    L.orc_tree_free(h)
    ok = ok and int(s[2]) == ref.n_p2p and int(s[3]) == ref.n_m2l
    return ok and _m2l_reciprocal(L)


def test_unmutated_copy_passes(tmp_path):
    L = _build(tmp_path, "clean", "#define ORC_MAXLEVEL 21", "#define ORC_MAXLEVEL 21")
    assert _pins_pass(L)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    L = _build(tmp_path, name, old, new)
    assert not _pins_pass(L)
