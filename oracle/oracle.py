"""ctypes wrapper of the FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE: only the tests, the smoke check and the CPU-baseline legs
of the benchmark use it. Expansions use full storage: entry (n, m) of an order-P
expansion, 0 <= n < P and -n <= m <= n, is at index n*n + n + m.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_i64 = ctypes.POINTER(ctypes.c_int64)
_i32 = ctypes.POINTER(ctypes.c_int32)
_u32 = ctypes.POINTER(ctypes.c_uint32)
_u64 = ctypes.POINTER(ctypes.c_uint64)
_vp = ctypes.c_void_p


def build(force=False):
    """Compile liboracle.so with gcc (FP64, no FMA contraction, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.orc_direct.argtypes = [ctypes.c_int64, _d, _d, ctypes.c_int64, _i64, _d, _d]
            L.orc_regular.argtypes = [ctypes.c_int, _d, _vp]
            L.orc_irregular.argtypes = [ctypes.c_int, _d, _vp]
            L.orc_p2m.argtypes = [ctypes.c_int, ctypes.c_int64, _d, _d, _d, _vp]
            L.orc_m2m.argtypes = [ctypes.c_int, _vp, _d, _d, _vp]
            L.orc_m2l.argtypes = [ctypes.c_int, _vp, _d, _d, _vp]
            L.orc_l2l.argtypes = [ctypes.c_int, _vp, _d, _d, _vp]
            L.orc_l2p.argtypes = [ctypes.c_int, _vp, _d, ctypes.c_int64, _d, _d, _d]
            L.orc_tree_build.argtypes = [ctypes.c_int64, _d, ctypes.c_int, ctypes.c_double]
            L.orc_tree_build.restype = _vp
            L.orc_tree_free.argtypes = [_vp]
            L.orc_tree_sizes.argtypes = [_vp, _i64]
            L.orc_tree_box.argtypes = [_vp, _d]
            L.orc_tree_particles.argtypes = [_vp, _u32, _u64, _i64]
            L.orc_tree_cells.argtypes = [_vp, _i32, _u64, _i64, _i64, _i64, _i32, _i64]
            L.orc_tree_lists.argtypes = [_vp, _i64, _i64, _i64, _i64]
            L.orc_cell_centre.argtypes = [_vp, ctypes.c_int64, _d]
            L.orc_tree_evaluate.argtypes = [_vp, _d, ctypes.c_int, _d, _d, _vp, _vp]
            L.orc_tree_evaluate.restype = ctypes.c_int
            L.orc_fmm.argtypes = [ctypes.c_int64, _d, _d, ctypes.c_int, ctypes.c_double, ctypes.c_int, _d, _d]
            L.orc_fmm.restype = ctypes.c_int
            L.orc_max_p.restype = ctypes.c_int
            L.orc_set_threads.argtypes = [ctypes.c_int]
            L.orc_get_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def nm(n, m):
    """Full-storage index of expansion entry (n, m)."""
    return n * n + n + m


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _p(a, t=_d):
    return a.ctypes.data_as(t)


def direct(x, q, targets=None):
    """FP64 direct sum; returns (phi, grad) at ``targets`` (all when None)."""
    x = _f64(x, (-1, 3))
    q = _f64(q, (-1,))
    n = x.shape[0]
    if targets is None:
        nt, tp = n, None
    else:
        t = np.ascontiguousarray(targets, dtype=np.int64)
        nt, tp = t.shape[0], _p(t, _i64)
    phi = np.zeros(nt)
    grad = np.zeros((nt, 3))
    lib().orc_direct(n, _p(x), _p(q), nt, tp, _p(phi), _p(grad))
    return phi, grad


def regular(P, x):
    out = np.zeros(P * P, dtype=np.complex128)
    lib().orc_regular(P, _p(_f64(x, (3,))), out.ctypes.data)
    return out


def irregular(P, x):
    out = np.zeros(P * P, dtype=np.complex128)
    lib().orc_irregular(P, _p(_f64(x, (3,))), out.ctypes.data)
    return out


def p2m(P, x, q, c):
    x = _f64(x, (-1, 3))
    q = _f64(q, (-1,))
    M = np.zeros(P * P, dtype=np.complex128)
    lib().orc_p2m(P, x.shape[0], _p(x), _p(q), _p(_f64(c, (3,))), M.ctypes.data)
    return M


def m2m(P, M, c, c2):
    M = np.ascontiguousarray(M, dtype=np.complex128)
    out = np.zeros(P * P, dtype=np.complex128)
    lib().orc_m2m(P, M.ctypes.data, _p(_f64(c, (3,))), _p(_f64(c2, (3,))), out.ctypes.data)
    return out


def m2l(P, M, cM, cL):
    M = np.ascontiguousarray(M, dtype=np.complex128)
    out = np.zeros(P * P, dtype=np.complex128)
    lib().orc_m2l(P, M.ctypes.data, _p(_f64(cM, (3,))), _p(_f64(cL, (3,))), out.ctypes.data)
    return out


def l2l(P, L, c, c2):
    L = np.ascontiguousarray(L, dtype=np.complex128)
    out = np.zeros(P * P, dtype=np.complex128)
    lib().orc_l2l(P, L.ctypes.data, _p(_f64(c, (3,))), _p(_f64(c2, (3,))), out.ctypes.data)
    return out


def l2p(P, L, c, x):
    L = np.ascontiguousarray(L, dtype=np.complex128)
    x = _f64(x, (-1, 3))
    phi = np.zeros(x.shape[0])
    grad = np.zeros((x.shape[0], 3))
    lib().orc_l2p(P, L.ctypes.data, _p(_f64(c, (3,))), x.shape[0], _p(x), _p(phi), _p(grad))
    return phi, grad


class Tree:
    """Morton octree plus dual-traversal interaction lists, built by the oracle."""

    def __init__(self, x, ncrit, theta):
        self._x = _f64(x, (-1, 3))
        self._h = lib().orc_tree_build(self._x.shape[0], _p(self._x), int(ncrit), float(theta))
        s = np.zeros(7, dtype=np.int64)
        lib().orc_tree_sizes(self._h, _p(s, _i64))
        (self.ncells, self.depth, self.n_p2p, self.n_m2l, self.nleaves, self.n,
         self.interactions) = [int(v) for v in s]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_tree_free(h)
            self._h = None

    def box(self):
        b = np.zeros(4)
        lib().orc_tree_box(self._h, _p(b))
        return b[:3].copy(), float(b[3])

    def particles(self):
        ic = np.zeros((self.n, 3), dtype=np.uint32)
        key = np.zeros(self.n, dtype=np.uint64)
        perm = np.zeros(self.n, dtype=np.int64)
        lib().orc_tree_particles(self._h, _p(ic, _u32), _p(key, _u64), _p(perm, _i64))
        return ic, key, perm

    def cells(self):
        c = self.ncells
        out = dict(level=np.zeros(c, np.int32), anchor=np.zeros(c, np.uint64),
                   begin=np.zeros(c, np.int64), end=np.zeros(c, np.int64),
                   child=np.zeros(c, np.int64), nchild=np.zeros(c, np.int32),
                   parent=np.zeros(c, np.int64))
        lib().orc_tree_cells(self._h, _p(out["level"], _i32), _p(out["anchor"], _u64),
                             _p(out["begin"], _i64), _p(out["end"], _i64), _p(out["child"], _i64),
                             _p(out["nchild"], _i32), _p(out["parent"], _i64))
        return out

    def lists(self):
        c = self.ncells
        pp = np.zeros(c + 1, np.int64)
        pi = np.zeros(max(self.n_p2p, 1), np.int64)
        mp = np.zeros(c + 1, np.int64)
        mi = np.zeros(max(self.n_m2l, 1), np.int64)
        lib().orc_tree_lists(self._h, _p(pp, _i64), _p(pi, _i64), _p(mp, _i64), _p(mi, _i64))
        return (pp, pi[: self.n_p2p]), (mp, mi[: self.n_m2l])

    def centre(self, c):
        out = np.zeros(3)
        lib().orc_cell_centre(self._h, int(c), _p(out))
        return out

    def evaluate(self, q, P, expansions=False):
        q = _f64(q, (-1,))
        phi = np.zeros(self.n)
        grad = np.zeros((self.n, 3))
        M = L = None
        mp = lp = None
        if expansions:
            M = np.zeros((self.ncells, P * P), dtype=np.complex128)
            L = np.zeros((self.ncells, P * P), dtype=np.complex128)
            mp, lp = M.ctypes.data, L.ctypes.data
        rc = lib().orc_tree_evaluate(self._h, _p(q), int(P), _p(phi), _p(grad), mp, lp)
        if rc != 0:
            raise ValueError("oracle evaluate rejected P=%r" % P)
        if expansions:
            return phi, grad, M, L
        return phi, grad


def fmm(x, q, P, theta, ncrit):
    """Whole FMM: (phi, grad) in input order."""
    x = _f64(x, (-1, 3))
    q = _f64(q, (-1,))
    phi = np.zeros(x.shape[0])
    grad = np.zeros((x.shape[0], 3))
    rc = lib().orc_fmm(x.shape[0], _p(x), _p(q), int(P), float(theta), int(ncrit), _p(phi), _p(grad))
    if rc != 0:
        raise ValueError("oracle fmm rejected its arguments")
    return phi, grad


def set_threads(n):
    """Threads of the oracle's OpenMP loops over targets (results do not depend on it)."""
    lib().orc_set_threads(int(n))


def get_threads():
    return int(lib().orc_get_threads())
