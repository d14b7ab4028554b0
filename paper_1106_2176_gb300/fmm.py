"""Python binding of the C ABI in include/fmm.h (ctypes; argument marshalling only).

Every step of the FMM runs in the CUDA kernels of libfmm.so; this module only
passes pointers, sizes and the current CUDA stream. There is no CPU path: if the
library is missing or no sm_103 GPU is present, the calls raise.

    from paper_1106_2176_gb300 import FMM
    f = FMM(N, p=8, theta=0.5, ncrit=64, precision="mixed")
    f.build(x, q)            # torch CUDA tensors (n,3) and (n,), float32 or float64
    phi, grad = f.evaluate() # torch CUDA tensors in the input order

Host numpy arrays are accepted too (the library copies them; FMM_HOST_MEM).
"""
import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "libfmm.so")
_HEADER = os.path.join(_HERE, "..", "include", "fmm.h")

FMM_OK, FMM_EINVAL, FMM_ENOMEM, FMM_ESTATE, FMM_ECUDA, FMM_ENONFINITE, FMM_ENODEV = 0, -1, -2, -3, -4, -5, -6
FMM_F32, FMM_F64, FMM_HOST_MEM = 0, 1, 0x100
FMM_FP64, FMM_MIXED = 0, 1
FMM_M2L_AUTO, FMM_M2L_TENSOR, FMM_M2L_CUDACORE, FMM_M2L_ROTATION = 0, 1, 2, 3
FMM_PEAK_FP32_FMA, FMM_PEAK_FP32X2_FMA, FMM_PEAK_TF32_MMA = 0, 1, 2

_ERRNAMES = {FMM_EINVAL: "FMM_EINVAL", FMM_ENOMEM: "FMM_ENOMEM", FMM_ESTATE: "FMM_ESTATE",
             FMM_ECUDA: "FMM_ECUDA", FMM_ENONFINITE: "FMM_ENONFINITE", FMM_ENODEV: "FMM_ENODEV"}


class FMMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_ERRNAMES.get(code, "FMM_E?"), code, msg))
        self.code = code


class fmm_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("ncells", ctypes.c_int64), ("nleaves", ctypes.c_int64),
                ("depth", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("n_p2p_pairs", ctypes.c_int64), ("n_m2l_pairs", ctypes.c_int64),
                ("n_m2l_irregular", ctypes.c_int64), ("n_interactions", ctypes.c_int64),
                ("n_stencil", ctypes.c_int64), ("m2l_engine", ctypes.c_int32), ("async_error", ctypes.c_int32),
                ("ms_build", ctypes.c_double), ("ms_evaluate", ctypes.c_double),
                ("ms_p2m", ctypes.c_double), ("ms_m2m", ctypes.c_double), ("ms_m2l", ctypes.c_double),
                ("ms_l2l", ctypes.c_double), ("ms_l2p", ctypes.c_double), ("ms_p2p", ctypes.c_double),
                ("ms_combine", ctypes.c_double), ("kernel_launches", ctypes.c_int64),
                ("uniform_path", ctypes.c_int32), ("lattice_levels", ctypes.c_int32)]


class fmm_tree_sizes(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("ncells", ctypes.c_int64), ("n_p2p", ctypes.c_int64),
                ("n_m2l", ctypes.c_int64), ("depth", ctypes.c_int32), ("p", ctypes.c_int32)]


_lib = None
_vp = ctypes.c_void_p


def declared_symbols():
    """Names of the functions include/fmm.h declares."""
    src = open(_HEADER).read()
    return sorted(set(re.findall(r"^\s*FMM_API\s+(?:int|const char \*)\s*(fmm_\w+)\s*\(", src, re.M)))


def lib():
    """Load libfmm.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIBPATH):
        raise RuntimeError("libfmm.so is not built; run paper_1106_2176_gb300._build.build()")
    L = ctypes.CDLL(_LIBPATH)
    i64, i32, d = ctypes.c_int64, ctypes.c_int, ctypes.c_double
    L.fmm_create.argtypes = [i64, i32, d, i32, ctypes.POINTER(_vp)]
    L.fmm_set_precision.argtypes = [_vp, i32]
    L.fmm_set_m2l_engine.argtypes = [_vp, i32]
    L.fmm_set_overlap.argtypes = [_vp, i32]
    L.fmm_set_m2l_pool.argtypes = [_vp, i32]
    L.fmm_set_m2l_lattice.argtypes = [_vp, ctypes.c_int]
    L.fmm_set_stream.argtypes = [_vp, _vp]
    L.fmm_set_uniform_path.argtypes = [_vp, ctypes.c_int]
    L.fmm_m2l_rotation_host.argtypes = [ctypes.c_int, _vp, _vp, _vp]
    L.fmm_build.argtypes = [_vp, _vp, _vp, i64, i32]
    L.fmm_evaluate.argtypes = [_vp, _vp, _vp]
    L.fmm_get_stats.argtypes = [_vp, ctypes.POINTER(fmm_stats)]
    L.fmm_get_stats_mean.argtypes = [_vp, i32, ctypes.POINTER(fmm_stats)]
    L.fmm_get_tree_sizes.argtypes = [_vp, ctypes.POINTER(fmm_tree_sizes)]
    L.fmm_export_tree.argtypes = [_vp] + [_vp] * 14
    L.fmm_export_expansions.argtypes = [_vp, _vp, _vp]
    L.fmm_direct.argtypes = [_vp, _vp, _vp, i64, _vp, i64, _vp, _vp]
    L.fmm_morton_sort_noalloc.argtypes = [_vp, i64, i32, _vp, _vp, _vp]
    L.fmm_update_charges.argtypes = [_vp, _vp, _vp]
    L.fmm_energy.argtypes = [_vp, _vp, _vp, _vp, ctypes.POINTER(d)]
    L.fmm_energy_adjoint.argtypes = [_vp, d, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
    L.fmm_measure_peak.argtypes = [i32, i32, i32, ctypes.POINTER(d)]
    L.fmm_batch_create.argtypes = [_vp, i32, _vp, _vp, ctypes.POINTER(_vp)]
    L.fmm_batch_evaluate.argtypes = [_vp, _vp]
    L.fmm_batch_status.argtypes = [_vp, ctypes.POINTER(i32), ctypes.POINTER(i64)]
    L.fmm_batch_items.argtypes = [_vp, i32, i64] + [ctypes.POINTER(i32)] * 4
    L.fmm_batch_withhold.argtypes = [_vp, i32, i64]
    L.fmm_batch_destroy.argtypes = [_vp]
    L.fmm_destroy.argtypes = [_vp]
    L.fmm_last_error.argtypes = [_vp]
    L.fmm_last_error.restype = ctypes.c_char_p
    for name in declared_symbols():
        getattr(L, name).restype = getattr(L, name).restype if name == "fmm_last_error" else ctypes.c_int
    _lib = L
    return L


def _check(rc, h=None):
    if rc != FMM_OK:
        msg = lib().fmm_last_error(h).decode(errors="replace")
        raise FMMError(rc, msg)


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _stream_ptr():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class FMM:
    """Handle of one FMM configuration (N, p, theta, ncrit) on the current GPU."""

    def __init__(self, N, p=8, theta=0.5, ncrit=64, precision="fp64", m2l_engine="auto", overlap=True,
                 uniform_path=True, m2l_pool=-1, m2l_lattice=True):
        self._h = _vp()
        _check(lib().fmm_create(int(N), int(p), float(theta), int(ncrit), ctypes.byref(self._h)))
        self.N, self.p, self.theta, self.ncrit = int(N), int(p), float(theta), int(ncrit)
        self.set_precision(precision)
        self.set_m2l_engine(m2l_engine)
        self.set_overlap(overlap)
        self.set_uniform_path(uniform_path)
        self.set_m2l_pool(m2l_pool)
        self.set_m2l_lattice(m2l_lattice)
        self._n = 0
        self._dtype = None
        self._host = False

    # -- configuration -------------------------------------------------------
    def set_precision(self, precision):
        mode = {"fp64": FMM_FP64, "mixed": FMM_MIXED}[precision]
        _check(lib().fmm_set_precision(self._h, mode), self._h)
        self.precision = precision

    def set_m2l_engine(self, engine):
        e = {"auto": FMM_M2L_AUTO, "tensor": FMM_M2L_TENSOR, "cudacore": FMM_M2L_CUDACORE,
             "rotation": FMM_M2L_ROTATION}[engine]
        _check(lib().fmm_set_m2l_engine(self._h, e), self._h)

    def set_overlap(self, on):
        """True: far and near field run concurrently; False: in turn (per-phase times)."""
        _check(lib().fmm_set_overlap(self._h, 1 if on else 0), self._h)
        self.overlap = bool(on)

    def set_uniform_path(self, on):
        """True: full octrees skip the traversal (lattice-stencil lists); False: always traverse."""
        _check(lib().fmm_set_uniform_path(self._h, 1 if on else 0), self._h)
        self.uniform_path = bool(on)

    def set_m2l_pool(self, max_cells):
        """Levels with at most max_cells cells pool the 8 octants' same-level M2L
        tiles (-1: the default, 4 tiles' worth; 0: never). Next build."""
        _check(lib().fmm_set_m2l_pool(self._h, int(max_cells)), self._h)
        self.m2l_pool = int(max_cells)

    def set_m2l_lattice(self, on):
        """True: the tensor-core M2L brings the sources of complete levels
        (8^4 cells and more) by TMA tile loads from a lattice copy of M~;
        False: per-row lookups and gathers everywhere. Same results. Next build."""
        _check(lib().fmm_set_m2l_lattice(self._h, 1 if on else 0), self._h)
        self.m2l_lattice = bool(on)

    # -- the two calls of the method ------------------------------------------
    def build(self, x, q):
        """x: (n, 3), q: (n,); torch CUDA tensors or host numpy arrays, float32 or float64."""
        if _is_torch(x):
            import torch
            if x.dtype not in (torch.float32, torch.float64) or q.dtype != x.dtype:
                raise TypeError("x and q must both be float32 or both float64")
            if not (x.is_cuda and q.is_cuda):
                raise TypeError("torch tensors must be on the GPU; pass numpy arrays for host memory")
            x = x.contiguous()
            q = q.contiguous()
            dt = FMM_F64 if x.dtype == torch.float64 else FMM_F32
            self._keep = (x, q)
            _check(lib().fmm_set_stream(self._h, _stream_ptr()), self._h)
            _check(lib().fmm_build(self._h, _vp(x.data_ptr()), _vp(q.data_ptr()), x.shape[0], dt), self._h)
            self._host = False
            self._torch_dtype = x.dtype
            self._device = x.device
        else:
            x = np.ascontiguousarray(x)
            if x.dtype not in (np.float32, np.float64):
                x = x.astype(np.float64)
            q = np.ascontiguousarray(q, dtype=x.dtype)
            dt = FMM_F64 if x.dtype == np.float64 else FMM_F32
            self._keep = (x, q)
            _check(lib().fmm_set_stream(self._h, None), self._h)
            _check(lib().fmm_build(self._h, _vp(x.ctypes.data), _vp(q.ctypes.data), x.shape[0], dt | FMM_HOST_MEM),
                   self._h)
            self._host = True
            self._np_dtype = x.dtype
        self._n = x.shape[0]
        self._dtype = dt
        return self

    def evaluate(self, phi=None, grad=None):
        """Potential and gradient at every particle of the last build, input order."""
        n = self._n
        if self._dtype is None:  # no build yet: the library reports FMM_ESTATE
            _check(lib().fmm_evaluate(self._h, None, None), self._h)
        if self._host:
            phi = np.empty(n, dtype=self._np_dtype) if phi is None else phi
            grad = np.empty((n, 3), dtype=self._np_dtype) if grad is None else grad
            _check(lib().fmm_evaluate(self._h, _vp(phi.ctypes.data), _vp(grad.ctypes.data)), self._h)
            return phi, grad
        import torch
        if phi is None:
            phi = torch.empty(n, dtype=self._torch_dtype, device=self._device)
        if grad is None:
            grad = torch.empty((n, 3), dtype=self._torch_dtype, device=self._device)
        _check(lib().fmm_set_stream(self._h, _stream_ptr()), self._h)
        _check(lib().fmm_evaluate(self._h, _vp(phi.data_ptr()), _vp(grad.data_ptr())), self._h)
        return phi, grad

    # -- weighted energy and its adjoint ---------------------------------------
    def update_charges(self, q, w=None):
        """New charges q (times w if given) on the built tree; same kind and dtype as at build."""
        if self._host:
            _check(lib().fmm_update_charges(self._h, _vp(q.ctypes.data), _vp(w.ctypes.data) if w is not None else None),
                   self._h)
            return
        _check(lib().fmm_set_stream(self._h, _stream_ptr()), self._h)
        _check(lib().fmm_update_charges(self._h, _vp(q.data_ptr()), _vp(w.data_ptr()) if w is not None else None),
               self._h)

    def energy(self, w, q, phi):
        """1/2 sum w q phi (FP64), device tensors of the build's dtype."""
        out = ctypes.c_double()
        _check(lib().fmm_set_stream(self._h, _stream_ptr()), self._h)
        _check(lib().fmm_energy(self._h, _vp(w.data_ptr()), _vp(q.data_ptr()), _vp(phi.data_ptr()), ctypes.byref(out)),
               self._h)
        return out.value

    def energy_adjoint(self, gE, w, q, phi, grad, psi, gpsi, dq=True, dx=True, dw=True):
        """(gE dE/dq, gE dE/dx, gE dE/dw) from the two evaluations (charges q, then w q)."""
        import torch
        n = self._n
        mk = lambda shape: torch.empty(shape, dtype=self._torch_dtype, device=self._device)
        oq = mk(n) if dq else None
        ox = mk((n, 3)) if dx else None
        ow = mk(n) if dw else None
        ptr = lambda t: _vp(t.data_ptr()) if t is not None else None
        _check(lib().fmm_set_stream(self._h, _stream_ptr()), self._h)
        _check(lib().fmm_energy_adjoint(self._h, float(gE), ptr(w), ptr(q), ptr(phi), ptr(grad), ptr(psi), ptr(gpsi),
                                        ptr(oq), ptr(ox), ptr(ow)), self._h)
        return oq, ox, ow

    # -- introspection ---------------------------------------------------------
    def stats(self, mean_of=None):
        """Counters and phase times (ms) of the last build and evaluation, or,
        with mean_of=k, the phase times averaged over the last k of each."""
        s = fmm_stats()
        if mean_of is None:
            _check(lib().fmm_get_stats(self._h, ctypes.byref(s)), self._h)
        else:
            _check(lib().fmm_get_stats_mean(self._h, int(mean_of), ctypes.byref(s)), self._h)
        return {k: getattr(s, k) for k, _ in fmm_stats._fields_}

    def tree_sizes(self):
        s = fmm_tree_sizes()
        _check(lib().fmm_get_tree_sizes(self._h, ctypes.byref(s)), self._h)
        return {k: getattr(s, k) for k, _ in fmm_tree_sizes._fields_}

    def export_tree(self):
        sz = self.tree_sizes()
        n, c = sz["n"], sz["ncells"]
        out = dict(keys=np.zeros(n, np.uint64), perm=np.zeros(n, np.int32), level=np.zeros(c, np.int32),
                   anchor=np.zeros(c, np.uint64), begin=np.zeros(c, np.int32), end=np.zeros(c, np.int32),
                   child=np.zeros(c, np.int32), nchild=np.zeros(c, np.int32), parent=np.zeros(c, np.int32),
                   p2p_ptr=np.zeros(c + 1, np.int64), p2p_idx=np.zeros(max(sz["n_p2p"], 1), np.int32),
                   m2l_ptr=np.zeros(c + 1, np.int64), m2l_idx=np.zeros(max(sz["n_m2l"], 1), np.int32),
                   box=np.zeros(4))
        order = ["keys", "perm", "level", "anchor", "begin", "end", "child", "nchild", "parent", "p2p_ptr",
                 "p2p_idx", "m2l_ptr", "m2l_idx", "box"]
        _check(lib().fmm_export_tree(self._h, *[_vp(out[k].ctypes.data) for k in order]), self._h)
        out["p2p_idx"] = out["p2p_idx"][: sz["n_p2p"]]
        out["m2l_idx"] = out["m2l_idx"][: sz["n_m2l"]]
        return out

    def export_expansions(self):
        sz = self.tree_sizes()
        M = np.zeros((sz["ncells"], self.p * self.p))
        L = np.zeros((sz["ncells"], self.p * self.p))
        _check(lib().fmm_export_expansions(self._h, _vp(M.ctypes.data), _vp(L.ctypes.data)), self._h)
        return M, L

    def direct(self, x, q, targets=None):
        """FP64 direct sum on the GPU (torch CUDA float64 tensors); targets: int64 indices or None."""
        import torch
        x = x.to(torch.float64).contiguous()
        q = q.to(torch.float64).contiguous()
        n = x.shape[0]
        if targets is None:
            nt, tp = n, None
        else:
            targets = targets.to(device=x.device, dtype=torch.int64).contiguous()
            nt, tp = targets.shape[0], _vp(targets.data_ptr())
        phi = torch.empty(nt, dtype=torch.float64, device=x.device)
        grad = torch.empty((nt, 3), dtype=torch.float64, device=x.device)
        _check(lib().fmm_set_stream(self._h, _stream_ptr()), self._h)
        _check(lib().fmm_direct(self._h, _vp(x.data_ptr()), _vp(q.data_ptr()), n, tp, nt, _vp(phi.data_ptr()),
                                _vp(grad.data_ptr())), self._h)
        return phi, grad

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().fmm_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def measure_peak(kind, param=0, reps=3):
    """Measured TFLOP/s of one pipe of the current GPU: "fp32" (scalar FMA),
    "fp32x2" (packed pair FMA) or "tf32" (tcgen05 MMA, N = param: 128 or 256)."""
    k = {"fp32": FMM_PEAK_FP32_FMA, "fp32x2": FMM_PEAK_FP32X2_FMA, "tf32": FMM_PEAK_TF32_MMA}[kind]
    out = ctypes.c_double()
    _check(lib().fmm_measure_peak(k, int(param), int(reps), ctypes.byref(out)))
    return out.value


def m2l_rotation_host(p, u, M):
    """Rotation-based M2L of one packed expansion on the host (FP64): L for
    translation u = c_L - c_M. Runs the library's host code; no GPU needed."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    M = np.ascontiguousarray(M, dtype=np.float64)
    if M.shape != (p * p,) or u.shape != (3,):
        raise ValueError("M must have p^2 entries and u 3")
    out = np.zeros(p * p)
    _check(lib().fmm_m2l_rotation_host(int(p), _vp(u.ctypes.data), _vp(M.ctypes.data), _vp(out.ctypes.data)))
    return out
