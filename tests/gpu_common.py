"""Helpers shared by the GPU tests: build the library once, move inputs to the
device, compare against the oracle."""
import numpy as np
import pytest

from paper_1106_2176_gb300 import _build


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


_built = False


def ensure_built():
    global _built
    if not _built:
        _build.build()
        _built = True


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run_fmm(x, q, p, theta, ncrit, precision="fp64", dtype=np.float64, engine="auto", m2l_pool=-1, m2l_lattice=True):
    """FMM through the C ABI on device tensors; returns (phi, grad, handle)."""
    torch = torch_cuda()
    ensure_built()
    from paper_1106_2176_gb300 import FMM
    xt = torch.tensor(np.asarray(x, dtype=dtype), device="cuda")
    qt = torch.tensor(np.asarray(q, dtype=dtype), device="cuda")
    f = FMM(len(q), p=p, theta=theta, ncrit=ncrit, precision=precision, m2l_engine=engine, m2l_pool=m2l_pool,
            m2l_lattice=m2l_lattice)
    f.build(xt, qt)
    phi, grad = f.evaluate()
    torch.cuda.synchronize()
    return phi.cpu().numpy().astype(np.float64), grad.cpu().numpy().astype(np.float64), f


def unscale(M, L, level, R0, p):
    """Turn exported scaled real expansions into complex full-storage ones
    (entry n*n + n + m), multiplying back by the cell widths w = 2 R0 / 2^level."""
    C = M.shape[0]
    w = 2.0 * R0 / (2.0 ** np.asarray(level, dtype=np.float64))
    outM = np.zeros((C, p * p), complex)
    outL = np.zeros((C, p * p), complex)
    for n in range(p):
        for m in range(0, n + 1):
            re = n * n + (0 if m == 0 else 2 * m - 1)
            for X, out, sc in ((M, outM, w ** n), (L, outL, w ** (-(n + 1)))):
                v = X[:, re] + (1j * X[:, n * n + 2 * m] if m else 0.0)
                v = v * sc
                out[:, n * n + n + m] = v
                out[:, n * n + n - m] = (-1) ** m * np.conj(v)
    return outM, outL
