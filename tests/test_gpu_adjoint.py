"""Adjoint of the weighted FMM energy (fmm_update_charges, fmm_energy,
fmm_energy_adjoint behind a torch.autograd.Function) against the FP64
direct-sum gradient and against central differences of the FMM energy.

Differentiation workload: N = 10^6 Plummer sphere (scale 1, truncated at
r = 20), charges U[0,1]/N, weights N(0,1), p = 8, theta = 0.5."""
import numpy as np
import pytest

import oracle
from paper_1106_2176_gb300 import inputs

from gpu_common import ensure_built, rel, torch_cuda

pytestmark = pytest.mark.gpu


def _setup(n, seed, dtype):
    x, _ = inputs.plummer(n, seed)
    rng = np.random.default_rng(seed + 100)
    q = rng.uniform(0, 1, n) / n
    w = rng.standard_normal(n)
    return x.astype(dtype), q.astype(dtype), w.astype(dtype)


def test_adjoint_matches_direct_sum_gradient_1e6():
    torch = torch_cuda()
    ensure_built()
    from paper_1106_2176_gb300.autograd import fmm_energy
    n = 1_000_000
    x, q, w = _setup(n, 7, np.float32)
    xt = torch.tensor(x, device="cuda", requires_grad=True)
    qt = torch.tensor(q, device="cuda", requires_grad=True)
    wt = torch.tensor(w, device="cuda", requires_grad=True)
    E = fmm_energy(xt, qt, wt, p=8, theta=0.5, ncrit=64, precision="mixed")
    E.backward()
    t = inputs.sample_targets(n, 1024, seed=8)
    x64, q64, w64 = x.astype(np.float64), q.astype(np.float64), w.astype(np.float64)
    phi, gphi = oracle.direct(x64, q64, targets=t)
    psi, gpsi = oracle.direct(x64, w64 * q64, targets=t)
    dq = 0.5 * (w64[t] * phi + psi)
    dx = 0.5 * q64[t, None] * (w64[t, None] * gphi + gpsi)
    dw = 0.5 * q64[t] * phi
    assert rel(qt.grad.cpu().numpy()[t], dq) < 1e-5
    assert rel(xt.grad.cpu().numpy()[t], dx) < 1e-5
    assert rel(wt.grad.cpu().numpy()[t], dw) < 1e-5


def test_adjoint_matches_central_differences():
    # FP64 path; h = 1e-4 of a leaf's width, 16 seeded coordinates away from
    # the bounding box, so the tree does not change under the perturbation
    torch = torch_cuda()
    ensure_built()
    from paper_1106_2176_gb300 import FMM
    from paper_1106_2176_gb300.autograd import fmm_energy
    n = 20000
    x, q, w = _setup(n, 9, np.float64)
    kw = dict(p=8, theta=0.5, ncrit=64, precision="fp64")
    xt = torch.tensor(x, device="cuda", requires_grad=True)
    qt = torch.tensor(q, device="cuda", requires_grad=True)
    wt = torch.tensor(w, device="cuda")
    E = fmm_energy(xt, qt, wt, **kw)
    E.backward()
    f = FMM(n, **kw)
    f.build(torch.tensor(x, device="cuda"), torch.tensor(q, device="cuda"))
    st = f.stats()
    box = f.export_tree()["box"]
    leaf = 2.0 * box[3] / 2 ** st["depth"]
    h = 1e-4 * leaf
    rng = np.random.default_rng(10)
    r = np.linalg.norm(x, axis=1)
    inner = np.flatnonzero(r < np.quantile(r, 0.5))
    ks = rng.choice(inner, 16, replace=False)
    ds = rng.integers(0, 3, 16)

    def energy(xa):
        with torch.no_grad():
            return float(fmm_energy(torch.tensor(xa, device="cuda"), torch.tensor(q, device="cuda"), wt, **kw))

    gx = xt.grad.cpu().numpy()
    # the adjoint is the exact derivative of the exact energy evaluated with
    # the FMM's phi and psi; the derivative of the FMM energy differs from it
    # by the FMM's gradient error (p = 8: ~4e-7 relative in L2), hence the
    # floor of 1e-5 of the RMS gradient
    rms = float(np.sqrt(np.mean(gx ** 2)))
    for k, d in zip(ks, ds):
        xp, xm = x.copy(), x.copy()
        xp[k, d] += h
        xm[k, d] -= h
        fd = (energy(xp) - energy(xm)) / (2 * h)
        assert abs(fd - gx[k, d]) <= 1e-5 * abs(gx[k, d]) + 1e-5 * rms
