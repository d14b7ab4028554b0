"""The adjoint of the weighted energy E = 1/2 sum w_i q_i phi_i, pinned on the
FP64 direct sum: the closed forms (symmetric kernel, psi the potential of the
charges w q)
    dE/dq_k = 1/2 (w_k phi_k + psi_k),   dE/dx_k = 1/2 q_k (w_k grad phi_k + grad psi_k)
against central differences of E itself."""
import numpy as np

import oracle


def _energy(x, q, w):
    phi, _ = oracle.direct(x, q)
    return 0.5 * float(np.sum(w * q * phi))


def test_energy_adjoint_closed_forms_match_central_differences():
    rng = np.random.default_rng(41)
    n = 200
    x = rng.uniform(-1, 1, (n, 3))
    q = rng.uniform(-1, 1, n)
    w = rng.standard_normal(n)
    phi, gphi = oracle.direct(x, q)
    psi, gpsi = oracle.direct(x, w * q)
    dq = 0.5 * (w * phi + psi)
    dx = 0.5 * q[:, None] * (w[:, None] * gphi + gpsi)
    h = 1e-6
    for k in (0, 17, 99, 199):
        qp, qm = q.copy(), q.copy()
        qp[k] += h
        qm[k] -= h
        fd = (_energy(x, qp, w) - _energy(x, qm, w)) / (2 * h)
        assert abs(fd - dq[k]) <= 1e-7 * (abs(dq[k]) + 1e-3)
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[k, d] += h
            xm[k, d] -= h
            fd = (_energy(xp, q, w) - _energy(xm, q, w)) / (2 * h)
            assert abs(fd - dx[k, d]) <= 1e-6 * (abs(dx[k, d]) + 1e-3)
