"""Seeded synthetic inputs shared by the GPU path, the oracle, the tests and the
benchmark. This module holds none of the method's arithmetic: it only draws
particle positions and charges.

The paper's test problems use randomly placed points in a cube (Sec. 3.1,
Sec. 4); the Plummer sphere stands in for a clustered astrophysical
distribution. All draws use numpy's PCG64 ``default_rng(seed)``.
"""
import numpy as np


def uniform_cube(n, seed=1, dtype=np.float64):
    """n positions uniform in [-1, 1]^3 and charges uniform in [-1, 1]."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1.0, 1.0, size=(n, 3))
    q = rng.uniform(-1.0, 1.0, size=n)
    return x.astype(dtype), q.astype(dtype)


def plummer(n, seed=4, rmax=20.0, dtype=np.float64):
    """Plummer sphere of scale radius 1 truncated at rmax (radii drawn as
    1 / sqrt(U^(-2/3) - 1), resampling those above rmax, isotropic directions),
    with charges uniform in [0, 1] / n."""
    rng = np.random.default_rng(seed)
    r = np.empty(n)
    filled = 0
    while filled < n:
        u = rng.uniform(0.0, 1.0, size=2 * (n - filled) + 16)
        u = u[u > 0.0]
        rr = 1.0 / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
        rr = rr[np.isfinite(rr) & (rr <= rmax)]
        take = min(rr.size, n - filled)
        r[filled:filled + take] = rr[:take]
        filled += take
    ct = rng.uniform(-1.0, 1.0, size=n)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=n)
    st = np.sqrt(1.0 - ct * ct)
    x = np.stack([r * st * np.cos(ph), r * st * np.sin(ph), r * ct], axis=1)
    q = rng.uniform(0.0, 1.0, size=n) / n
    return x.astype(dtype), q.astype(dtype)


def sample_targets(n, k, seed=2):
    """k distinct target indices in [0, n), sorted, drawn without replacement."""
    rng = np.random.default_rng(seed)
    k = min(k, n)
    return np.sort(rng.choice(n, size=k, replace=False)).astype(np.int64)
