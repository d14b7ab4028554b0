"""The lattice statements behind the full-octree fast path, checked against the
oracle's tree on full octrees (every leaf on the deepest level L, every level
full): the same-level M2L pairs of level l are, for each octant o, the stencil
vectors v with 3 < fl(theta^2 |v|^2) whose parent offset floor((o + v) / 2) is
not accepted, counted per axis as the lattice coordinates of parity o_d whose
partner x + v_d stays inside [0, 2^l); the P2P pairs are the offsets the MAC
rejects, cut at the lattice boundary of level L."""
import math

import numpy as np
import pytest

import oracle
from paper_1106_2176_gb300 import inputs


def _lattice_count(S, par, v):
    lo, hi = max(0, -v), min(S, S - v)
    if hi <= lo:
        return 0
    return (hi + 1 - par) // 2 - (lo + 1 - par) // 2


def _stencils(c, R):
    st = []
    for o in range(8):
        od = (o & 1, (o >> 1) & 1, (o >> 2) & 1)
        vs = []
        for vx in range(-R, R + 1):
            for vy in range(-R, R + 1):
                for vz in range(-R, R + 1):
                    if not (3.0 < c * float(vx * vx + vy * vy + vz * vz)):
                        continue
                    u = [math.floor((od[d] + v) / 2) for d, v in enumerate((vx, vy, vz))]
                    if 3.0 < c * float(u[0] ** 2 + u[1] ** 2 + u[2] ** 2):
                        continue
                    vs.append((vx, vy, vz))
        st.append(vs)
    return st


@pytest.mark.parametrize("n,ncrit,theta,seed", [(16384, 64, 0.5, 1), (50000, 32, 0.4, 5), (4096, 100, 0.3, 7)])
def test_closed_forms_match_oracle_lists(n, ncrit, theta, seed):
    x, _ = inputs.uniform_cube(n, seed)
    T = oracle.Tree(x, ncrit, theta)
    L = T.depth
    assert T.nleaves == 8 ** L and T.ncells == (8 ** (L + 1) - 1) // 7  # a full octree
    c = theta * theta
    R = min(2 * math.ceil(math.sqrt(3.0 / c)) + 3, 2 ** L - 1)
    st = _stencils(c, R)
    m2l = 0
    for l in range(1, L + 1):
        S = 2 ** l
        for o in range(8):
            for v in st[o]:
                m2l += (_lattice_count(S, o & 1, v[0]) * _lattice_count(S, (o >> 1) & 1, v[1]) *
                        _lattice_count(S, (o >> 2) & 1, v[2]))
    assert m2l == T.n_m2l
    # P2P: per leaf, the rejected offsets that stay inside the lattice of level L
    S = 2 ** L
    Rn = min(int(math.isqrt(int(3.0 / c) + 1)) + 2, S - 1)
    near = [(vx, vy, vz) for vx in range(-Rn, Rn + 1) for vy in range(-Rn, Rn + 1) for vz in range(-Rn, Rn + 1)
            if not (3.0 < c * float(vx * vx + vy * vy + vz * vz))]
    p2p = 0
    for v in near:
        p2p += np.prod([S - abs(vd) if abs(vd) < S else 0 for vd in v])
    assert p2p == T.n_p2p
