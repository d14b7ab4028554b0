"""Uniform-tree fast path (Sec. 5: on a uniform distribution the cells and
lists follow from the Morton index): on full octrees the lattice-stencil lists
give the traversal's lists, counts and bitwise the same potentials; trees that
are not full take the traversal."""
import numpy as np
import pytest

from paper_1106_2176_gb300 import inputs

from gpu_common import ensure_built, torch_cuda

pytestmark = pytest.mark.gpu

KEYS = ("ncells", "nleaves", "depth", "n_p2p_pairs", "n_m2l_pairs", "n_m2l_irregular", "n_interactions")


def _run(x, q, p, theta, ncrit, uniform_path, precision="mixed"):
    torch = torch_cuda()
    ensure_built()
    from paper_1106_2176_gb300 import FMM
    f = FMM(len(q), p=p, theta=theta, ncrit=ncrit, precision=precision, uniform_path=uniform_path)
    f.build(torch.tensor(x, device="cuda"), torch.tensor(q, device="cuda"))
    phi, grad = f.evaluate()
    s = f.stats()
    f.close()
    return phi, grad, s


@pytest.mark.parametrize("n,p,theta,ncrit,precision", [(100_000, 6, 0.5, 64, "mixed"), (40_000, 8, 0.4, 32, "fp64"),
                                                       (1_000_000, 8, 0.5, 128, "mixed")])
def test_fast_path_equals_traversal(n, p, theta, ncrit, precision):
    torch = torch_cuda()
    x, q = inputs.uniform_cube(n, 21, dtype=np.float32)
    pa, ga, sa = _run(x, q, p, theta, ncrit, True, precision)
    pb, gb, sb = _run(x, q, p, theta, ncrit, False, precision)
    assert sa["uniform_path"] == 1 and sb["uniform_path"] == 0
    for k in KEYS:
        assert sa[k] == sb[k], k
    assert sa["n_m2l_irregular"] == 0
    assert torch.equal(pa, pb) and torch.equal(ga, gb)


def test_adaptive_tree_takes_traversal():
    x, q = inputs.plummer(50_000, 4)
    _, _, s = _run(x.astype(np.float32), q.astype(np.float32), 6, 0.5, 64, True)
    assert s["uniform_path"] == 0
