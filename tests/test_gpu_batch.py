"""Batched evaluation of many independent systems as one CUDA graph: the graph
replay gives bitwise the results of one launch sequence per system, and each
system stays within the error budget against the FP64 direct sum. Batching
workload in small: sizes log-uniform in [10^3, 2 10^4], half uniform cube and
half Plummer, charges U[-1,1], p = 6, theta = 0.5, mixed precision; one leaf
size for all, or one per size bucket from the tuner."""
import numpy as np
import pytest

import oracle
from paper_1106_2176_gb300 import inputs

from gpu_common import ensure_built, rel, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("ncrit", [64, "auto"])
def test_graph_batch_matches_per_system_launches_and_direct_sum(ncrit):
    torch = torch_cuda()
    ensure_built()
    from paper_1106_2176_gb300.batch import FMMBatch
    rng = np.random.default_rng(5)
    systems, host = [], []
    for k in range(48):
        n = int(10 ** rng.uniform(3, np.log10(2e4)))
        x = inputs.uniform_cube(n, 500 + k)[0] if k % 2 == 0 else inputs.plummer(n, 500 + k)[0]
        q = rng.uniform(-1, 1, n)
        x32, q32 = x.astype(np.float32), q.astype(np.float32)
        host.append((x32, q32))
        systems.append((torch.tensor(x32, device="cuda"), torch.tensor(q32, device="cuda")))
    b = FMMBatch(systems, p=6, theta=0.5, ncrit=ncrit, precision="mixed", streams=8)
    if ncrit == "auto":
        assert b.ncrit_by_bucket and set(b.ncrit_by_bucket.values()) <= {32, 64, 128, 256}
    ref = [(p.clone(), g.clone()) for p, g in b.evaluate_each()]
    torch.cuda.synchronize()
    for p, g in b.out:
        p.zero_()
        g.zero_()
    b.replay()
    torch.cuda.synchronize()
    for (p, g), (pr, gr) in zip(b.out, ref):
        assert torch.equal(p, pr) and torch.equal(g, gr)
    for (x32, q32), (p, g) in zip(host, b.out):
        n = len(q32)
        t = inputs.sample_targets(n, 32, seed=n)
        pd, gd = oracle.direct(x32.astype(np.float64), q32.astype(np.float64), targets=t)
        assert rel(p.cpu().numpy()[t], pd) < 1e-4 and rel(g.cpu().numpy()[t], gd) < 1e-4
    b.close()
