"""Batched evaluation of many independent systems: the batch engine
(persistent kernels over device work queues, fmm_batch_* in include/fmm.h),
directly and replayed from a CUDA graph, and the per-system launches captured
in one graph, each give bitwise the results of one launch sequence per system;
each system stays within the error budget against the FP64 direct sum. A
withheld work item makes the dependency waits give up, bounded, with an error
status and a usable context. Batching workload in small: sizes log-uniform in
[10^3, 2 10^4], half uniform cube and half Plummer, charges U[-1,1], p = 6,
theta = 0.5, mixed precision; one leaf size for all, or one per size bucket
from the tuner. Each system's bound is its own FP64 FMM error on the same
targets plus 2e-6."""
import time

import numpy as np
import pytest

import oracle
from paper_1106_2176_gb300 import inputs

from gpu_common import ensure_built, rel, run_fmm, torch_cuda

pytestmark = pytest.mark.gpu

MIXED_SLACK = 2e-6


def make_systems(torch, count, seed=5, lo=3, hi=np.log10(2e4)):
    rng = np.random.default_rng(seed)
    systems, host = [], []
    for k in range(count):
        n = int(10 ** rng.uniform(lo, hi))
        x = inputs.uniform_cube(n, 500 + k)[0] if k % 2 == 0 else inputs.plummer(n, 500 + k)[0]
        q = rng.uniform(-1, 1, n)
        x32, q32 = x.astype(np.float32), q.astype(np.float32)
        host.append((x32, q32))
        systems.append((torch.tensor(x32, device="cuda"), torch.tensor(q32, device="cuda")))
    return systems, host


def clear(torch, b):
    for p, g in b.out:
        p.fill_(float("nan"))
        g.fill_(float("nan"))
    torch.cuda.synchronize()


def assert_same(b, ref):
    for i, ((p, g), (pr, gr)) in enumerate(zip(b.out, ref)):
        assert torch_equal(p, pr) and torch_equal(g, gr), i


def torch_equal(a, b):
    return bool((a == b).all()) and a.shape == b.shape


@pytest.mark.parametrize("mode,ncrit", [("persistent", 64), ("persistent", "auto"), ("graph", 64)])
def test_batch_matches_per_system_launches_and_direct_sum(mode, ncrit):
    torch = torch_cuda()
    ensure_built()
    from paper_1106_2176_gb300.batch import FMMBatch
    systems, host = make_systems(torch, 48)
    b = FMMBatch(systems, p=6, theta=0.5, ncrit=ncrit, precision="mixed", streams=8, mode=mode)
    if ncrit == "auto":
        assert b.ncrit_by_bucket and set(b.ncrit_by_bucket.values()) <= {32, 64, 128, 256}
    ref = [(p.clone(), g.clone()) for p, g in b.evaluate_each()]
    torch.cuda.synchronize()
    clear(torch, b)
    b.evaluate()
    torch.cuda.synchronize()
    assert_same(b, ref)
    if mode == "persistent":
        e, launches = b.status()
        assert e == 0 and launches <= 8
    # twice more from one graph: the queues and counters reset on the device
    for _ in range(2):
        clear(torch, b)
        b.replay()
        torch.cuda.synchronize()
        assert_same(b, ref)
    if mode == "persistent":
        assert b.status()[0] == 0
    # each system against the oracle's direct sum on 32 sampled targets:
    # within its own FP64 FMM's truncation error (same leaf size, same
    # targets) plus 2e-6
    for (x32, q32), f, (p, g) in zip(host, b.handles, b.out):
        n = len(q32)
        x64, q64 = x32.astype(np.float64), q32.astype(np.float64)
        t = inputs.sample_targets(n, 32, seed=n)
        pd, gd = oracle.direct(x64, q64, targets=t)
        p64, g64, f64 = run_fmm(x64, q64, 6, 0.5, f.ncrit, precision="fp64")
        f64.close()
        e64 = rel(p64[t], pd), rel(g64[t], gd)
        em = rel(p.cpu().numpy()[t], pd), rel(g.cpu().numpy()[t], gd)
        assert e64[0] < 1e-4 and e64[1] < 1e-4
        assert em[0] <= e64[0] + MIXED_SLACK and em[1] <= e64[1] + MIXED_SLACK, (n, em, e64)
    b.close()


@pytest.mark.parametrize("p", [3, 8, 10])
def test_batch_engine_other_orders(p):
    # p = 3 and 10 pad multipole rows to whole k-blocks; p = 8 does not
    torch = torch_cuda()
    ensure_built()
    from paper_1106_2176_gb300.batch import FMMBatch
    systems, _ = make_systems(torch, 12, seed=11, hi=4)
    b = FMMBatch(systems, p=p, theta=0.5, ncrit=64, precision="mixed")
    ref = [(x.clone(), y.clone()) for x, y in b.evaluate_each()]
    clear(torch, b)
    b.evaluate()
    torch.cuda.synchronize()
    assert_same(b, ref)
    assert b.status()[0] == 0
    b.close()


@pytest.mark.parametrize("pass_,kinds", [(0, (0,)), (0, (1,)), (1, (2,))])
def test_withheld_item_times_out_with_error_status(pass_, kinds):
    """Failure detection: one work item is removed from a queue, so the items
    that wait on its level never see it finish; their waits give up after
    about a second, set the error bit and the launch ends. The context stays
    usable and a fresh batch over the same handles is exact again."""
    torch = torch_cuda()
    ensure_built()
    from paper_1106_2176_gb300.batch import FMMBatch
    systems, _ = make_systems(torch, 6, seed=17, lo=3.5, hi=4)
    b = FMMBatch(systems, p=6, theta=0.5, ncrit=64, precision="mixed")
    ref = [(x.clone(), y.clone()) for x, y in b.evaluate_each()]
    # an item with dependants: level >= 1 upward (its parent waits), any L2L
    i = 0
    while True:
        s, kind, cell, level = b.item(pass_, i)
        if kind in kinds and level >= 1:
            break
        i += 1
    b.withhold(pass_, i)
    t0 = time.time()
    b.evaluate()
    e, _ = b.status()
    dt = time.time() - t0
    assert e & 1, e
    assert dt < 30.0
    # the context is usable: plain work and a new batch over the same handles
    z = torch.arange(1000, device="cuda", dtype=torch.float32).sum()
    assert float(z) == 999 * 1000 / 2
    b.reattach()
    clear(torch, b)
    b.evaluate()
    torch.cuda.synchronize()
    assert b.status()[0] == 0
    assert_same(b, ref)
    b.close()


def test_batch_engine_tiny_and_shallow_systems():
    # systems whose trees stop at the root (one particle, two, a handful), at
    # level 1 or 2, next to deeper ones: work lists without M2M, L2L or M2L
    # items, leaves padded to even counts, and the result still bitwise that
    # of each system's own evaluation
    torch = torch_cuda()
    ensure_built()
    from paper_1106_2176_gb300.batch import FMMBatch
    rng = np.random.default_rng(23)
    systems = []
    for k, n in enumerate([1, 2, 7, 64, 65, 500, 3000, 1, 20000]):
        x = inputs.uniform_cube(n, 700 + k)[0] if k % 2 == 0 else inputs.plummer(n, 700 + k)[0]
        q = rng.uniform(-1, 1, n)
        systems.append((torch.tensor(x.astype(np.float32), device="cuda"), torch.tensor(q.astype(np.float32), device="cuda")))
    b = FMMBatch(systems, p=6, theta=0.5, ncrit=64, precision="mixed")
    ref = [(x.clone(), y.clone()) for x, y in b.evaluate_each()]
    clear(torch, b)
    b.evaluate()
    torch.cuda.synchronize()
    assert b.status()[0] == 0
    assert_same(b, ref)
    # a single particle feels nothing
    assert float(b.out[0][0][0]) == 0.0 and torch.all(b.out[0][1] == 0)
    b.close()
