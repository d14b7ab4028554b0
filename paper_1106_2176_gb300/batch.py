"""Many independent FMM systems evaluated together.

Each system keeps its own handle (tree, lists, expansions), built once. Two
ways to evaluate the whole batch:

- mode "persistent" (default): the library's batch engine (fmm_batch_* in
  include/fmm.h). One evaluation is about eight launches whatever the number of
  systems; persistent kernels draw (system, phase, cell or tile) work items from
  device queues, and the upward and downward passes wait, bounded, on
  per-system level counters. The evaluation can be captured into a CUDA graph
  (capture / replay), so the whole batch is one graph launch.
- mode "graph": every system's own fmm_evaluate captured into one CUDA graph
  over a few streams (largest system first, each to the stream with the fewest
  particles so far): thousands of kernels per replay.

One launch sequence per system, in turn, is the baseline (evaluate_each).
Every mode gives each system bitwise the result of its own fmm_evaluate.
"""
import ctypes
import math

import torch

from .fmm import FMM, _check, _stream_ptr, _vp, lib

NCRIT_CANDIDATES = (32, 64, 128, 256)


def _throughput_ms(members, p, theta, ncrit, precision, streams, reps=2):
    """Time to evaluate the given systems side by side, one stream each (the
    way a batch replay runs them)."""
    hs, outs = [], []
    for x, q in members:
        f = FMM(x.shape[0], p=p, theta=theta, ncrit=ncrit, precision=precision, overlap=False)
        f.build(x, q)
        hs.append(f)
        outs.append(f.evaluate())
    torch.cuda.synchronize()
    cur = torch.cuda.current_stream()
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for i, (f, o) in enumerate(zip(hs, outs)):
            s = streams[i % len(streams)]
            s.wait_stream(cur)
            with torch.cuda.stream(s):
                f.evaluate(*o)
        for s in streams:
            cur.wait_stream(s)
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    for f in hs:
        f.close()
    return best


def size_bucket(n):
    """Half a decade of n: floor(2 log10 n)."""
    return int(math.floor(2 * math.log10(max(int(n), 1))))


def assign_streams(sizes, nstreams):
    """Largest system first, each to the stream with the fewest particles so
    far (ties to the lowest stream); returns the stream of each system."""
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    load = [0] * nstreams
    lane = [0] * len(sizes)
    for i in order:
        s = min(range(nstreams), key=lambda k: (load[k], k))
        lane[i] = s
        load[s] += int(sizes[i])
    return lane


def _engine_ms(members, p, theta, ncrit, precision, m2l_pool, reps=5):
    """Device time of one batch-engine evaluation of the given systems (best
    of reps)."""
    hs, outs = [], []
    for x, q in members:
        f = FMM(x.shape[0], p=p, theta=theta, ncrit=ncrit, precision=precision, overlap=False, m2l_pool=m2l_pool)
        f.build(x, q)
        hs.append(f)
        outs.append(f.evaluate())
    torch.cuda.synchronize()
    n = len(hs)
    b = _vp()
    _check(lib().fmm_batch_create((_vp * n)(*[f._h for f in hs]), n, (_vp * n)(*[o[0].data_ptr() for o in outs]),
                                  (_vp * n)(*[o[1].data_ptr() for o in outs]), ctypes.byref(b)))
    best = float("inf")
    try:
        for _ in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            _check(lib().fmm_batch_evaluate(b, _stream_ptr()))
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
    finally:
        lib().fmm_batch_destroy(b)
        for f in hs:
            f.close()
    return best


def tune_buckets(systems, p, theta, precision, candidates=NCRIT_CANDIDATES, nstreams=8, per_bucket=8, engine=False,
                 m2l_pool=-1):
    """ncrit per size bucket (half a decade of n). Per-system launches
    (engine=False): the candidate that evaluates up to per_bucket members of
    the bucket (spread over its sizes), side by side on nstreams streams, in
    the least time. Batch engine (engine=True): the candidate whose engine
    evaluation of up to 16 per_bucket members takes the least device time.
    Returns ({bucket: ncrit}, bucket of each system)."""
    bucket = [size_bucket(x.shape[0]) for x, _ in systems]
    streams = [torch.cuda.Stream() for _ in range(nstreams)]
    choice = {}
    for b in sorted(set(bucket)):
        members = sorted((i for i in range(len(systems)) if bucket[i] == b), key=lambda i: systems[i][0].shape[0])
        k = min(16 * per_bucket if engine else per_bucket, len(members))
        pick = [systems[members[(j * (len(members) - 1)) // max(k - 1, 1)]] for j in range(k)]
        if engine:
            ms = {nc: _engine_ms(pick, p, theta, nc, precision, m2l_pool) for nc in candidates}
        else:
            ms = {nc: _throughput_ms(pick, p, theta, nc, precision, streams) for nc in candidates}
        choice[b] = min(ms, key=lambda k: (ms[k], k))
    return choice, bucket


class FMMBatch:
    def __init__(self, systems, p=6, theta=0.5, ncrit=64, precision="mixed", streams=8, mode="persistent",
                 m2l_pool=-1):
        """systems: list of (x (n, 3), q (n,)) CUDA tensors of one dtype.
        ncrit: a leaf size for every system, "auto" for one per size bucket
        (tuned), or a {bucket: ncrit} dict from an earlier tuning.
        mode: "persistent" (the batch engine) or "graph" (per-system launches in one graph).
        m2l_pool: pooling threshold of the same-level M2L tiles (FMM.set_m2l_pool)."""
        if mode not in ("persistent", "graph"):
            raise ValueError("mode must be 'persistent' or 'graph'")
        self.mode = mode
        self.handles, self.out = [], []
        if ncrit == "auto":
            self.ncrit_by_bucket, bucket = tune_buckets(systems, p, theta, precision, nstreams=max(1, int(streams)),
                                                        engine=mode == "persistent", m2l_pool=m2l_pool)
            per = [self.ncrit_by_bucket[b] for b in bucket]
        elif isinstance(ncrit, dict):
            self.ncrit_by_bucket = dict(ncrit)
            per = [self.ncrit_by_bucket[size_bucket(x.shape[0])] for x, _ in systems]
        else:
            self.ncrit_by_bucket = None
            per = [int(ncrit)] * len(systems)
        for (x, q), nc in zip(systems, per):
            f = FMM(x.shape[0], p=p, theta=theta, ncrit=nc, precision=precision, overlap=False, m2l_pool=m2l_pool)
            f.build(x, q)
            self.handles.append(f)
            self.out.append(f.evaluate())  # warm-up: every workspace exists from here on
        torch.cuda.synchronize()
        self.nstreams = max(1, int(streams))
        self.lane = assign_streams([x.shape[0] for x, _ in systems], self.nstreams)
        self.graph = self.graph_streams = None
        self.particles = sum(int(x.shape[0]) for x, _ in systems)
        self._b = _vp()
        if mode == "persistent":
            self.reattach()

    def reattach(self):
        """(Re)creates the batch engine over the built handles: fresh work
        lists, queues and counters (after a failed evaluation, for instance)."""
        self.graph = None
        if self._b.value:
            lib().fmm_batch_destroy(self._b)
            self._b = _vp()
        n = len(self.handles)
        hs = (_vp * n)(*[f._h for f in self.handles])
        ph = (_vp * n)(*[p_.data_ptr() for p_, _ in self.out])
        gr = (_vp * n)(*[g_.data_ptr() for _, g_ in self.out])
        _check(lib().fmm_batch_create(hs, n, ph, gr, ctypes.byref(self._b)))

    def evaluate_each(self):
        """One launch sequence per system, in turn on the current stream."""
        for f, (phi, grad) in zip(self.handles, self.out):
            f.evaluate(phi, grad)
        return self.out

    def evaluate(self):
        """Every system, on the current stream: the batch engine, or in
        "graph" mode the per-system launches over the streams."""
        if self.mode == "persistent":
            _check(lib().fmm_batch_evaluate(self._b, _stream_ptr()))
            return self.out
        return self.evaluate_streams()

    def evaluate_streams(self):
        """Every system's own launch sequence, spread over the streams."""
        cur = torch.cuda.current_stream()
        streams = getattr(self, "_streams", None) or [torch.cuda.Stream() for _ in range(self.nstreams)]
        self._streams = streams
        for s in streams:
            s.wait_stream(cur)
        for i, (f, (phi, grad)) in enumerate(zip(self.handles, self.out)):
            with torch.cuda.stream(streams[self.lane[i]]):
                f.evaluate(phi, grad)
        for s in streams:
            cur.wait_stream(s)
        return self.out

    def _capture(self, fn):
        self._streams = [torch.cuda.Stream() for _ in range(self.nstreams)]
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        return g

    def capture(self):
        self.graph = self._capture(self.evaluate)

    def replay(self):
        """evaluate() as one graph launch; results in self.out."""
        if self.graph is None:
            self.capture()
        self.graph.replay()
        return self.out

    def replay_streams(self):
        """evaluate_streams() as one graph launch (thousands of kernels)."""
        if getattr(self, "graph_streams", None) is None:
            self.graph_streams = self._capture(self.evaluate_streams)
        self.graph_streams.replay()
        return self.out

    def status(self):
        """(async_error, kernels per evaluation) of the batch engine: bit 0 a
        dependency wait of the upward or downward pass gave up, bit 1 the
        tensor-core M2L, bit 2 the P2P (synchronises)."""
        e, k = ctypes.c_int(), ctypes.c_int64()
        _check(lib().fmm_batch_status(self._b, ctypes.byref(e), ctypes.byref(k)))
        return e.value, k.value

    def item(self, pass_, index):
        """Work item `index` of pass 0 (upward) or 1 (downward): (system, kind, cell, level);
        kind 0 P2M, 1 M2M, 2 L2L, 3 L2P."""
        v = [ctypes.c_int() for _ in range(4)]
        _check(lib().fmm_batch_items(self._b, int(pass_), int(index), *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def withhold(self, pass_, index):
        """Failure-detection tests: drop one work item from the queue of pass
        0 (upward) or 1 (downward); the items that depend on it time out."""
        _check(lib().fmm_batch_withhold(self._b, int(pass_), int(index)))

    def close(self):
        self.graph = self.graph_streams = None
        if getattr(self, "_b", None) and self._b.value:
            lib().fmm_batch_destroy(self._b)
            self._b = _vp()
        for f in self.handles:
            f.close()
        self.handles = []
