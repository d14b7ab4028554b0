"""Many independent FMM systems evaluated as one CUDA graph.

Each system keeps its own handle (tree, lists, expansions). After a warm-up
evaluation nothing in fmm_evaluate allocates or synchronises, so the
evaluations of all systems are captured once into a CUDA graph and replayed
with one launch. The systems are spread over a few streams (largest first,
each to the stream with the fewest particles so far), so that small systems,
which cannot fill the GPU alone, run side by side. One launch sequence per
system, in turn, is the baseline (evaluate_each).
"""
import math

import torch

from .fmm import FMM

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


def tune_buckets(systems, p, theta, precision, candidates=NCRIT_CANDIDATES, nstreams=8, per_bucket=8):
    """ncrit per size bucket (half a decade of n): the candidate that
    evaluates up to per_bucket members of the bucket (spread over its sizes),
    side by side on nstreams streams, in the least time.
    Returns ({bucket: ncrit}, bucket of each system)."""
    bucket = [size_bucket(x.shape[0]) for x, _ in systems]
    streams = [torch.cuda.Stream() for _ in range(nstreams)]
    choice = {}
    for b in sorted(set(bucket)):
        members = sorted((i for i in range(len(systems)) if bucket[i] == b), key=lambda i: systems[i][0].shape[0])
        k = min(per_bucket, len(members))
        pick = [systems[members[(j * (len(members) - 1)) // max(k - 1, 1)]] for j in range(k)]
        ms = {nc: _throughput_ms(pick, p, theta, nc, precision, streams) for nc in candidates}
        choice[b] = min(ms, key=lambda k: (ms[k], k))
    return choice, bucket


class FMMBatch:
    def __init__(self, systems, p=6, theta=0.5, ncrit=64, precision="mixed", streams=8):
        """systems: list of (x (n, 3), q (n,)) CUDA tensors of one dtype.
        ncrit: a leaf size for every system, or "auto" for one per size bucket."""
        self.handles, self.out = [], []
        if ncrit == "auto":
            self.ncrit_by_bucket, bucket = tune_buckets(systems, p, theta, precision, nstreams=max(1, int(streams)))
            per = [self.ncrit_by_bucket[b] for b in bucket]
        else:
            self.ncrit_by_bucket = None
            per = [int(ncrit)] * len(systems)
        for (x, q), nc in zip(systems, per):
            f = FMM(x.shape[0], p=p, theta=theta, ncrit=nc, precision=precision, overlap=False)
            f.build(x, q)
            self.handles.append(f)
            self.out.append(f.evaluate())  # warm-up: every workspace exists from here on
        torch.cuda.synchronize()
        self.nstreams = max(1, int(streams))
        self.lane = assign_streams([x.shape[0] for x, _ in systems], self.nstreams)
        self.graph = None
        self.particles = sum(int(x.shape[0]) for x, _ in systems)

    def evaluate_each(self):
        """One launch sequence per system, in turn on the current stream."""
        for f, (phi, grad) in zip(self.handles, self.out):
            f.evaluate(phi, grad)
        return self.out

    def capture(self):
        streams = [torch.cuda.Stream() for _ in range(self.nstreams)]
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            cap = torch.cuda.current_stream()
            for s in streams:
                s.wait_stream(cap)
            for i, (f, (phi, grad)) in enumerate(zip(self.handles, self.out)):
                with torch.cuda.stream(streams[self.lane[i]]):
                    f.evaluate(phi, grad)
            for s in streams:
                cap.wait_stream(s)
        self.graph = g
        self._streams = streams

    def replay(self):
        """Every system's evaluation, one graph launch; results in self.out."""
        if self.graph is None:
            self.capture()
        self.graph.replay()
        return self.out

    def close(self):
        self.graph = None
        for f in self.handles:
            f.close()
        self.handles = []
