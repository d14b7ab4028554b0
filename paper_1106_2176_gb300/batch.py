"""Many independent FMM systems evaluated as one CUDA graph.

Each system keeps its own handle (tree, lists, expansions). After a warm-up
evaluation nothing in fmm_evaluate allocates or synchronises, so the
evaluations of all systems are captured once into a CUDA graph and replayed
with one launch. The systems are spread over a few streams (largest first,
each to the stream with the fewest particles so far), so that small systems,
which cannot fill the GPU alone, run side by side. One launch sequence per
system, in turn, is the baseline (evaluate_each).
"""
import torch

from .fmm import FMM


class FMMBatch:
    def __init__(self, systems, p=6, theta=0.5, ncrit=64, precision="mixed", streams=8):
        """systems: list of (x (n, 3), q (n,)) CUDA tensors of one dtype."""
        self.handles, self.out = [], []
        for x, q in systems:
            f = FMM(x.shape[0], p=p, theta=theta, ncrit=ncrit, precision=precision, overlap=False)
            f.build(x, q)
            self.handles.append(f)
            self.out.append(f.evaluate())  # warm-up: every workspace exists from here on
        torch.cuda.synchronize()
        self.nstreams = max(1, int(streams))
        order = sorted(range(len(systems)), key=lambda i: -systems[i][0].shape[0])
        load = [0] * self.nstreams
        self.lane = [0] * len(systems)
        for i in order:
            s = min(range(self.nstreams), key=lambda k: load[k])
            self.lane[i] = s
            load[s] += systems[i][0].shape[0]
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
