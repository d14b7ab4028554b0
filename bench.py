#!/usr/bin/env python3
"""FMM throughput on GB300: particles/s for the 3-D Laplace FMM.

Workload (the paper's OpenMP / strong-scaling size, Sec. 3.1 and Sec. 4):
N = 10^7 particles uniform in [-1, 1]^3, charges uniform in [-1, 1], FP32
positions and charges, p = 8 terms, theta = 0.5, ncrit picked by the
autotuner, mixed precision. One step = fmm_build + fmm_evaluate (tree, lists,
P2M, M2M, M2L, L2L, L2P, P2P, unsort) with the inputs resident in HBM.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line. With torchrun each rank runs an independent replica on
its own GPU (the single-GPU method has no exchange step); value is the sum of
the particles of all ranks divided by the slowest rank's time.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FMM particles/s at N=1e7 at ≤1e-4 rel-L2 err, mixed vs FP64; P2P % FP32 peak"
FLOP_PER_INTERACTION = 20
# leaf size of the reference arm when --ncrit is not given: the value the GPU
# arm's tuner picks for N = 10^7, p = 8, theta = 0.5 (its line records it)
REFERENCE_NCRIT = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=10_000_000)
    ap.add_argument("--p", type=int, default=8)
    ap.add_argument("--theta", type=float, default=0.5)
    ap.add_argument("--ncrit", type=int, default=0, help="0 = autotune")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--targets", type=int, default=4096, help="sampled targets for the error check")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=100_000)
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg (profiling runs)")
    ap.add_argument("--batch", type=int, default=512, help="systems in the batched-evaluation leg (0 = skip)")
    ap.add_argument("--batch-modes", default="each,graph,engine,engine_graph",
                    help="batched-evaluation modes to time (profiling runs take one)")
    ap.add_argument("--batch-pool-sweep", default="0,64,4096",
                    help="M2L tile pooling thresholds (cells) timed with the batch engine besides the default 512 ('' = none)")
    ap.add_argument("--diff-n", type=int, default=1_000_000, help="particles in the differentiation leg (0 = skip)")
    ap.add_argument("--engines-n", type=int, default=1_000_000,
                    help="particles of the M2L engine comparison at p = 8, 10, 16 (0 = skip)")
    ap.add_argument("--overlap", type=int, default=0, choices=[0, 1],
                    help="0 (default): far and near field in turn on one stream, so the P2P events time the kernel "
                         "alone; 1: on concurrent streams")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [c.strip() for c in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm_, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm_)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle on a bounded sample of the workload
# ---------------------------------------------------------------------------
def cpu_oracle_rate(n_sample, p, theta, ncrit, seed=3):
    import numpy as np
    import oracle
    from paper_1106_2176_gb300 import inputs
    x, q = inputs.uniform_cube(n_sample, seed, dtype=np.float32)
    x, q = x.astype(np.float64), q.astype(np.float64)
    t0 = time.perf_counter()
    oracle.fmm(x, q, p, theta, ncrit)
    dt = time.perf_counter() - t0
    return n_sample / dt, dt


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def cpu_baselines(ncrit3):
    """The FP64 oracle FMM on one core and on all cores for the plain, the
    precision and the scale workloads (bounded samples of the last two)."""
    import numpy as np
    import oracle
    from paper_1106_2176_gb300 import inputs
    oracle.build()
    allc = os.cpu_count() or 1
    cases = [("plain FP64: uniform cube N=16384 (full), p=6, theta=0.5, ncrit=64", 16384, 6, 0.5, 64, 1, None),
             ("precision: uniform cube, sample N=20000 of 10^6, p=10, theta=0.4, ncrit=64", 20000, 10, 0.4, 64, 1, None),
             ("scale: uniform cube, sample N=100000 of 10^7, FP32 inputs, p=8, theta=0.5, ncrit=%d" % ncrit3, 100000, 8,
              0.5, ncrit3, 3, np.float32)]
    out = []
    for desc, n, p, theta, ncrit, seed, dt in cases:
        x, q = inputs.uniform_cube(n, seed, dtype=dt or np.float64)
        x, q = x.astype(np.float64), q.astype(np.float64)
        row = {"workload": desc, "n": n}
        for cores in (1, allc):
            oracle.set_threads(cores)
            t0 = time.perf_counter()
            oracle.fmm(x, q, p, theta, ncrit)
            dt_s = time.perf_counter() - t0
            row["cores_%d" % cores] = {"seconds": dt_s, "particles_per_s": n / dt_s}
        out.append(row)
    oracle.set_threads(allc)
    return {"cpu_model": cpu_model(), "host_cores": allc, "runs": out}


def run_reference(a, rank):
    if rank != 0:
        return
    import oracle
    oracle.build()
    ncrit = a.ncrit or REFERENCE_NCRIT
    ns = a.cpu_sample
    cores = oracle.get_threads()
    for _ in range(a.warmup):
        cpu_oracle_rate(ns, a.p, a.theta, ncrit)
    times = []
    for _ in range(a.steps):
        _, dt = cpu_oracle_rate(ns, a.p, a.theta, ncrit)
        times.append(dt)
    ms = 1000.0 * sum(times) / len(times)
    value = ns / (ms / 1000.0)
    sample = ("oracle FMM (FP64, OpenMP over target cells) on N=%d of the same uniform-cube workload, p=%d, "
              "theta=%g, ncrit=%d; the FMM's cost is linear in N, so particles/s of the sample stands for "
              "the full size" % (ns, a.p, a.theta, ncrit))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": a.gpus,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "uniform cube N=%d (sampled: %d), p=%d, theta=%g, FP32 positions/charges"
                      % (a.n, ns, a.p, a.theta)},
           "cpu_baseline": {"value": value, "unit": "particles/s", "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def p2p_traffic(interactions, n):
    """DRAM bytes per P2P launch from the committed ncu summary, scaled to this
    workload by particle count; None when the kernel source changed since."""
    path = os.path.join(ROOT, "profiles", "p2p_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
        src = open(os.path.join(ROOT, "paper_1106_2176_gb300", "csrc", "p2p.cu"), "rb").read()
        if d.get("source_sha256") != hashlib.sha256(src).hexdigest():
            return None
        return d["dram_bytes"] * (n / d["n"])
    except Exception:
        return None


def phase_rooflines(phase, st, N, p, peaks, fp32_peak, tf32_peak):
    """Achieved rates of the phases other than P2P, from algorithmic bytes or
    flops per phase (the minimal work each phase must do, FP32 storage). The
    tree, M2M, L2L and the combine move data: HBM-bound, against the measured
    copy bandwidth. P2M and L2P run the regular-harmonic recurrences per
    particle: ALU-bound, against the measured FP32 FMA peak. M2L against the
    measured TF32 tensor-core peak."""
    pp4 = 4 * p * p  # bytes of one expansion
    ntri = p * (p + 1) // 2  # (n, m >= 0) terms
    nc, nl = st["ncells"], st["nleaves"]
    by = {
        # 8 LSD passes over (key 8 B, index 4 B), read and written, plus the
        # gather of the sorted float4 particles (16 B in, 16 B out)
        "build": 8 * 2 * 12 * N + 32 * N,
        # every non-root cell's multipole read once, every parent written once
        "m2m": (nc - 1) * pp4 + (nc - nl) * pp4,
        # every non-root cell's local expansion read, updated and written; its parent read
        "l2l": 3 * (nc - 1) * pp4,
        # far and near double4 and the permutation in, phi and grad (FP32) out
        "combine": 64 * N + 4 * N + 16 * N,
    }
    # per particle and (n, m >= 0) term: the recurrence step of R_n^m (a
    # complex multiply by a real and a real-complex multiply-add: 6 flop),
    # then P2M adds q conj(R) into M (4 flop); L2P forms phi (4 flop) and the
    # three gradient components from the degree below (12 flop)
    fl = {"p2m": 10 * ntri * N, "l2p": 22 * ntri * N}
    ms = {"build": phase["ms_build"], "p2m": phase["ms_p2m"], "m2m": phase["ms_m2m"], "l2l": phase["ms_l2l"],
          "l2p": phase["ms_l2p"], "combine": phase["ms_combine"]}
    hbm = float(peaks.get("hbm_gbs", 6783.5))
    out = {}
    for k, b in by.items():
        if ms[k] > 0:
            gbs = b / (ms[k] / 1000.0) / 1e9
            out[k] = {"bound": "hbm", "bytes": b, "ms": ms[k], "achieved": gbs, "peak": hbm, "unit": "GB/s",
                      "frac": gbs / hbm}
    for k, f in fl.items():
        if ms[k] > 0:
            tf = f / (ms[k] / 1000.0) / 1e12
            out[k] = {"bound": "alu", "flops": f, "ms": ms[k], "achieved": tf, "peak": fp32_peak, "unit": "TFLOP/s",
                      "frac": tf / fp32_peak}
    flops = 2.0 * p ** 4 * st["n_m2l_pairs"]
    if phase["ms_m2l"] > 0:
        tf = flops / (phase["ms_m2l"] / 1000.0) / 1e12
        out["m2l"] = {"bound": "tensor", "flops": flops, "ms": phase["ms_m2l"], "achieved": tf, "peak": tf32_peak,
                      "unit": "TFLOP/s", "frac": tf / tf32_peak,
                      "note": "useful 2 p^4 flop per pair against the measured TF32 MMA peak; the split-TF32 "
                              "scheme issues 3 MMA passes of it"}
    return out


def job_rate(n_per_rank, ms, world, dist=None, device="cpu"):
    """Whole-job rate of a step: every rank's particles over the slowest rank's
    time (MAX over ranks). Returns (particles/s, ms of the slowest rank)."""
    import torch
    if dist is not None and world > 1:
        t = torch.tensor([float(ms)], device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return n_per_rank * world / (ms / 1000.0), ms


def run_e2e(a, x, q, N, ncrit, world, dist, dev):
    """Same metric through the C ABI with pinned host buffers: every step copies
    x and q to the device and phi and grad back."""
    import torch
    from paper_1106_2176_gb300 import FMM
    xh = torch.from_numpy(x).pin_memory()
    qh = torch.from_numpy(q).pin_memory()
    ph = torch.empty(N, dtype=torch.float32).pin_memory()
    gh = torch.empty((N, 3), dtype=torch.float32).pin_memory()
    fh = FMM(N, p=a.p, theta=a.theta, ncrit=ncrit, precision=a.precision, overlap=bool(a.overlap))
    for _ in range(2):
        fh.build(xh.numpy(), qh.numpy())
        fh.evaluate(ph.numpy(), gh.numpy())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        fh.build(xh.numpy(), qh.numpy())
        fh.evaluate(ph.numpy(), gh.numpy())
    torch.cuda.synchronize()
    e2e_ms = 1000.0 * (time.perf_counter() - t0) / a.steps
    e2e_value, e2e_ms = job_rate(N, e2e_ms, world, dist, dev)
    fh.close()
    e2e = {"value": e2e_value, "unit": "particles/s", "ms_per_step": e2e_ms,
           "h2d_bytes_per_step": int(x.nbytes + q.nbytes), "d2h_bytes_per_step": int(ph.numpy().nbytes + gh.numpy().nbytes)}

    return e2e


def run_batch(a, dev):
    """Many small systems evaluated together: the batch engine (persistent
    kernels over device work queues, about eight launches per evaluation),
    directly and as one CUDA-graph launch, against every system's own launch
    sequence captured in one graph over 8 streams, and against one launch
    sequence per system in turn. Sizes log-uniform in [1e3, 1e5], even systems
    a uniform cube, odd ones a Plummer sphere, charges U[-1,1], FP32, p = 6,
    theta = 0.5, mixed precision, ncrit tuned per size bucket. Error of each
    system: relative L2 on 32 sampled targets against the library's FP64
    direct sum."""
    import numpy as np
    import torch
    from paper_1106_2176_gb300 import inputs
    from paper_1106_2176_gb300.batch import FMMBatch

    rng = np.random.default_rng(5)
    systems = []
    for k in range(a.batch):
        n = int(10 ** rng.uniform(3, 5))
        x = inputs.uniform_cube(n, 1000 + k)[0] if k % 2 == 0 else inputs.plummer(n, 1000 + k)[0]
        q = rng.uniform(-1, 1, n)
        systems.append((torch.tensor(x.astype(np.float32), device=dev), torch.tensor(q.astype(np.float32), device=dev)))
    b = FMMBatch(systems, p=6, theta=0.5, ncrit="auto", precision="mixed", streams=8, mode="persistent")

    def timed(fn, reps):
        for _ in range(max(a.warmup, 3)):
            fn()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return sum(ts) / len(ts)

    reps = max(a.steps, 3)
    modes = set(a.batch_modes.split(","))
    t_each = t_streams = t_engine = t_engine_graph = launches_each = None
    if "each" in modes:
        k0 = sum(f.stats()["kernel_launches"] for f in b.handles)
        t_each = timed(b.evaluate_each, reps)
        launches_each = (sum(f.stats()["kernel_launches"] for f in b.handles) - k0) // (reps + max(a.warmup, 3))
    if "graph" in modes:
        t_streams = timed(b.replay_streams, reps)
    if "engine" in modes:
        t_engine = timed(b.evaluate, reps)
    if "engine_graph" in modes:
        t_engine_graph = timed(b.replay, reps)
    if t_engine is None and t_engine_graph is None:
        b.evaluate()
    err, launches_engine = b.status()
    out_nc = b.ncrit_by_bucket
    e_phi = e_grad = 0.0
    for (x, q), f, (phi, grad) in zip(systems, b.handles, b.out):
        n = x.shape[0]
        t = torch.as_tensor(inputs.sample_targets(n, 32, seed=n), device=dev)
        pd, gd = f.direct(x, q, t)
        e_phi = max(e_phi, float(torch.linalg.norm(phi[t].double() - pd) / torch.linalg.norm(pd)))
        e_grad = max(e_grad, float(torch.linalg.norm(grad[t].double() - gd) / torch.linalg.norm(gd)))
    best = min([t for t in (t_engine, t_engine_graph) if t is not None] or
               [t for t in (t_streams, t_each) if t is not None])
    ratio = lambda t: t / best if t is not None else None
    out = {"workload": "%d systems, n log-uniform in [1e3, 1e5], half uniform cube, half Plummer, q U[-1,1], FP32, "
                       "p=6, theta=0.5, mixed precision" % a.batch,
           "systems": a.batch, "particles": b.particles,
           "engine_ms": t_engine, "engine_graph_ms": t_engine_graph,
           "per_system_graph_ms": t_streams, "per_system_launches_ms": t_each,
           "speedup_vs_per_system_launches": ratio(t_each), "speedup_vs_per_system_graph": ratio(t_streams),
           "particles_per_s": b.particles / (best / 1000.0), "async_error": err,
           "max_rel_l2_phi": e_phi, "max_rel_l2_grad": e_grad, "error_targets_per_system": 32,
           "ncrit_by_half_decade": {str(k / 2): v for k, v in (b.ncrit_by_bucket or {}).items()},
           "streams": b.nstreams, "kernel_launches_engine": launches_engine,
           "kernel_launches_per_system_launches": launches_each,
           "interactions": sum(int(f.stats()["n_interactions"]) for f in b.handles),
           "m2l_pairs": sum(int(f.stats()["n_m2l_pairs"]) for f in b.handles),
           "m2l_pairs_across_levels": sum(int(f.stats()["n_m2l_irregular"]) for f in b.handles)}
    # the M2L tile shape: levels with at most `pool` cells pool their 8
    # octants' tiles; the engine timed with other thresholds (same leaf sizes)
    sweep = {"512 (default)": t_engine}
    for pool in [int(v) for v in a.batch_pool_sweep.split(",") if v.strip()]:
        b.close()
        b = FMMBatch(systems, p=6, theta=0.5, ncrit=out_nc, precision="mixed", streams=8, mode="persistent", m2l_pool=pool)
        sweep[str(pool)] = timed(b.evaluate, reps)
        assert b.status()[0] == 0
    out["engine_ms_by_m2l_pool_cells"] = sweep
    b.close()
    return out


def run_diff(a, dev):
    """Weighted energy E = 1/2 sum w q phi and its gradients through the
    autograd Function: N Plummer sphere, q U[0,1]/N, w N(0,1), FP32, p = 8,
    theta = 0.5, mixed precision. One step = forward (build, evaluate, energy)
    + backward (new charges w q, evaluate, adjoint). Error: relative L2 of
    dE/dx, dE/dq on 1,024 sampled particles against the library's FP64 direct
    sums of phi and psi."""
    import numpy as np
    import torch
    from paper_1106_2176_gb300 import FMM, inputs
    from paper_1106_2176_gb300.autograd import fmm_energy

    n = a.diff_n
    x, _ = inputs.plummer(n, 7)
    rng = np.random.default_rng(107)
    q = rng.uniform(0, 1, n) / n
    w = rng.standard_normal(n)
    xt = torch.tensor(x.astype(np.float32), device=dev, requires_grad=True)
    qt = torch.tensor(q.astype(np.float32), device=dev, requires_grad=True)
    wt = torch.tensor(w.astype(np.float32), device=dev, requires_grad=True)

    def step():
        xt.grad = qt.grad = wt.grad = None
        E = fmm_energy(xt, qt, wt, p=8, theta=0.5, ncrit=64, precision="mixed")
        E.backward()
        return E

    for _ in range(max(a.warmup, 3)):
        step()
    ts = []
    for _ in range(max(a.steps, 3)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        step()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = sum(ts) / len(ts)
    t = torch.as_tensor(inputs.sample_targets(n, 1024, seed=8), device=dev)
    x64, q64, w64 = xt.detach().double(), qt.detach().double(), wt.detach().double()
    g = FMM(n, p=8, theta=0.5, ncrit=64, precision="fp64")
    phi, gphi = g.direct(x64, q64, t)
    psi, gpsi = g.direct(x64, w64 * q64, t)
    g.close()
    dq = 0.5 * (w64[t] * phi + psi)
    dx = 0.5 * q64[t, None] * (w64[t, None] * gphi + gpsi)

    def rel(u, v):
        return float(torch.linalg.norm(u.double() - v) / torch.linalg.norm(v))

    return {"workload": "weighted energy and its gradients, Plummer sphere N=%d, q U[0,1]/N, w N(0,1), FP32, p=8, "
                        "theta=0.5, ncrit=64, mixed precision" % n,
            "N": n, "ms_per_step": ms, "particles_per_s": n / (ms / 1000.0),
            "step": "forward (build, evaluate, energy) + backward (charges w q, evaluate, adjoint)",
            "rel_l2_dE_dx": rel(xt.grad[t], dx), "rel_l2_dE_dq": rel(qt.grad[t], dq), "error_targets": 1024}


def run_m2l_engines(a, dev):
    """M2L launch time of each engine at p = 8, 10, 16 on one uniform cube
    (theta = 0.5, ncrit = 64, FP32 inputs, mixed precision, far and near field
    in turn so the M2L events time the phase alone): the split-TF32 tensor-core
    contraction (p <= 11), the dense CUDA-core contraction and the rotation
    engine. Error: relative L2 of phi on 512 sampled targets against the
    library's FP64 direct sum."""
    import numpy as np
    import torch
    from paper_1106_2176_gb300 import FMM, inputs

    n = a.engines_n
    x, q = inputs.uniform_cube(n, 17, dtype=np.float32)
    xt, qt = torch.tensor(x, device=dev), torch.tensor(q, device=dev)
    t = torch.as_tensor(inputs.sample_targets(n, 512, seed=5), device=dev)
    g = FMM(n, p=2, theta=0.5, ncrit=64, precision="fp64")
    pd, _ = g.direct(xt.double(), qt.double(), t)
    g.close()
    out = {"workload": "uniform cube N=%d, FP32, theta=0.5, ncrit=64, mixed precision" % n}
    for p in (8, 10, 16):
        row = {}
        for eng in ("tensor", "cudacore", "rotation"):
            if eng == "tensor" and p > 11:
                continue
            f = FMM(n, p=p, theta=0.5, ncrit=64, precision="mixed", m2l_engine=eng, overlap=False)
            f.build(xt, qt)
            phi, grad = f.evaluate()
            ms = []
            for _ in range(2):
                f.evaluate(phi, grad)
                ms.append(f.stats()["ms_m2l"])
            st = f.stats()
            err = float(torch.linalg.norm(phi[t].double() - pd) / torch.linalg.norm(pd))
            row[eng] = {"ms_m2l": min(ms), "rel_l2_phi": err, "m2l_pairs": st["n_m2l_pairs"]}
            f.close()
        out["p%d" % p] = row
    return out


def main():
    a = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        if a.impl == "ours":
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if a.impl == "ours" else "gloo")
    if a.impl == "reference":
        run_reference(a, rank)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    import numpy as np
    from paper_1106_2176_gb300 import FMM, _build, inputs, tune

    _build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    N = a.n
    x, q = inputs.uniform_cube(N, 3 + rank, dtype=np.float32)
    xt = torch.tensor(x, device=dev)
    qt = torch.tensor(q, device=dev)

    ncrit = a.ncrit
    tune_ms = None
    if ncrit == 0:
        ncrit, tune_ms = tune.tune_ncrit(xt, qt, a.p, a.theta, precision=a.precision)
    f = FMM(N, p=a.p, theta=a.theta, ncrit=ncrit, precision=a.precision, overlap=bool(a.overlap))
    phi = torch.empty(N, dtype=torch.float32, device=dev)
    grad = torch.empty((N, 3), dtype=torch.float32, device=dev)
    for _ in range(max(a.warmup, 3)):
        f.build(xt, qt)
        f.evaluate(phi, grad)
    torch.cuda.synchronize()

    # measured peaks of the FP32 FMA pipe (scalar and packed pairs) and of
    # the TF32 tensor-core MMA: the denominators of the roofline fractions
    from paper_1106_2176_gb300.fmm import measure_peak
    pk = {"fp32_fma": measure_peak("fp32"), "fp32x2_fma": measure_peak("fp32x2"),
          "tf32_mma_n128": measure_peak("tf32", 128), "tf32_mma_n256": measure_peak("tf32", 256)}
    fp32_peak = max(pk["fp32_fma"], pk["fp32x2_fma"])
    tf32_peak = max(pk["tf32_mma_n128"], pk["tf32_mma_n256"])
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    st0 = f.stats()
    clocks = Clocks(local if os.environ.get("CUDA_VISIBLE_DEVICES") is None else local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        f.build(xt, qt)
        f.evaluate(phi, grad)
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1) / a.steps
    # phase times of the timed steps (the last min(steps, 32)): the CUDA
    # events the library recorded on its launching streams inside the region
    st1 = f.stats(mean_of=min(a.steps, 32))
    phase = {k: st1[k] for k in ("ms_build", "ms_p2m", "ms_m2m", "ms_m2l", "ms_l2l", "ms_l2p", "ms_p2p",
                                 "ms_combine", "ms_evaluate")}
    launches = (st1["kernel_launches"] - st0["kernel_launches"]) // a.steps
    value, ms = job_rate(N, ms, world, dist, dev)

    # accuracy: sampled targets against the FP64 direct sum on the GPU
    rel = lambda u, v: float(torch.linalg.norm(u - v) / torch.linalg.norm(v))
    x64, q64 = xt.double(), qt.double()
    err_phi = err_grad = None
    tg = []
    if a.targets > 0:
        tg = inputs.sample_targets(N, a.targets, seed=3)
        tgt = torch.tensor(tg, device=dev)
        pd, gd = f.direct(x64, q64, tgt)
        err_phi = rel(phi[tgt].double(), pd)
        err_grad = rel(grad[tgt].double(), gd)

    # FP64 path on the same GPU (one step, for the mixed-vs-FP64 comparison)
    fp64 = None
    if not a.no_fp64 and rank == 0 and a.targets > 0:
        f64 = FMM(N, p=a.p, theta=a.theta, ncrit=ncrit, precision="fp64")
        p64 = torch.empty(N, dtype=torch.float64, device=dev)
        g64 = torch.empty((N, 3), dtype=torch.float64, device=dev)
        f64.build(x64, q64)
        f64.evaluate(p64, g64)
        torch.cuda.synchronize()
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        f64.build(x64, q64)
        f64.evaluate(p64, g64)
        b1.record(stream)
        torch.cuda.synchronize()
        ms64 = b0.elapsed_time(b1)
        fp64 = {"value": N / (ms64 / 1000.0), "unit": "particles/s", "ms_per_step": ms64,
                "rel_l2_phi": rel(p64[tgt], pd), "rel_l2_grad": rel(g64[tgt], gd),
                "mixed_speedup": ms64 / ms}
        f64.close()
        del p64, g64

    # the same build through the dual traversal (fast path off), for the
    # comparison of the two ways of making the lists
    uni = {"used": bool(st1["uniform_path"]), "build_ms": phase["ms_build"]}
    if st1["uniform_path"]:
        f.set_uniform_path(False)
        bt = []
        for _ in range(3):
            f.build(xt, qt)
            bt.append(f.stats()["ms_build"])
        f.set_uniform_path(True)
        f.build(xt, qt)
        uni["build_ms_traversal"] = min(bt)

    # the device-buffer handle and inputs are done with: the end-to-end leg
    # through the C ABI with pinned host buffers runs with the device to itself
    f.close()
    del xt, qt, phi, grad, x64, q64
    if a.targets > 0:
        del pd, gd, tgt
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    e2e = None
    if not a.no_e2e:
        e2e = run_e2e(a, x, q, N, ncrit, world, dist, dev)

    # roofline of the dominant kernel (P2P, FP32 FMA pipe)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_nominal = nsm * 128 * 2 * sm_max * 1e6 / 1e12
    inter = st1["n_interactions"]
    p2p_avg = phase["ms_p2p"]
    achieved = FLOP_PER_INTERACTION * inter / (p2p_avg / 1000.0) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": p2p_traffic(inter, N),
                "kernel": "p2p_pr_k<2>" if a.precision == "mixed" else "p2p_k<double>",
                "peak_note": "measured: FP32 FMA-chain microbenchmark (fmm_measure_peak, best of scalar FMA and "
                             "packed f32x2 FMA, full occupancy) on this GPU before the timed region; 20 flop per "
                             "interaction",
                "peak_nominal": peak_nominal, "frac_nominal": achieved / peak_nominal,
                "peak_nominal_note": "%d SMs x 128 lanes x 2 flop x %.0f MHz (max SM clock)" % (nsm, sm_max),
                "peaks_measured_tflops": pk, "interactions": inter, "p2p_ms": p2p_avg}
    phases_roof = phase_rooflines(phase, st1, N, a.p, peaks, fp32_peak, tf32_peak)

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cb = cpu_baselines(ncrit)
        allc = cb["host_cores"]
        run3 = cb["runs"][2]["cores_%d" % allc]
        cpu = {"value": run3["particles_per_s"], "unit": "particles/s", "cores": allc, "kind": "oracle",
               "sample": "FP64 oracle FMM on N=%d of the same uniform-cube workload (p=%d, theta=%g, ncrit=%d), "
                         "%.1f s on all %d host cores (%s)" % (cb["runs"][2]["n"], a.p, a.theta, ncrit,
                                                              run3["seconds"], allc, cb["cpu_model"]),
               "configs": cb}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": world, "steps": a.steps,
               "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32" if a.precision == "mixed" else "f64", "data": "synthetic",
               "config": {"workload": "uniform cube N=%d, charges U[-1,1], FP32 positions and charges, p=%d, theta=%g, "
                                      "%s precision" % (N, a.p, a.theta, a.precision),
                          "N": N, "p": a.p, "theta": a.theta, "ncrit": ncrit, "ncrit_tuning_ms": tune_ms,
                          "precision": a.precision, "parallelism": "replicas" if world > 1 else "single",
                          "schedule": "far and near field concurrent" if a.overlap else "far field, then near field",
                          "l2": "inputs (x, q: %d MB) and the step's working set exceed the 129 MB L2"
                                % ((x.nbytes + q.nbytes) // 2 ** 20)},
               "rel_l2_phi": err_phi, "rel_l2_grad": err_grad, "error_targets": len(tg),
               "fp64": fp64, "phases_ms": phase, "tree": {k: st1[k] for k in ("ncells", "nleaves", "depth",
                                                                             "n_p2p_pairs", "n_m2l_pairs",
                                                                             "n_m2l_irregular", "n_interactions",
                                                                             "m2l_engine")},
               "roofline": roofline, "phase_rooflines": phases_roof, "cpu_baseline": cpu, "e2e": e2e,
               "gpu_launches": launches, "clocks": ck, "uniform_path": uni}
    if rank == 0:
        if world == 1 and a.batch > 0:
            out["batch"] = run_batch(a, dev)
        if world == 1 and a.diff_n > 0:
            out["differentiation"] = run_diff(a, dev)
        if world == 1 and a.engines_n > 0:
            out["m2l_engines"] = run_m2l_engines(a, dev)
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
