"""Leaf-size autotuner: times build + evaluate for a few ncrit candidates and
keeps the fastest.

Sec. 3.1 of the paper balances P2P against M2L through the depth of the tree
(the number of particles per leaf); here that balance is measured instead of
guessed. For a uniform cube the tree depth changes only when ncrit crosses a
power of 8 times N / 8^l, so a handful of candidates covers it.
"""
import json
import os

DEFAULT_CANDIDATES = (32, 64, 128, 256, 512)


def tune_ncrit(x, q, p, theta, precision="mixed", candidates=DEFAULT_CANDIDATES, reps=2, cache=None, key=None):
    """Return (best_ncrit, {ncrit: ms}) for torch CUDA inputs x, q."""
    import torch
    from .fmm import FMM

    if cache and key and os.path.exists(cache):
        try:
            d = json.load(open(cache))
            if key in d:
                return int(d[key]["ncrit"]), d[key]["ms"]
        except Exception:
            pass
    from .fmm import FMMError

    times = {}
    seen_depth = {}
    for nc in candidates:
        f = FMM(x.shape[0], p=p, theta=theta, ncrit=nc, precision=precision)
        try:
            f.build(x, q)
            f.evaluate()
        except FMMError:  # e.g. lists beyond 2^31 entries for too small a leaf: not a candidate
            f.close()
            continue
        depth = f.stats()["depth"]
        sig = (depth, f.stats()["nleaves"])
        if sig in seen_depth:  # same tree as a smaller candidate: same cost
            times[nc] = times[seen_depth[sig]]
            f.close()
            continue
        seen_depth[sig] = nc
        st = torch.cuda.current_stream()
        best = float("inf")
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(st)
            f.build(x, q)
            f.evaluate()
            b.record(st)
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        times[nc] = best
        f.close()
    if not times:
        raise RuntimeError("tune_ncrit: no candidate leaf size could be built")
    best_nc = min(times, key=lambda k: (times[k], k))
    if cache and key:
        try:
            d = json.load(open(cache)) if os.path.exists(cache) else {}
            d[key] = {"ncrit": best_nc, "ms": times}
            json.dump(d, open(cache, "w"), indent=1)
        except Exception:
            pass
    return best_nc, times
