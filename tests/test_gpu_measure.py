"""Measurement entry points: the arithmetic peaks the roofline fractions
divide by (fmm_measure_peak) and the phase times averaged over recent calls
(fmm_get_stats_mean)."""
import numpy as np
import pytest

from paper_1106_2176_gb300 import inputs

from gpu_common import ensure_built, torch_cuda

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_plausible():
    torch = torch_cuda()
    ensure_built()
    from paper_1106_2176_gb300.fmm import measure_peak
    props = torch.cuda.get_device_properties(0)
    # FP32: 128 FMA lanes per SM; the clock lies between a low power state and
    # the 2.2 GHz no Blackwell part exceeds
    lanes = props.multi_processor_count * 128 * 2
    for kind in ("fp32", "fp32x2"):
        t = measure_peak(kind, reps=2)
        assert 0.3 * lanes * 1.0e9 / 1e12 < t < lanes * 2.2e9 / 1e12, (kind, t)
    # TF32 dense is far above the CUDA cores and below the BF16 dense rate
    for n in (128, 256):
        t = measure_peak("tf32", n, reps=2)
        assert 3 * lanes * 1.0e9 / 1e12 < t < 2600.0, (n, t)


def test_stats_mean_over_recent_calls():
    torch = torch_cuda()
    ensure_built()
    from paper_1106_2176_gb300 import FMM
    from paper_1106_2176_gb300.fmm import FMMError
    x, q = inputs.uniform_cube(50000, 21, dtype=np.float32)
    f = FMM(50000, p=6, theta=0.5, ncrit=64, precision="mixed", overlap=False)
    xt, qt = torch.tensor(x, device="cuda"), torch.tensor(q, device="cuda")
    with pytest.raises(FMMError):
        f.stats(mean_of=1)  # nothing built yet
    for _ in range(40):  # more calls than the 32 timing slots
        f.build(xt, qt)
        f.evaluate()
    last = f.stats()
    one = f.stats(mean_of=1)
    for k in ("ms_build", "ms_evaluate", "ms_p2p", "ms_m2l"):
        assert one[k] == pytest.approx(last[k], rel=1e-6)
    mean = f.stats(mean_of=32)
    assert mean["ms_evaluate"] > 0 and mean["ms_p2p"] > 0 and mean["ms_build"] > 0
    # the phases of an evaluation in turn add up to at most the evaluation
    parts = sum(mean[k] for k in ("ms_p2m", "ms_m2m", "ms_m2l", "ms_l2l", "ms_l2p", "ms_p2p", "ms_combine"))
    assert parts <= mean["ms_evaluate"] * 1.01
    with pytest.raises(FMMError):
        f.stats(mean_of=33)
    f.close()
