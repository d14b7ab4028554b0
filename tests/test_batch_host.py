"""Host logic of the batched evaluation: size buckets and the assignment of
systems to streams (largest first, least-loaded stream)."""
import numpy as np

from paper_1106_2176_gb300.batch import assign_streams, size_bucket


def test_size_buckets_are_half_decades():
    assert [size_bucket(n) for n in (1, 9, 10, 31, 32, 999, 1000, 3162, 3163, 10**5)] == [0, 1, 2, 2, 3, 5, 6, 6, 7, 10]


def test_stream_assignment_is_greedy_and_balanced():
    rng = np.random.default_rng(0)
    sizes = [int(10 ** rng.uniform(3, 5)) for _ in range(512)]
    lane = assign_streams(sizes, 8)
    assert len(lane) == 512 and set(lane) == set(range(8))
    load = np.bincount(lane, weights=sizes, minlength=8)
    # longest-processing-time bound: no stream exceeds the mean by more than the largest system
    assert load.max() - load.mean() <= max(sizes)
    assert assign_streams(sizes, 8) == lane  # deterministic


def test_stream_assignment_small_cases():
    assert assign_streams([], 4) == []
    assert assign_streams([5], 4) == [0]
    assert assign_streams([3, 3, 3], 2) == [0, 1, 0]
    assert assign_streams([1, 10, 5], 1) == [0, 0, 0]
