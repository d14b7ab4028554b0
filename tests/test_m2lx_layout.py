"""The shared-memory layout of the FP32 different-level M2L: the committed
header is what the generator writes; every lane's runs cover the (n, m)
triangle once; each load of I(u) and M~ stays inside the half-warp's tables;
and at every step of the inner loop the 16 lanes of a half-warp load 16
entries in 16 different bank pairs (a float2 entry e sits in 4-byte banks 2e,
2e+1 mod 32), so the loads are free of bank conflicts."""
import pytest

from paper_1106_2176_gb300 import m2lx_layout as ml


def test_header_is_generated():
    assert open(ml.HEADER_PATH).read() == ml.header()


@pytest.mark.parametrize("P", range(ml.PMIN, ml.PMAX + 1))
def test_runs_cover_the_triangle_once(P):
    R, C, runs = ml.layout(P)
    assert len(runs) <= 16
    got = sorted((n, m0 + i) for n, m0, ln in runs for i in range(ln))
    assert got == sorted((n, m) for n in range(P) for m in range(n + 1))
    assert all(1 <= ln <= R for _, _, ln in runs)


@pytest.mark.parametrize("P", range(ml.PMIN, ml.PMAX + 1))
def test_loads_in_bounds_and_free_of_bank_conflicts(P):
    R, C, runs = ml.layout(P)
    rp, size = ml.rowptr(P, R, C)
    Q = 2 * P - 1
    # rows do not overlap and sit on their residues
    for l in range(Q):
        assert (rp[l] - C * l) % 16 == 0
        if l:
            assert rp[l] - l >= rp[l - 1] + l - 1 + 1
    for j in range(P):
        for t in range(2 * j + R):
            entries = []
            for n, m0, ln in runs:
                e = rp[j + n] + m0 - j + t
                assert rp[j + n] - (j + n) <= e < size
                # an entry read beyond the row feeds only outputs m >= m0 + ln
                for i in range(R):
                    k = t - i - j
                    if -j <= k <= j and i < ln:
                        assert -(j + n) <= m0 + i + k <= j + n
                entries.append(e)
            assert len({e % 16 for e in entries}) == len(entries), (j, t)
