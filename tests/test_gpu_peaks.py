"""The roofline denominators: measured pipe rates on the GPU of the run.

The tensor-core two-row step issues M128 N64 K8 and M128 N16 K8 TF32
instructions; their measured rates bound it below the N256 peak.  Rates of
smaller N may not exceed those of larger N by more than noise, the N256 rate
of the shape probe is the tensor-core figure of peps_measure_peaks, and an
unsupported N is refused before anything runs.
"""
import pytest

pytestmark = pytest.mark.gpu


def test_mma_shape_rates_are_ordered_and_match_the_peak():
    from paper_1611_09467_gb300.peps import PepsError, measure_mma_shape, measure_peaks

    peaks = measure_peaks()
    assert 0 < peaks["fp64_simt"] < peaks["fp32_simt"] < peaks["tf32_tcgen05"]
    r = {n: measure_mma_shape(n) for n in (16, 64, 256)}
    assert all(v > 0 for v in r.values())
    assert r[16] <= 1.05 * r[64] and r[64] <= 1.05 * r[256]
    assert abs(r[256] / peaks["tf32_tcgen05"] - 1.0) < 0.1
    with pytest.raises(PepsError):
        measure_mma_shape(48)
