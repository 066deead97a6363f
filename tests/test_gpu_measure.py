"""aqc_measure_fp64_fma: the FP64 FMA rate that the complex128 step's ALU roofline divides by."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_3938_gb300 as P

    P.build()
    yield


def test_fp64_fma_rate_is_plausible_and_scales_with_work():
    from paper_1311_3938_gb300 import _native as N

    s = torch.cuda.current_stream().cuda_stream
    tf1, ms1 = N.aqc_measure_fp64_fma(0, s, 1 << 12)
    tf2, ms2 = N.aqc_measure_fp64_fma(0, s, 1 << 14)
    # between a tenth of a TFLOP/s and more than any GPU's FP64 rate; four times the work takes
    # about four times as long once launch overhead is small
    assert 0.1 < tf2 < 200.0, tf2
    assert 2.5 < ms2 / ms1 < 5.0, (ms1, ms2)
    for bad in (0, -1, (1 << 24) + 1):
        with pytest.raises(N.AqcError) as e:
            N.aqc_measure_fp64_fma(0, s, bad)
        assert e.value.code == N.AQC_E_INVAL
