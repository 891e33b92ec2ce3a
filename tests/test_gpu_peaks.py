"""The pipe-throughput probe that the roofline's peak and the operation
weights come from (mc_pipe_probe, paper_2212_02197_gb300.peaks)."""
import pytest

from paper_2212_02197_gb300 import mc, peaks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_02197_gb300 import _build

    _build.build()


def test_probe_rejects_bad_arguments():
    for kind, iters in ((-1, 16), (len(peaks.KINDS), 16), (0, 0)):
        with pytest.raises(mc.McError) as e:
            mc.pipe_probe(kind, iters)
        assert e.value.status == mc.MC_EINVAL


def test_measured_peaks_are_plausible():
    r = peaks.measure(iters=1 << 12, repeats=1)
    # GB300: FP64 fma nominally 2 per SM per clock (1.26 TFLOP/s at 2.07 GHz),
    # FP32 many times more
    assert 0.3 < r["fp64_tflops"] < 2.0, r
    assert r["fp32_tflops"] > 10 * r["fp64_tflops"], r
    w = r["weights_dfma"]
    for k in ("exp_table", "exp_lib", "div", "rcp", "log", "sqrt", "sincospi"):
        assert 1.0 < w[k] < 60.0, (k, w)
    assert w["exp_table"] < w["exp_lib"], w
