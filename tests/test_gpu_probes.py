"""The library's two machine probes (the peaks the design decisions rest on)
run and give plausible rates."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_08384_gb300 import build
    build.build()


def test_fp32_fma_rate_is_plausible():
    import paper_2609_08384_gb300 as br
    v = br.fp32_fma_rate()
    # FP32 lanes x 2 flops x clock: tens of TFLOP/s on any recent GPU, at most
    # the nominal 152 SMs x 128 lanes x 2 x 2.1 GHz on GB300
    assert 5.0 < v < 90.0, v


def test_dsmem_exchange_rate_runs_and_rejects_bad_sizes():
    import paper_2609_08384_gb300 as br
    for c in (4, 8):
        v = br.dsmem_exchange_rate(c, 96 * 1024)
        assert 0.1 < v < 100.0, (c, v)
    with pytest.raises(br.BrahmsError) as ei:
        br.dsmem_exchange_rate(3, 96 * 1024)
    assert ei.value.status == br.BRAHMS_E_ARG
