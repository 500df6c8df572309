"""The FP64 instruction-mix probe (rot_measure_fp64_mix): every mix runs and
reports a rate within the device's nominal FP64 pipe, and the rotation mix the
kernels use (rounded products as DFMAs with a -0 addend) issues at least as
fast as the same mix with DMUL products -- the reason the kernels use it."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_01852_gb300 import api, build
    build.build()
    return api


def test_fp64_mix_probe_rates(api):
    props = torch.cuda.get_device_properties(0)
    nominal = props.multi_processor_count * 2 * 2.1e9      # FP64 lanes per second, above the max clock
    rates = {}
    for kind in api.FP64_MIX_KINDS:
        r, ms = api.measure_fp64_mix(kind, 8, 2)
        assert ms > 0
        assert 0 < r <= 1.05 * nominal, (kind, r)
        rates[kind] = r
    assert rates["rotation_fma_smem"] >= 0.98 * rates["rotation_smem"], rates
