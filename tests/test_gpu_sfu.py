"""The measured MUFU rate is a plausible SFU issue rate.

The roofline of the operator kernels takes 16 MUFU results per clock per SM
from the CUDA throughput table; sl1m_measure_sfu measures it.  At 152 SMs and
clocks between 1.0 and 2.1 GHz, 16/clk/SM is 2.4e12 to 5.1e12 results/s;
the check allows 8 to 32 per clock at those clocks, which catches a timing
or counting mistake of 2x either way, and requires the two measurements to
be repeatable within 10%."""
import pytest

pytestmark = pytest.mark.gpu


def test_measured_mufu_rate_is_plausible_and_repeatable(gpu_lib):
    import torch
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    ctx = gpu_lib.Context(0)
    a = ctx.measure_sfu()
    b = ctx.measure_sfu()
    for k in ("sincos_per_s", "ex2_per_s"):
        for m in (a, b):
            assert 8 * n_sm * 1.0e9 <= m[k] <= 32 * n_sm * 2.1e9, (k, m[k])
        assert abs(a[k] - b[k]) <= 0.1 * max(a[k], b[k])
    ctx.close()
