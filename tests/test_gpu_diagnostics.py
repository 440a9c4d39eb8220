"""The FP64 throughput probe behind the FP64 rooflines: a finite, positive
rate in the range a GPU can have, consistent with its own timing, for all
warps and for a subset."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mask,nwarp", [(0xFF, 8), (0x0, 8), (0x11, 2)])
def test_fp64_fma_rate_is_consistent(mask, nwarp):
    import torch
    import paper_2510_24175_gb300 as m
    r = m.mhd_fp64_fma_rate(mask)
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    assert r["ms"] > 0.0
    # lanes = SMs x 32 x active warps x 20000 rounds x 16 chains
    assert r["lane_fma_per_s"] == pytest.approx(
        nsm * 32 * nwarp * 20000 * 16 / (r["ms"] * 1e-3), rel=1e-6)
    # between a very slow FP64 unit and a full-rate one (64 lanes/clk/SM)
    assert 0.1 < r["lanes_per_clk_per_sm"] < 80.0
