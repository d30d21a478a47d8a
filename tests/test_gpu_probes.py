"""The measurement library's probes run and give rates in the range the GB300's units allow (needs a GPU)."""
import pytest
import torch

from paper_1401_7494_gb300 import probes, rct

pytestmark = pytest.mark.gpu


def test_probe_rates_are_plausible(cuda_device):
    sms = torch.cuda.get_device_properties(cuda_device).multi_processor_count
    clk = 2.2e9                                          # above the maximum SM clock
    l1 = probes.rct_probe_l1_bandwidth(1024)
    assert 0.2 * 128 * sms * 1.0e9 < l1 < 1.05 * 128 * sms * clk, l1      # at most 128 B/clk/SM
    l2 = probes.rct_probe_l2_sectors(512)
    assert 1e10 < l2 < l1 / 32, l2                       # sectors from L2: well below the L1 path
    hbm = probes.rct_probe_update_stream(1 << 30)
    assert 1e12 < hbm < 1e13, hbm
    pair = probes.rct_probe_texture(5, rct.RCT_PROJ_F32, 2.6, 2.6, 512)
    assert pair > 1e10


def test_gather_pattern_probe_orders_footprints(cuda_device):
    """The footprint probe: lanes on one cell or along one row (a few cache lines) gather much faster than
    lanes spread over four rows ten pixels apart; the first two both run at the probe's instruction rate
    (measured 0.999e12 and 1.012e12 cells/s on one box), so they are compared within noise only.  Its limits
    are checked."""
    import numpy as np
    same = np.zeros((32, 2))
    row = np.stack([np.arange(32) * 3.0, np.zeros(32)], axis=1)            # 93 px of one row
    spread = np.stack([(np.arange(32) % 8) * 10.0, (np.arange(32) // 8) * 10.0], axis=1)
    r_same = probes.rct_probe_gather_pattern(same, 0.0, 10.4, 256)
    r_row = probes.rct_probe_gather_pattern(row, 0.0, 10.4, 256)
    r_spread = probes.rct_probe_gather_pattern(spread, 0.0, 10.4, 256)
    assert r_same > 0.9 * r_row and min(r_same, r_row) > 1.3 * r_spread and r_spread > 1e9, (r_same, r_row, r_spread)
    with pytest.raises(rct.RctError):
        probes.rct_probe_gather_pattern(np.stack([np.zeros(32), np.arange(32) * 2.0], axis=1), 0.0, 1.0, 64)


def test_probe_argument_errors(cuda_device):
    for call in (lambda: probes.rct_probe_l1_bandwidth(1), lambda: probes.rct_probe_l2_sectors(0),
                 lambda: probes.rct_probe_texture(9, rct.RCT_PROJ_F32, 1.0, 1.0, 64),
                 lambda: probes.rct_probe_update_stream(10)):
        with pytest.raises(rct.RctError) as e:
            call()
        assert e.value.status == rct.RCT_EINVAL
