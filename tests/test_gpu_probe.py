"""The measured lop3.b32 rate lands near the nominal integer-logic peak the
roofline uses (148 SMs x 64 lanes/clk x the SM clock)."""
import pytest
import torch

import paper_1310_6978_b300 as F

pytestmark = pytest.mark.gpu


def test_lop3_rate_near_nominal_peak():
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = sms * 64 * 2.032e9 / 1e12
    rate = F.probe_lop3_rate()
    # below the top clock the rate drops in proportion; far above it the probe would be wrong
    assert 0.5 * nominal < rate < 1.1 * nominal, (rate, nominal)
