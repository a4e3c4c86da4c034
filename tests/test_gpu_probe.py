"""mcg_issue_probe: the measured issue rates that serve as the walks'
roofline denominators.  Each must lie below the rate the GPU's unit counts
and clock allow (four schedulers x 32 lanes per SM per cycle for the
single-precision kinds) and the FP64 rate far below the FP32 one (GB300's
double-precision pipe is a small fraction of its FP32 lanes)."""
import pytest
import torch

from paper_1709_07469_gb300 import build as B
from paper_1709_07469_gb300 import mcgrav as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    B.build()
    M.load()


def test_probe_rates_are_below_the_unit_count_bound():
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    bound = sms * 4 * 32 * 2.2e9          # above GB300's 2070 MHz maximum clock
    ffma, s0 = M.mcg_issue_probe(0, 1024)
    mixed, s1 = M.mcg_issue_probe(1, 1024)
    dfma, s2 = M.mcg_issue_probe(2, 256)
    assert min(s0, s1, s2) > 0.0
    assert 0.3 * bound < ffma < bound
    assert 0.3 * bound < mixed < bound
    assert 0.0 < dfma < ffma / 8.0
