"""The L2 atomic-rate measurement that bounds the transport's scoring: every
add lands (the buffer sums to the number of adds), and adds spread over an
L2-resident buffer are not slower than adds funnelled onto 32 words."""
import pytest

pytestmark = pytest.mark.gpu


def test_l2_atomic_rate_counts_every_add():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_2307_01416_gb300 import vpmc
    spread = vpmc.measure_l2_atomics(1 << 22, 64)
    assert spread["sum"] == 2 * spread["adds"] and spread["adds_per_s"] > 1e9
    funnel = vpmc.measure_l2_atomics(32, 16)
    assert funnel["sum"] == 2 * funnel["adds"]
    assert spread["adds_per_s"] > funnel["adds_per_s"]
    with pytest.raises(vpmc.VpmcError):
        vpmc.measure_l2_atomics(1000, 4)          # not a power of two
