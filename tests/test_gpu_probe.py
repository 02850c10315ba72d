"""The pair-rate probe behind the bench's roofline: every form the density
kernels run has a probe, each returns a plausible rate, and the 64-bit form
is not faster than the 32-bit one."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dpc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2207_04649_gb300 as m
    m.lib()
    return m


def test_probe_forms(dpc):
    rates = {}
    for d, mode in [(3, 0), (3, 1), (3, 2), (8, 0), (8, 1)]:
        r, ms = dpc.dpc_probe_pair_rate(0, d, mode)
        assert 1e10 < r < 1e14 and ms > 0
        rates[(d, mode)] = r
    assert rates[(8, 1)] <= 1.05 * rates[(8, 0)]
    assert rates[(3, 1)] <= 1.05 * rates[(3, 0)]
    for d, mode in [(4, 2), (3, 3), (0, 0), (9, 1)]:
        with pytest.raises(dpc.DpcError):
            dpc.dpc_probe_pair_rate(0, d, mode)
