"""The pair-rate probes behind the bench's rooflines: every form the density
kernels run has a probe, and so does the ring search's expanded form; each
returns a plausible rate, the 64-bit form is not faster than the 32-bit one,
and the ring's test is not faster than the density test it contains."""
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
    for d, mode in [(3, 0), (3, 1), (3, 2), (8, 0), (8, 1), (3, 3), (2, 3), (4, 2), (4, 3)]:
        r, ms = dpc.dpc_probe_pair_rate(0, d, mode)
        assert 1e10 < r < 1e14 and ms > 0
        rates[(d, mode)] = r
    assert rates[(8, 1)] <= 1.05 * rates[(8, 0)]
    assert rates[(3, 1)] <= 1.05 * rates[(3, 0)]
    # the ring search's test does the density test's work and more
    assert rates[(3, 3)] <= 1.05 * rates[(3, 2)]
    for d, mode in [(5, 2), (5, 3), (3, 4), (0, 0), (9, 1)]:
        with pytest.raises(dpc.DpcError):
            dpc.dpc_probe_pair_rate(0, d, mode)
