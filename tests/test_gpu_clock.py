"""The SM-clock readout of the split-product kernel (td_profile_clock,
td_group_clock): a measurement aid, checked for plausibility and for its
read-and-clear contract; it must not change any result."""
import numpy as np
import pytest

from paper_2603_06010_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_06010_b300 import td
    return torch, td


def _plausible(mhz):
    # B300: at most 2032 MHz; power and thermal limits take it lower, never to a standstill
    assert 100.0 < mhz < 2400.0, mhz


def test_segment_clock_read_and_clear(env):
    torch, td = env
    acf = inputs.acf_from_psd(2048, 2048.0)
    seg = td.Segment(acf)
    R = (torch.randn(512, 2048, device="cuda") * float(np.sqrt(acf[0]))).float()
    out = torch.empty(512, dtype=torch.float64, device="cuda")
    seg.profile(True)
    seg.loglike_into(R, out, td.options(path=td.TD_PATH_TENSOR))
    torch.cuda.synchronize()
    first = out.clone()
    _plausible(seg.profile_clock())
    with pytest.raises(td.TdError):   # cleared: nothing ran since
        seg.profile_clock()
    seg.loglike_into(R, out, td.options(path=td.TD_PATH_TENSOR))
    _plausible(seg.profile_clock())
    seg.profile(False)
    assert torch.equal(first, out)   # the readout changes no result
    seg.close()


def test_group_clock(env):
    torch, td = env
    segs, Rs, outs = [], [], []
    for n, K in ((1024, 64), (3000, 200)):
        acf = inputs.acf_from_psd(n, 4096.0)
        segs.append(td.Segment(acf))
        Rs.append((torch.randn(K, n, device="cuda") * float(np.sqrt(acf[0]))).float())
        outs.append(torch.empty(K, dtype=torch.float64, device="cuda"))
    g = td.Group(segs, Rs, outs)
    g.launch()
    g.check()
    _plausible(g.clock())
    with pytest.raises(td.TdError):
        g.clock()
    g.graph_launch()
    _plausible(g.clock())
    g.close()
    for s in segs:
        s.close()
