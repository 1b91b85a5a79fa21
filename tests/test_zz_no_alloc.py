"""td_loglike_batch_noalloc against td_loglike_batch, through the C ABI.

The no-alloc entry point is for callers that cannot allocate device memory
while they run (an application whose device memory is reserved by its own
pool, a hard memory cap, or a loop that must not enter cudaMalloc): its
scratch is a fixed device array inside the library.  This file is collected
last and must pass both alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

from paper_2603_06010_b300 import inputs

pytestmark = pytest.mark.gpu

CHI2_REL, DLOGL_ABS = 1e-7, 1e-3   # the bar the parity tests hold the tensor-core path to


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _both(torch, seg, R_kn):
    R = torch.from_numpy(np.ascontiguousarray(R_kn)).cuda()
    K = R.shape[0]
    ref_ll = torch.empty(K, dtype=torch.float64, device="cuda")
    ref_chi = torch.empty(K, dtype=torch.float64, device="cuda")
    seg.loglike_into(R, ref_ll, chi2=ref_chi)
    na_ll = torch.full((K,), np.nan, dtype=torch.float64, device="cuda")
    na_chi = torch.full((K,), np.nan, dtype=torch.float64, device="cuda")
    seg.loglike_noalloc_into(R, na_ll, chi2=na_chi)
    torch.cuda.synchronize()
    seg.check()
    return (ref_ll.cpu().numpy(), ref_chi.cpu().numpy(), na_ll.cpu().numpy(), na_chi.cpu().numpy())


def test_noalloc_matches_batch_entry_point_twice(torch_cuda, gpu_lib):
    from paper_2603_06010_b300 import td
    n, fs = 1500, 2048.0
    mask = np.ones(n, np.uint8)
    mask[600:700] = 0
    seg = td.Segment(inputs.acf_from_psd(n, fs), mask)
    batches = [inputs.noise_residuals(n, fs, 300, 41, mask=mask),   # first call: sets up the scratch
               inputs.noise_residuals(n, fs, 77, 43, mask=mask)]    # second call reuses it
    for R in batches:
        ref_ll, ref_chi, na_ll, na_chi = _both(torch_cuda, seg, R)
        assert np.all(np.isfinite(na_ll))
        assert np.max(np.abs(na_chi - ref_chi) / ref_chi) <= CHI2_REL
        assert np.max(np.abs(na_ll - ref_ll)) <= DLOGL_ABS


def test_noalloc_small_segment_against_oracle(torch_cuda, gpu_lib):
    """Below 512 kept samples the default precision takes ten products; so must this call."""
    import oracle
    from paper_2603_06010_b300 import td
    n, fs = 300, 2048.0
    mask = np.ones(n, np.uint8)
    mask[100:160] = 0                        # N' = 240
    acf = inputs.acf_from_psd(n, fs)
    seg = td.Segment(acf, mask)
    o = oracle.OracleSegment(acf, mask)
    for seed, K in ((51, 40), (53, 7)):
        R = inputs.noise_residuals(n, fs, K, seed, mask=mask)
        ref_ll, ref_chi, na_ll, na_chi = _both(torch_cuda, seg, R)
        exp_chi = o.chi2(R)
        exp_ll = oracle.loglike_from_chi2(exp_chi, o.logdet, o.n_kept)
        assert np.max(np.abs(na_chi - exp_chi) / exp_chi) <= CHI2_REL
        assert np.max(np.abs(na_ll - exp_ll)) <= DLOGL_ABS
        assert np.max(np.abs(na_chi - ref_chi) / ref_chi) <= CHI2_REL


def test_noalloc_largest_batch_that_fits(torch_cuda, gpu_lib):
    """N' = 8192 with K = 504 is the widest batch the fixed scratch holds."""
    from paper_2603_06010_b300 import td
    n, fs = 8192, 2048.0
    seg = td.Segment(inputs.acf_from_psd(n, fs))
    R = inputs.noise_residuals(n, fs, 504, 55)
    ref_ll, ref_chi, na_ll, na_chi = _both(torch_cuda, seg, R)
    assert np.all(np.isfinite(na_ll))
    assert np.max(np.abs(na_chi - ref_chi) / ref_chi) <= CHI2_REL
    assert np.max(np.abs(na_ll - ref_ll)) <= DLOGL_ABS


def test_noalloc_rejects_batches_beyond_its_scratch(torch_cuda, gpu_lib):
    from paper_2603_06010_b300 import td
    n = 8192
    seg = td.Segment(inputs.white_acf(n, 1.0))
    K = 600   # 8 K N' > 32 MiB
    R = torch_cuda.zeros((K, n), dtype=torch_cuda.float32, device="cuda")
    out = torch_cuda.empty(K, dtype=torch_cuda.float64, device="cuda")
    with pytest.raises(td.TdError) as e:
        seg.loglike_noalloc_into(R, out)
    assert e.value.code == td.TD_ERR_INVALID
    assert "scratch" in str(e.value)
