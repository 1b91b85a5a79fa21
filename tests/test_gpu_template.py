"""Template-input form (fixed data vector, templates per evaluation) and the
SNRs of Sec. II.B item 7 against the CPU FP64 oracle's definitions."""
import numpy as np
import pytest

import oracle
from paper_2603_06010_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _case(n=2048, fs=2048.0, gaps=2, K=40):
    seg_in = inputs.make_segment(n, fs, 6006, n_gaps=gaps, gap_len=256)
    H = inputs.template_batch(seg_in, K, 6007)
    return seg_in, H


@pytest.mark.parametrize("gaps", [0, 2])
def test_template_batch_matches_oracle(torch_cuda, gpu_lib, gaps):
    from paper_2603_06010_b300 import td
    seg_in, H = _case(gaps=gaps)
    d = seg_in.d[seg_in.kept]
    o = oracle.OracleSegment(seg_in.acf, seg_in.mask)
    seg = td.Segment(seg_in.acf, seg_in.mask)
    seg.set_data(d)
    dd_exp = oracle.inner(o, d, d)
    assert abs(seg.data_inner - dd_exp) <= 1e-7 * dd_exp
    K = H.shape[0]
    Hd = torch_cuda.from_numpy(H).cuda()
    out = {k: torch_cuda.empty(K, dtype=torch_cuda.float64, device="cuda")
           for k in ("logL", "chi2", "hh", "dh", "rho_mf", "rho_eff2")}
    seg.template_into(Hd, out["logL"], chi2=out["chi2"], hh=out["hh"], dh=out["dh"], rho_mf=out["rho_mf"],
                      rho_eff2=out["rho_eff2"])
    torch_cuda.cuda.synchronize()
    seg.check()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    H64 = H.astype(np.float64)
    R = d[None, :] - H64                     # exact d - h (the oracle's definition)
    chi2 = o.chi2(R)
    ll = oracle.loglike_from_chi2(chi2, o.logdet, o.n_kept)
    assert np.max(np.abs(got["chi2"] - chi2) / chi2) <= 1e-7
    assert np.max(np.abs(got["logL"] - ll)) <= 1e-3
    for k in range(0, K, 7):
        h = H64[k]
        hh = oracle.inner(o, h, h)
        assert abs(got["hh"][k] - hh) <= 1e-6 * hh + 1e-9
        assert abs(got["rho_mf"][k] - oracle.mf_snr(o, d, h)) <= 1e-5 * max(1.0, abs(got["rho_mf"][k]))
        assert abs(got["rho_eff2"][k] - oracle.eff_snr2(o, d, h)) <= 1e-3
        assert abs(got["dh"][k] - oracle.inner(o, d, h)) <= 1e-3
    seg.close()


def test_template_logl_equals_residual_path(torch_cuda, gpu_lib):
    """Without the SNR outputs the batch is exactly the residual path on fl32(d - h)."""
    from paper_2603_06010_b300 import td
    seg_in, H = _case(gaps=1, K=24)
    d = seg_in.d[seg_in.kept]
    seg = td.Segment(seg_in.acf, seg_in.mask)
    seg.set_data(d)
    Hd = torch_cuda.from_numpy(H).cuda()
    ll = torch_cuda.empty(H.shape[0], dtype=torch_cuda.float64, device="cuda")
    seg.template_into(Hd, ll)
    R = (d[None, :] - H.astype(np.float64)).astype(np.float32)
    ll2 = seg.loglike(torch_cuda.from_numpy(R).cuda())
    torch_cuda.cuda.synchronize()
    assert np.array_equal(ll.cpu().numpy(), ll2.cpu().numpy())
    seg.close()


def test_template_needs_data(torch_cuda, gpu_lib):
    from paper_2603_06010_b300 import td
    seg_in, H = _case(gaps=0, K=2)
    seg = td.Segment(seg_in.acf, seg_in.mask)
    ll = torch_cuda.empty(2, dtype=torch_cuda.float64, device="cuda")
    with pytest.raises(td.TdError):
        seg.template_into(torch_cuda.from_numpy(H).cuda(), ll)
    seg.close()
