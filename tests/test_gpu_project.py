"""Detector projection and placement fused ahead of the template path
(Sec. II.B waveform conditioning, Sec. III.A data projection and
conditioning) against the CPU FP64 oracle."""
import ctypes

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


def _dev(torch, *arrays):
    return [None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


def _outs(torch, K):
    return {k: torch.empty(K, dtype=torch.float64, device="cuda")
            for k in ("logL", "chi2", "hh", "dh", "rho_mf", "rho_eff2")}


@pytest.mark.parametrize("gaps,lw", [(0, 1024), (2, 1024), (2, 3000), (3, 77)])
def test_project_matches_oracle(torch_cuda, gpu_lib, gaps, lw):
    from paper_2603_06010_b300 import td
    n, K = 2048, 37
    seg_in = inputs.make_segment(n, 2048.0, 7100 + gaps, n_gaps=gaps, gap_len=200)
    hp, hc, fp, fc, off = inputs.polarization_batch(seg_in, K, lw, 7200 + lw)
    off[0], off[1], off[2] = -lw, n, -lw // 2          # fully before, fully after, straddling the start
    d = seg_in.d[seg_in.kept]
    o = oracle.OracleSegment(seg_in.acf, seg_in.mask)
    seg = td.Segment(seg_in.acf, seg_in.mask)
    seg.set_data(d)
    hpd, hcd, fpd, fcd, offd = _dev(torch_cuda, hp, hc, fp, fc, off)
    out = _outs(torch_cuda, K)
    seg.project_into(hpd, hcd, fpd, fcd, offd, out["logL"], chi2=out["chi2"], hh=out["hh"], dh=out["dh"],
                     rho_mf=out["rho_mf"], rho_eff2=out["rho_eff2"])
    torch_cuda.cuda.synchronize()
    seg.check()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    R = np.stack([oracle.projected_residual(o, d, hp[k], hc[k], fp[k], fc[k], off[k]) for k in range(K)])
    chi2 = o.chi2(R)
    ll = oracle.loglike_from_chi2(chi2, o.logdet, o.n_kept)
    assert np.max(np.abs(got["chi2"] - chi2) / chi2) <= 1e-7
    assert np.max(np.abs(got["logL"] - ll)) <= 1e-3
    dd = oracle.inner(o, d, d)
    for k in range(0, K, 5):
        h = oracle.project_template(n, hp[k], hc[k], fp[k], fc[k], off[k])[o.kept]
        hh = oracle.inner(o, h, h)
        assert abs(got["hh"][k] - hh) <= 1e-6 * hh + 1e-9, k
        assert abs(got["dh"][k] - oracle.inner(o, d, h)) <= 1e-3, k
        assert abs(got["rho_eff2"][k] - (dd - chi2[k])) <= 1e-3, k
        if hh > 0:
            # rho_mf = <d, h> / sqrt(<h, h>): the 1e-3 bar on <d, h> becomes
            # 1e-3 / sqrt(<h, h>) (templates mostly off the segment have small <h, h>)
            assert abs(got["rho_mf"][k] - oracle.mf_snr(o, d, h)) <= 1e-3 / np.sqrt(hh), k
    # the three placed off the segment subtract nothing: logL of d itself
    ll_d = oracle.loglike_from_chi2(o.chi2(d[None, :]), o.logdet, o.n_kept)[0]
    assert np.all(np.abs(got["logL"][:2] - ll_d) <= 1e-3)
    seg.close()


def test_project_equals_template_path_bitwise(torch_cuda, gpu_lib):
    """The fused templates are fl32(fl32(fp hp) + fl32(fc hc)) placed and
    gathered: td_template_batch on those templates, built here with float32
    numpy, gives the same bits for every output."""
    from paper_2603_06010_b300 import td
    n, K, lw = 1500, 50, 900
    seg_in = inputs.make_segment(n, 2048.0, 7300, n_gaps=1, gap_len=150)
    hp, hc, fp, fc, off = inputs.polarization_batch(seg_in, K, lw, 7301)
    d = seg_in.d[seg_in.kept]
    seg = td.Segment(seg_in.acf, seg_in.mask)
    seg.set_data(d)
    H = np.zeros((K, seg_in.n_kept), np.float32)
    t = seg_in.kept
    for k in range(K):
        u = t - off[k]
        on = (u >= 0) & (u < lw)
        H[k, on] = np.float32(fp[k]) * hp[k, u[on]] + np.float32(fc[k]) * hc[k, u[on]]
    hpd, hcd, fpd, fcd, offd = _dev(torch_cuda, hp, hc, fp, fc, off)
    a, b = _outs(torch_cuda, K), _outs(torch_cuda, K)
    seg.project_into(hpd, hcd, fpd, fcd, offd, a["logL"], chi2=a["chi2"], hh=a["hh"], dh=a["dh"],
                     rho_mf=a["rho_mf"], rho_eff2=a["rho_eff2"])
    seg.template_into(torch_cuda.from_numpy(H).cuda(), b["logL"], chi2=b["chi2"], hh=b["hh"], dh=b["dh"],
                      rho_mf=b["rho_mf"], rho_eff2=b["rho_eff2"])
    torch_cuda.cuda.synchronize()
    seg.check()
    for key in a:
        assert torch_cuda.equal(a[key], b[key]), key
    seg.close()


def test_project_one_polarization_and_empty_waveform(torch_cuda, gpu_lib):
    from paper_2603_06010_b300 import td
    n, K, lw = 1200, 9, 500
    seg_in = inputs.make_segment(n, 2048.0, 7400)
    hp, hc, fp, fc, off = inputs.polarization_batch(seg_in, K, lw, 7401)
    d = seg_in.d
    o = oracle.OracleSegment(seg_in.acf)
    seg = td.Segment(seg_in.acf)
    seg.set_data(d)
    hpd, fpd, offd = _dev(torch_cuda, hp, fp, off)
    ll = torch_cuda.empty(K, dtype=torch_cuda.float64, device="cuda")
    seg.project_into(hpd, None, fpd, None, offd, ll)
    torch_cuda.cuda.synchronize()
    seg.check()
    R = np.stack([oracle.projected_residual(o, d, hp[k], None, fp[k], 0.0, off[k]) for k in range(K)])
    exp = oracle.loglike_from_chi2(o.chi2(R), o.logdet, o.n_kept)
    assert np.max(np.abs(ll.cpu().numpy() - exp)) <= 1e-3
    # lw = 0: every template is zero
    seg.project_into(hpd, None, fpd, None, offd, ll, lw=0)
    torch_cuda.cuda.synchronize()
    seg.check()
    ll_d = oracle.loglike_from_chi2(o.chi2(d[None, :]), o.logdet, o.n_kept)[0]
    assert np.all(np.abs(ll.cpu().numpy() - ll_d) <= 1e-3)
    seg.close()


def test_project_errors_and_empty_batch(torch_cuda, gpu_lib):
    from paper_2603_06010_b300 import td
    n = 600
    seg = td.Segment(inputs.acf_from_psd(n, 2048.0))
    hp = torch_cuda.zeros((4, 100), dtype=torch_cuda.float32, device="cuda")
    fp = torch_cuda.zeros(4, dtype=torch_cuda.float64, device="cuda")
    off = torch_cuda.zeros(4, dtype=torch_cuda.int64, device="cuda")
    ll = torch_cuda.full((4,), 7.0, dtype=torch_cuda.float64, device="cuda")
    out = td.TemplateOut(ll.data_ptr(), None, None, None, None, None)
    L = td.lib()
    # no data vector yet
    assert L.td_project_batch(seg.handle, hp.data_ptr(), None, 100, 100, 4, fp.data_ptr(), None, off.data_ptr(),
                              ctypes.byref(out), None, None) == td.TD_ERR_INVALID
    seg.set_data(np.zeros(n))
    bad = [
        (None, None, 100, 100, 4, fp.data_ptr(), None, off.data_ptr()),          # hp NULL
        (hp.data_ptr(), hp.data_ptr(), 100, 100, 4, fp.data_ptr(), None, off.data_ptr()),   # hc without fc
        (hp.data_ptr(), None, 50, 100, 4, fp.data_ptr(), None, off.data_ptr()),  # ldw < lw
        (hp.data_ptr(), None, 100, -1, 4, fp.data_ptr(), None, off.data_ptr()),  # lw < 0
        (hp.data_ptr(), None, 100, 100, -1, fp.data_ptr(), None, off.data_ptr()),   # K < 0
        (hp.data_ptr(), None, 100, 100, 4, None, None, off.data_ptr()),          # fp NULL
        (hp.data_ptr(), None, 100, 100, 4, fp.data_ptr(), None, None),           # offset NULL
        (hp.data_ptr(), None, 100, 100, 70000, fp.data_ptr(), None, off.data_ptr()),  # K > 65535
    ]
    for a in bad:
        assert L.td_project_batch(seg.handle, *a, ctypes.byref(out), None, None) == td.TD_ERR_INVALID, a
    assert L.td_project_batch(seg.handle, hp.data_ptr(), None, 100, 100, 0, fp.data_ptr(), None, off.data_ptr(),
                              ctypes.byref(out), None, None) == td.TD_OK
    torch_cuda.cuda.synchronize()
    seg.check()
    assert np.all(ll.cpu().numpy() == 7.0)
    seg.close()


def test_project_network_shares_polarizations(torch_cuda, gpu_lib):
    """Three detectors (PSD scales 1.0, 1.3, 2.1, gapped) take the same hp, hc
    arrays with their own antenna factors and offsets; the joint logL is the
    sum (Sec. II.B item 3)."""
    from paper_2603_06010_b300 import td
    n, K, lw = 2048, 24, 1500
    rng = np.random.default_rng(7500)
    base = inputs.make_segment(n, 2048.0, 7501, n_gaps=1, gap_len=128)
    hp, hc, _, _, _ = inputs.polarization_batch(base, K, lw, 7502)
    hpd, hcd = _dev(torch_cuda, hp, hc)
    joint = np.zeros(K)
    exp = np.zeros(K)
    for det, scale in enumerate((1.0, 1.3, 2.1)):
        seg_in = inputs.make_segment(n, 2048.0, 7510 + det, n_gaps=2, gap_len=128, scale=scale)
        fp, fc = rng.uniform(-1, 1, K), rng.uniform(-1, 1, K)
        off = rng.integers(-200, n - lw + 200, K).astype(np.int64)
        d = seg_in.d[seg_in.kept]
        o = oracle.OracleSegment(seg_in.acf, seg_in.mask)
        seg = td.Segment(seg_in.acf, seg_in.mask)
        seg.set_data(d)
        fpd, fcd, offd = _dev(torch_cuda, fp, fc, off)
        ll = torch_cuda.empty(K, dtype=torch_cuda.float64, device="cuda")
        seg.project_into(hpd, hcd, fpd, fcd, offd, ll)
        torch_cuda.cuda.synchronize()
        seg.check()
        joint += ll.cpu().numpy()
        R = np.stack([oracle.projected_residual(o, d, hp[k], hc[k], fp[k], fc[k], off[k]) for k in range(K)])
        exp += oracle.loglike_from_chi2(o.chi2(R), o.logdet, o.n_kept)
        seg.close()
    assert np.max(np.abs(joint - exp)) <= 1e-3
