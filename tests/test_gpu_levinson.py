"""Whitening operator built by the Levinson-Durbin recursion (td_factor_many
with TD_FACTOR_NO_FP64) against the CPU FP64 oracle and closed forms.

For a gap-free segment the rows of L^{-1} are the normalised prediction-error
filters, so this build must give the same logdet and the same logL/chi2 (to
the bar: |dlogL| <= 1e-3, chi2 rel <= 1e-7) as the Cholesky route.
"""
import json
import os
import zlib

import numpy as np
import pytest

import oracle
from paper_2603_06010_b300 import inputs

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CHI_REL, LL_ABS = 1e-7, 1e-3


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _ll(torch, td, seg, R_kn, prec=None, path=None):
    kw = {}
    if prec is not None:
        kw["precision"] = prec
    if path is not None:
        kw["path"] = path
    R = torch.from_numpy(np.ascontiguousarray(R_kn)).cuda()
    ll, chi = seg.loglike(R, td.options(**kw), with_chi2=True)
    torch.cuda.synchronize()
    seg.check()
    return ll.cpu().numpy(), chi.cpu().numpy()


def _cmp(ll, chi, exp_ll, exp_chi, what):
    rel = np.max(np.abs(chi - exp_chi) / np.abs(exp_chi))
    dll = np.max(np.abs(ll - exp_ll))
    assert rel <= CHI_REL, f"{what}: chi2 rel {rel:.3e}"
    assert dll <= LL_ABS, f"{what}: |dlogL| {dll:.3e}"


CASES = [  # (name, n, fs, K)
    ("n1", 1, 1024.0, 2),
    ("n64", 64, 1024.0, 5),
    ("n255_k33", 255, 1024.0, 33),
    ("n1100_k257", 1100, 4096.0, 257),
    ("n4096_k8", 4096, 2048.0, 8),
    ("n3000_k300", 3000, 2048.0, 300),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_levinson_operator_parity(torch_cuda, gpu_lib, case):
    from paper_2603_06010_b300 import td
    name, n, fs, K = case
    acf = inputs.acf_from_psd(n, fs) if n > 1 else np.array([2.5])
    o = oracle.OracleSegment(acf)
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    R = inputs.noise_residuals(n, fs, K, 23) if n > 1 else rng.standard_normal((K, 1)).astype(np.float32)
    R = (R + 0.5 * rng.standard_normal(R.shape)).astype(np.float32)
    exp_chi = o.chi2(R)
    exp_ll = oracle.loglike_from_chi2(exp_chi, o.logdet, o.n_kept)
    seg = td.Segment(acf, factor=False)
    td.factor_many([seg])
    assert abs(seg.logdet - o.logdet) <= 1e-9 * max(1.0, abs(o.logdet))
    for prec in (td.TD_PREC_BF16X6, td.TD_PREC_BF16X10):
        ll, chi = _ll(torch_cuda, td, seg, R, prec)
        _cmp(ll, chi, exp_ll, exp_chi, f"{name} prec {prec}")
    # the FP64 factor is not formed on this route
    with pytest.raises(td.TdError):
        _ll(torch_cuda, td, seg, R, td.TD_PREC_FP64)
    seg.close()


def test_levinson_equals_cholesky_route_all_paths(torch_cuda, gpu_lib):
    """Both operator builds feed the same kernels; every path agrees within the bar."""
    from paper_2603_06010_b300 import td
    n, fs, K = 2000, 2048.0, 17
    acf = inputs.acf_from_psd(n, fs)
    R = inputs.noise_residuals(n, fs, K, 41)
    a = td.Segment(acf)
    b = td.Segment(acf, factor=False)
    td.factor_many([b])
    for path in (td.TD_PATH_TENSOR, td.TD_PATH_STREAM, td.TD_PATH_STREAM64, td.TD_PATH_SMALLK):
        la, ca = _ll(torch_cuda, td, a, R, path=path)
        lb, cb = _ll(torch_cuda, td, b, R, path=path)
        assert np.max(np.abs(ca - cb) / ca) <= CHI_REL, path
        assert np.max(np.abs(la - lb)) <= LL_ABS, path
    a.close()
    b.close()


def test_ar1_closed_form_n32768(torch_cuda, gpu_lib):
    """AR(1) noise at the largest segment length: logdet = N log s2 - log(1 - phi^2)
    and w_0 = r_0 sqrt(1 - phi^2)/sigma, w_t = (r_t - phi r_{t-1})/sigma."""
    from paper_2603_06010_b300 import td
    n, phi, s2, K = 32768, 0.9, 1.3, 24
    acf = inputs.ar1_acf(n, phi, s2)
    R = np.random.default_rng(77).standard_normal((K, n)).astype(np.float32)
    R64 = R.astype(np.float64)
    w = np.empty_like(R64)
    w[:, 0] = R64[:, 0] * np.sqrt(1.0 - phi * phi)
    w[:, 1:] = R64[:, 1:] - phi * R64[:, :-1]
    exp_chi = np.sum(w * w, axis=1) / s2
    exp_ld = n * np.log(s2) - np.log(1.0 - phi * phi)
    exp_ll = -0.5 * exp_chi - 0.5 * exp_ld - 0.5 * n * np.log(2 * np.pi)
    seg = td.Segment(acf, factor=False)
    td.factor_many([seg])
    assert abs(seg.logdet - exp_ld) <= 1e-9 * abs(exp_ld)
    ll, chi = _ll(torch_cuda, td, seg, R)
    _cmp(ll, chi, exp_ll, exp_chi, "AR(1) N=32768")
    seg.close()


def test_mixed_list_gapped_uses_cholesky(torch_cuda, gpu_lib):
    from paper_2603_06010_b300 import td
    n, fs = 1500, 2048.0
    acf = inputs.acf_from_psd(n, fs)
    mask = np.ones(n, np.uint8)
    mask[300:500] = 0
    segs = [td.Segment(acf, factor=False), td.Segment(acf, mask, factor=False)]
    td.factor_many(segs)
    for seg, m in zip(segs, (None, mask)):
        o = oracle.OracleSegment(acf, m)
        R = inputs.noise_residuals(n, fs, 9, 5, mask=m)
        exp_chi = o.chi2(R)
        ll, chi = _ll(torch_cuda, td, seg, R)
        _cmp(ll, chi, oracle.loglike_from_chi2(exp_chi, o.logdet, o.n_kept), exp_chi, "mixed")
        assert abs(seg.logdet - o.logdet) <= 1e-9 * abs(o.logdet)
        seg.close()


def test_levinson_not_positive_definite_pivot(torch_cuda, gpu_lib):
    """Tridiagonal Toeplitz (1, 0.8): its leading minors change sign at a pivot the
    oracle's dpotrf finds; the recursion must stop at the same kept sample."""
    from paper_2603_06010_b300 import td
    n = 40
    acf = np.zeros(n)
    acf[0], acf[1] = 1.0, 0.8
    with pytest.raises(oracle.NotPositiveDefinite) as ei:
        oracle.OracleSegment(acf)
    seg = td.Segment(acf, factor=False)
    with pytest.raises(td.TdError) as e2:
        td.factor_many([seg])
    assert e2.value.code == td.TD_ERR_NOT_PD
    assert seg.last_pivot == ei.value.pivot
    seg.close()


def _golden():
    with open(os.path.join(HERE, "golden", "full_size.json")) as f:
        return json.load(f)


def test_full_gapfree_n8192_via_levinson(torch_cuda, gpu_lib):
    """The gap-free N=8192, K=4096 batch with the operator built in O(N^2)."""
    from paper_2603_06010_b300 import td
    g = _golden()["gapfree_n8192_k4096"]
    seg_in = inputs.make_segment(g["n"], g["fs"], g["seed"], n_gaps=g["n_gaps"], gap_len=g["gap_len"],
                                 scale=g["scale"])
    R = inputs.residual_batch(seg_in, g["K"], g["rseed"])
    seg = td.Segment(seg_in.acf, factor=False)
    td.factor_many([seg])
    assert abs(seg.logdet - g["logdet"]) <= 1e-9 * abs(g["logdet"])
    ll, chi = _ll(torch_cuda, td, seg, R)
    cols = g["columns"]
    _cmp(ll[cols], chi[cols], np.array(g["logL"]), np.array(g["chi2"]), "gap-free N=8192 Levinson")
    seg.close()


def test_full_mix64_longest_segment(torch_cuda, gpu_lib):
    """The longest segment of the 64-segment mix (N=32257) against stored oracle values."""
    from paper_2603_06010_b300 import td
    g = _golden().get("mix64_longest")
    if g is None:
        pytest.skip("no stored values")
    acf = inputs.acf_from_psd(g["n"], g["fs"], a=g["a"], floor=g["floor"])
    R = inputs.noise_residuals(g["n"], g["fs"], g["K"], g["rseed"], a=g["a"], floor=g["floor"])
    cols = g["columns"]
    chk = [float(np.sum(R[c].astype(np.float64))) for c in cols]
    assert np.allclose(chk, g["r_checksum"], rtol=1e-6, atol=1e-3), "input generator drifted"
    seg = td.Segment(acf, factor=False)
    td.factor_many([seg])
    assert abs(seg.logdet - g["logdet"]) <= 1e-9 * abs(g["logdet"])
    ll, chi = _ll(torch_cuda, td, seg, R)
    _cmp(ll[cols], chi[cols], np.array(g["logL"]), np.array(g["chi2"]), "mix64 longest")
    seg.close()


def test_factor_many_mixed_batch_with_a_bad_segment(torch_cuda, gpu_lib):
    """One non positive definite ACF among good ones: the good ones are factored
    and evaluate correctly, the call reports TD_ERR_NOT_PD with the bad pivot."""
    from paper_2603_06010_b300 import td
    good = [inputs.acf_from_psd(n, 2048.0) for n in (300, 777)]
    bad = np.zeros(50)
    bad[0], bad[1] = 1.0, 0.8
    segs = [td.Segment(good[0], factor=False), td.Segment(bad, factor=False), td.Segment(good[1], factor=False)]
    with pytest.raises(td.TdError) as e:
        td.factor_many(segs)
    assert e.value.code == td.TD_ERR_NOT_PD
    assert segs[1].last_pivot == 2
    for seg, acf in ((segs[0], good[0]), (segs[2], good[1])):
        o = oracle.OracleSegment(acf)
        R = inputs.noise_residuals(acf.shape[0], 2048.0, 7, 3)
        exp_chi = o.chi2(R)
        ll, chi = _ll(torch_cuda, td, seg, R)
        _cmp(ll, chi, oracle.loglike_from_chi2(exp_chi, o.logdet, o.n_kept), exp_chi, "good segment")
    for s in segs:
        s.close()


def test_grouped_launch_over_levinson_segments(torch_cuda, gpu_lib):
    """The grouped launch on operators built by the recursion (the 64-segment
    mix's route), segments of uneven N and K, against the oracle."""
    from paper_2603_06010_b300 import td
    specs = [(520, 17), (1900, 140), (3000, 64), (700, 300)]
    segs, Rs, outs, exp = [], [], [], []
    for i, (n, K) in enumerate(specs):
        acf = inputs.acf_from_psd(n, 4096.0, a=-4.2 + 0.1 * i, floor=1.5 + 0.3 * i)
        R = inputs.noise_residuals(n, 4096.0, K, 40 + i, a=-4.2 + 0.1 * i, floor=1.5 + 0.3 * i)
        o = oracle.OracleSegment(acf)
        chi = o.chi2(R)
        exp.append((oracle.loglike_from_chi2(chi, o.logdet, o.n_kept), chi))
        segs.append(td.Segment(acf, factor=False))
        Rs.append(torch_cuda.from_numpy(R).cuda())
        outs.append(torch_cuda.empty(K, dtype=torch_cuda.float64, device="cuda"))
    td.factor_many(segs)
    g = td.Group(segs, Rs, outs)
    g.graph_launch()
    torch_cuda.cuda.synchronize()
    g.check()
    for out, (el, ec) in zip(outs, exp):
        assert np.max(np.abs(out.cpu().numpy() - el)) <= LL_ABS
    g.close()
    for s in segs:
        s.close()


def test_auto_precision_switches_above_32768(torch_cuda, gpu_lib):
    """TD_PREC_AUTO (the default): six products for 2048 <= N' <= 32768, ten
    beyond and below (same bits as the explicit choice)."""
    from paper_2603_06010_b300 import td
    assert td.options().precision == td.TD_PREC_AUTO
    for n, expect in ((300, td.TD_PREC_BF16X10), (2047, td.TD_PREC_BF16X10), (2048, td.TD_PREC_BF16X6),
                      (33000, td.TD_PREC_BF16X10)):
        acf = inputs.acf_from_psd(n, 4096.0)
        seg = td.Segment(acf, factor=False)
        td.factor_many([seg])
        R = np.random.default_rng(n).standard_normal((8, n)).astype(np.float32) * np.float32(np.sqrt(acf[0]))
        la, ca = _ll(torch_cuda, td, seg, R, td.TD_PREC_AUTO)
        le, ce = _ll(torch_cuda, td, seg, R, expect)
        assert np.array_equal(la, le) and np.array_equal(ca, ce), n
        seg.close()
