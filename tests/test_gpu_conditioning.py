"""The tensor-core paths where dynamic range is most likely to hurt them.

* Gapped AR(1) noise with phi = 0.99 and 0.999 (condition numbers of about
  4e4 and 4e6): whitened values are differences of nearly equal neighbours
  (r_t - phi^dt r_{t-1}), so the split products lose the cancellation ratio.
  Expected chi2 and log det come from the AR(1) closed form (the Markov
  whitening of any kept subsequence), not from the oracle.
* Strain-scale units (the ACF times 1e-42, residuals times 1e-21, as for
  detector strain): chi2 must not change and log det shifts by N' log 1e-42,
  on every path (dense tile shapes, FP64, refinement, Gohberg-Semencul,
  the recursion-built operator, grouped launches, the template form).
The bar is the one every parity test holds: chi2 relative <= 1e-7 and
|dlogL| <= 1e-3.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_06010_b300 import inputs
from tests.pins import ar1_whiten_closed_form

pytestmark = pytest.mark.gpu

CHI2_REL, DLOGL_ABS = 1e-7, 1e-3
LOG2PI = math.log(2 * math.pi)
S_ACF, S_R = 1e-42, 1e-21


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _run(torch, seg, R, opt):
    Rt = torch.from_numpy(np.ascontiguousarray(R)).cuda()
    ll, chi = seg.loglike(Rt, opt, with_chi2=True)
    torch.cuda.synchronize()
    seg.check()
    return ll.cpu().numpy(), chi.cpu().numpy()


def _bar(ll, chi, exp_ll, exp_chi, what):
    assert np.all(np.isfinite(ll)), what
    rel = float(np.max(np.abs(chi - exp_chi) / exp_chi))
    dll = float(np.max(np.abs(ll - exp_ll)))
    assert rel <= CHI2_REL and dll <= DLOGL_ABS, f"{what}: chi2 rel {rel:.3e}, |dlogL| {dll:.3e}"


def _paths(td, K):
    out = [("auto", td.TD_PATH_AUTO), ("tensor256", td.TD_PATH_TENSOR), ("tensor128", td.TD_PATH_TENSOR128),
           ("stream128", td.TD_PATH_STREAM128), ("stream64", td.TD_PATH_STREAM64)]
    if K <= 256:
        out.append(("smallk", td.TD_PATH_SMALLK))
    return out


AR_N = 3000
AR_MASK_SPANS = ((500, 1012), (1800, 1900), (2990, 3000))


@pytest.mark.parametrize("phi", [0.99, 0.999])
def test_ar1_ill_conditioned_gapped_dense_paths(torch_cuda, gpu_lib, phi):
    from paper_2603_06010_b300 import td
    mask = np.ones(AR_N, np.uint8)
    for a, b in AR_MASK_SPANS:
        mask[a:b] = 0
    t = np.flatnonzero(mask)
    seg = td.Segment(inputs.ar1_acf(AR_N, phi, 1.0), mask)
    for K in (8, 200, 300):
        R = inputs.ar1_noise(AR_N, phi, 1.0, K, 700 + K, mask)
        exp_chi, ld = np.empty(K), 0.0
        for k in range(K):
            w, ld = ar1_whiten_closed_form(R[k].astype(np.float64), t, phi, 1.0)
            exp_chi[k] = float(np.sum(w * w))
        exp_ll = -0.5 * exp_chi - 0.5 * ld - 0.5 * len(t) * LOG2PI
        # the factor's split products carry about 2^-46 of sum |a||b|; the Schur
        # complements here are ~1/(1 - phi^2) smaller than the terms they come from,
        # so log det keeps ~1e-9 relative at phi = 0.999 (the logL bar needs 2e-3 absolute)
        assert abs(seg.logdet - ld) <= 1e-7 * abs(ld)
        for pname, prec in (("auto", td.TD_PREC_AUTO), ("bf16x6", td.TD_PREC_BF16X6),
                            ("bf16x10", td.TD_PREC_BF16X10)):
            for path_name, path in _paths(td, K):
                ll, chi = _run(torch_cuda, seg, R, td.options(precision=prec, path=path))
                _bar(ll, chi, exp_ll, exp_chi, f"AR(1) phi={phi} K={K} {pname} {path_name}")
    seg.close()


def _strain_case(n, fs, gapped, K, seed):
    mask = None
    if gapped:
        mask = np.ones(n, np.uint8)
        mask[300:812] = 0
        mask[1500:1600] = 0
    acf = inputs.acf_from_psd(n, fs)
    o = oracle.OracleSegment(acf, mask)
    R = inputs.noise_residuals(n, fs, K, seed, mask=mask)
    Rs = (R.astype(np.float64) * S_R).astype(np.float32)
    # r_s^T (s C)^{-1} r_s with s = S_R^2 is the chi2 of r_s / S_R under C
    exp_chi = o.chi2(Rs.astype(np.float64) / S_R)
    exp_ll = -0.5 * exp_chi - 0.5 * (o.logdet + o.n_kept * math.log(S_ACF)) - 0.5 * o.n_kept * LOG2PI
    return acf * S_ACF, mask, Rs, exp_ll, exp_chi


@pytest.mark.parametrize("gapped", [False, True])
def test_strain_scale_every_dense_path(torch_cuda, gpu_lib, gapped):
    from paper_2603_06010_b300 import td
    n, fs = 2048, 2048.0
    for K in (8, 300):
        acf_s, mask, Rs, exp_ll, exp_chi = _strain_case(n, fs, gapped, K, 800 + K)
        seg = td.Segment(acf_s, mask)
        for pname, prec in (("auto", td.TD_PREC_AUTO), ("bf16x10", td.TD_PREC_BF16X10), ("fp64", td.TD_PREC_FP64)):
            paths = _paths(td, K) if pname != "fp64" else [("fp64", td.TD_PATH_AUTO)]
            for path_name, path in paths:
                ll, chi = _run(torch_cuda, seg, Rs, td.options(precision=prec, path=path))
                _bar(ll, chi, exp_ll, exp_chi, f"strain gapped={gapped} K={K} {pname} {path_name}")
        ll, chi = _run(torch_cuda, seg, Rs, td.options(precision=td.TD_PREC_BF16X3, refine=1))
        _bar(ll, chi, exp_ll, exp_chi, f"strain gapped={gapped} K={K} BF16X3 + refinement")
        seg.close()


def test_strain_scale_gsce_and_recursion_operator(torch_cuda, gpu_lib):
    from paper_2603_06010_b300 import td
    n, fs = 2048, 2048.0
    for K in (5, 300):
        acf_s, _, Rs, exp_ll, exp_chi = _strain_case(n, fs, False, K, 900 + K)
        g = td.Segment(acf_s, factor=False)
        g.gs_prepare()
        ll, chi = _run(torch_cuda, g, Rs, td.options(path=td.TD_PATH_GSCE))
        _bar(ll, chi, exp_ll, exp_chi, f"strain GSCE K={K}")
        g.close()
        lv = td.Segment(acf_s, factor=False)
        td.factor_many([lv])
        ll, chi = _run(torch_cuda, lv, Rs, td.options())
        _bar(ll, chi, exp_ll, exp_chi, f"strain recursion operator K={K}")
        lv.close()


def test_strain_scale_grouped_and_template_form(torch_cuda, gpu_lib):
    torch = torch_cuda
    from paper_2603_06010_b300 import td
    n, fs = 2048, 2048.0
    cases = [_strain_case(n, fs, gapped, K, 950 + K) for gapped, K in ((False, 40), (True, 200))]
    segs = [td.Segment(acf_s, mask) for acf_s, mask, _, _, _ in cases]
    Rs = [torch.from_numpy(c[2]).cuda() for c in cases]
    outs = [torch.empty(r.shape[0], dtype=torch.float64, device="cuda") for r in Rs]
    g = td.Group(segs, Rs, outs)
    g.launch()
    torch.cuda.synchronize()
    g.check()
    for (_, _, _, exp_ll, _), o in zip(cases, outs):
        dll = float(np.max(np.abs(o.cpu().numpy() - exp_ll)))
        assert dll <= DLOGL_ABS, f"strain grouped: |dlogL| {dll:.3e}"
    g.close()
    # template form: r_k = d - h_k with d and h at strain scale
    acf_s, mask, Rs0, _, _ = cases[1]
    seg = segs[1]
    kept = np.flatnonzero(mask)
    o = oracle.OracleSegment(acf_s / S_ACF, mask)
    rng = np.random.default_rng(97)
    d = rng.standard_normal(len(kept)) * math.sqrt(acf_s[0])
    H = (rng.standard_normal((6, len(kept))) * math.sqrt(acf_s[0]) * 0.1).astype(np.float32)
    seg.set_data(d)
    ll = torch.empty(6, dtype=torch.float64, device="cuda")
    seg.template_into(torch.from_numpy(H).cuda(), ll)
    torch.cuda.synchronize()
    seg.check()
    Rt = (d[None, :] - H.astype(np.float64)).astype(np.float32).astype(np.float64)
    exp_chi = o.chi2(Rt / S_R)
    exp_ll = -0.5 * exp_chi - 0.5 * (o.logdet + o.n_kept * math.log(S_ACF)) - 0.5 * o.n_kept * LOG2PI
    dll = float(np.max(np.abs(ll.cpu().numpy() - exp_ll)))
    assert dll <= DLOGL_ABS, f"strain template form: |dlogL| {dll:.3e}"
    for s in segs:
        s.close()
