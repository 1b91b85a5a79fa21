"""The Gohberg-Semencul path (TD_PATH_GSCE) against the CPU FP64 oracle.

chi2 = (|L_x^T r|^2 - |R_x r|^2) / x_0 with x = C^{-1} e_1 reaches r^T C^{-1} r
exactly in exact arithmetic, so the oracle is the dense definition.  Held
to the method's bar (chi2 1e-7 relative, |delta logL| 1e-3): with the
sheared twiddles the FP32 FFTs leave ~1.5e-8 rms relative at N = 1024 and
less above, the path's range being 1024 <= N <= 32768.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2603_06010_b300 import inputs

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GS_CHI2_REL = 1e-7
GS_DLOGL = 1e-3


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _gs(td, acf):
    seg = td.Segment(acf, factor=False)
    seg.gs_prepare()
    return seg


def _run(torch, td, seg, R_kn):
    R = torch.from_numpy(np.ascontiguousarray(R_kn)).cuda()
    logL, chi2 = seg.loglike(R, td.options(path=td.TD_PATH_GSCE), with_chi2=True)
    torch.cuda.synchronize()
    seg.check()
    return logL.cpu().numpy(), chi2.cpu().numpy()


# (n, fs, K): circulant lengths 2048 .. 16384, i.e. local lengths 256 .. 2048
# per CTA (register passes 3+3+2, 3+3+3, 3x3+1, 3x3+2), odd K (an unpaired
# last column), N not a power of two
CASES = [(1024, 1024.0, 3), (1100, 4096.0, 257), (2048, 2048.0, 64), (3000, 2048.0, 130),
         (4097, 2048.0, 33), (8192, 2048.0, 17)]


@pytest.mark.parametrize("n,fs,K", CASES, ids=[f"n{c[0]}_k{c[2]}" for c in CASES])
def test_gsce_parity(torch_cuda, gpu_lib, n, fs, K):
    from paper_2603_06010_b300 import td
    acf = inputs.acf_from_psd(n, fs)
    o = oracle.OracleSegment(acf)
    R = inputs.noise_residuals(n, fs, K, 101 + n)
    exp_chi = o.chi2(R)
    exp_ll = oracle.loglike_from_chi2(exp_chi, o.logdet, o.n_kept)
    seg = _gs(td, acf)
    assert abs(seg.logdet - o.logdet) <= 1e-9 * max(1.0, abs(o.logdet))
    ll, chi = _run(torch_cuda, td, seg, R)
    rel = np.max(np.abs(chi - exp_chi) / exp_chi)
    assert rel <= GS_CHI2_REL, f"n={n} K={K}: chi2 rel {rel:.3e}"
    assert np.max(np.abs(ll - exp_ll)) <= GS_DLOGL


def test_gsce_many_pairs_ragged(torch_cuda, gpu_lib):
    """Enough column pairs that each CTA carries two signals, with an odd K
    (the last pair's second column missing) and an odd number of pairs."""
    from paper_2603_06010_b300 import td
    n, fs, K = 2048, 2048.0, 1001
    acf = inputs.acf_from_psd(n, fs)
    o = oracle.OracleSegment(acf)
    R = inputs.noise_residuals(n, fs, K, 4242)
    exp_chi = o.chi2(R)
    ll, chi = _run(torch_cuda, td, _gs(td, acf), R)
    assert np.max(np.abs(chi - exp_chi) / exp_chi) <= GS_CHI2_REL
    assert np.max(np.abs(ll - oracle.loglike_from_chi2(exp_chi, o.logdet, o.n_kept))) <= GS_DLOGL


def test_gsce_white_noise_closed_form(torch_cuda, gpu_lib):
    """C = s2 I: x = e_1 / s2, R_x = 0, chi2 = |r|^2 / s2."""
    from paper_2603_06010_b300 import td
    n, s2 = 3000, 1.7
    R = np.random.default_rng(8).standard_normal((11, n)).astype(np.float32)
    R64 = R.astype(np.float64)
    exp_ll = -np.sum(R64 * R64, 1) / (2 * s2) - 0.5 * n * np.log(2 * np.pi * s2)
    ll, _ = _run(torch_cuda, td, _gs(td, inputs.white_acf(n, s2)), R)
    assert np.max(np.abs(ll - exp_ll)) < 1e-4


def test_gsce_ar1_closed_form(torch_cuda, gpu_lib):
    """AR(1): chi2 = (1 - phi^2) r_0^2 / s2 + sum_t (r_t - phi r_{t-1})^2 / s2 and
    log det = n log s2 - log(1 - phi^2)."""
    from paper_2603_06010_b300 import td
    n, phi, s2 = 2500, 0.8, 1.3
    acf = s2 * phi ** np.arange(n) / (1 - phi * phi)
    R = np.random.default_rng(9).standard_normal((6, n)).astype(np.float32)
    R64 = R.astype(np.float64)
    w = np.empty_like(R64)
    w[:, 0] = R64[:, 0] * np.sqrt(1 - phi * phi)
    w[:, 1:] = R64[:, 1:] - phi * R64[:, :-1]
    exp_chi = np.sum(w * w, 1) / s2
    seg = _gs(td, acf)
    assert abs(seg.logdet - (n * np.log(s2) - np.log(1 - phi * phi))) < 1e-8 * n
    _, chi = _run(torch_cuda, td, seg, R)
    assert np.max(np.abs(chi - exp_chi) / exp_chi) <= GS_CHI2_REL


def test_gsce_full_gapfree_n8192_k4096(torch_cuda, gpu_lib):
    """The benchmark batch (gap-free N=8192, K=4096) through GSCE, against the
    stored oracle columns."""
    from paper_2603_06010_b300 import td
    with open(os.path.join(HERE, "golden", "full_size.json")) as f:
        g = json.load(f)["gapfree_n8192_k4096"]
    seg_in = inputs.make_segment(g["n"], g["fs"], g["seed"], n_gaps=g["n_gaps"], gap_len=g["gap_len"],
                                 scale=g["scale"])
    R = inputs.residual_batch(seg_in, g["K"], g["rseed"])
    seg = _gs(td, seg_in.acf)
    assert abs(seg.logdet - g["logdet"]) <= 1e-9 * abs(g["logdet"])
    ll, chi = _run(torch_cuda, td, seg, R)
    cols = g["columns"]
    rel = np.max(np.abs(chi[cols] - np.array(g["chi2"])) / np.array(g["chi2"]))
    assert rel <= GS_CHI2_REL, rel
    assert np.max(np.abs(ll[cols] - np.array(g["logL"]))) <= GS_DLOGL


@pytest.mark.parametrize("n", [16384, 32768])
def test_gsce_long_ar1(torch_cuda, gpu_lib, n):
    """Circulant lengths 32768 and 65536 (4096 and 8192 values per CTA) on the
    AR(1) closed form."""
    from paper_2603_06010_b300 import td
    phi, s2 = 0.9, 0.7
    acf = s2 * phi ** np.arange(n) / (1 - phi * phi)
    R = np.random.default_rng(n).standard_normal((5, n)).astype(np.float32)
    R64 = R.astype(np.float64)
    w = np.empty_like(R64)
    w[:, 0] = R64[:, 0] * np.sqrt(1 - phi * phi)
    w[:, 1:] = R64[:, 1:] - phi * R64[:, :-1]
    exp_chi = np.sum(w * w, 1) / s2
    seg = _gs(td, acf)
    assert abs(seg.logdet - (n * np.log(s2) - np.log(1 - phi * phi))) < 1e-8 * n
    _, chi = _run(torch_cuda, td, seg, R)
    assert np.max(np.abs(chi - exp_chi) / exp_chi) <= GS_CHI2_REL


def test_gsce_ill_conditioned_ar1(torch_cuda, gpu_lib):
    """AR(1) with phi = 0.99 (condition number ~4e4), residuals drawn from the
    process itself: still within the bar (CPU emulation of the FP32 network:
    5.8e-8 at this phi, 8.6e-8 at phi = 0.999)."""
    from scipy.signal import lfilter
    from paper_2603_06010_b300 import td
    n, phi, s2 = 8192, 0.99, 1.0
    acf = s2 * phi ** np.arange(n) / (1 - phi * phi)
    rng = np.random.default_rng(99)
    z = rng.standard_normal((6, n))
    z[:, 0] /= np.sqrt(1 - phi * phi)
    R = lfilter([1.0], [1.0, -phi], z, axis=1).astype(np.float32)
    R64 = R.astype(np.float64)
    w = np.empty_like(R64)
    w[:, 0] = R64[:, 0] * np.sqrt(1 - phi * phi)
    w[:, 1:] = R64[:, 1:] - phi * R64[:, :-1]
    exp_chi = np.sum(w * w, 1) / s2
    _, chi = _run(torch_cuda, td, _gs(td, acf), R)
    assert np.max(np.abs(chi - exp_chi) / exp_chi) <= GS_CHI2_REL


def test_gsce_mix64_longest(torch_cuda, gpu_lib):
    """The longest gap-free segment of the 64-segment mix (N=32257) against
    stored oracle values."""
    from paper_2603_06010_b300 import td
    with open(os.path.join(HERE, "golden", "full_size.json")) as f:
        g = json.load(f)["mix64_longest"]
    acf = inputs.acf_from_psd(g["n"], g["fs"], a=g["a"], floor=g["floor"])
    R = inputs.noise_residuals(g["n"], g["fs"], g["K"], g["rseed"], a=g["a"], floor=g["floor"])
    seg = _gs(td, acf)
    assert abs(seg.logdet - g["logdet"]) <= 1e-9 * abs(g["logdet"])
    ll, chi = _run(torch_cuda, td, seg, R)
    cols = g["columns"]
    rel = np.max(np.abs(chi[cols] - np.array(g["chi2"])) / np.array(g["chi2"]))
    assert rel <= GS_CHI2_REL, rel
    assert np.max(np.abs(ll[cols] - np.array(g["logL"]))) <= GS_DLOGL


def test_gsce_alone_vs_in_batch(torch_cuda, gpu_lib):
    """A column's partner changes only its rounding."""
    from paper_2603_06010_b300 import td
    n = 4000
    seg = _gs(td, inputs.acf_from_psd(n, 2048.0))
    R = inputs.noise_residuals(n, 2048.0, 40, 77)
    full, _ = _run(torch_cuda, td, seg, R)
    for k in (0, 1, 17, 39):
        one, _ = _run(torch_cuda, td, seg, R[k:k + 1])
        assert abs(one[0] - full[k]) <= 1e-5 * abs(full[k]), k


def test_gsce_same_as_dense_paths(torch_cuda, gpu_lib):
    """A segment with both forms: GSCE and the ten-product dense path agree."""
    from paper_2603_06010_b300 import td
    n = 3000
    acf = inputs.acf_from_psd(n, 2048.0)
    seg = td.Segment(acf)
    seg.gs_prepare()
    assert abs(seg.logdet - oracle.OracleSegment(acf).logdet) <= 1e-9 * abs(seg.logdet)
    R = inputs.noise_residuals(n, 2048.0, 70, 5)
    Rd = torch_cuda.from_numpy(R).cuda()
    a = seg.loglike(Rd, td.options(path=td.TD_PATH_GSCE)).cpu().numpy()
    b = seg.loglike(Rd, td.options(precision=td.TD_PREC_BF16X10, path=td.TD_PATH_TENSOR128)).cpu().numpy()
    assert np.max(np.abs(a - b)) <= 1e-3


def test_gsce_auto_policy(torch_cuda, gpu_lib):
    """TD_PATH_AUTO on a prepared gap-free segment: GSCE for small batches, the
    dense product for large ones below N = 24576, GSCE when only prepared."""
    from paper_2603_06010_b300 import td
    n = 3000
    acf = inputs.acf_from_psd(n, 2048.0)
    both = td.Segment(acf)
    both.gs_prepare()
    dense = td.Segment(acf)
    only = td.Segment(acf, factor=False)
    only.gs_prepare()
    R = torch_cuda.from_numpy(inputs.noise_residuals(n, 2048.0, 300, 6)).cuda()

    def ll(seg, Rs, opt):
        out = seg.loglike(Rs.contiguous(), opt).cpu().numpy()
        seg.check()
        return out

    gs = td.options(path=td.TD_PATH_GSCE)
    small = R[:8]
    assert np.array_equal(ll(both, small, td.options()), ll(both, small, gs))
    assert np.array_equal(ll(only, small, td.options()), ll(only, small, gs))
    assert np.array_equal(ll(both, R, td.options()), ll(dense, R, td.options()))   # K = 300 > 256
    assert np.array_equal(ll(only, R, td.options()), ll(only, R, gs))
    # refinement is not a GSCE option: AUTO keeps the dense path for it
    ref = td.options(precision=td.TD_PREC_BF16X3, refine=1)
    assert np.array_equal(ll(both, small, ref), ll(dense, small, ref))


def test_gsce_errors(torch_cuda, gpu_lib):
    from paper_2603_06010_b300 import td
    n = 1500
    acf = inputs.acf_from_psd(n, 2048.0)
    mask = np.ones(n, np.uint8)
    mask[100:150] = 0
    gapped = td.Segment(acf, mask, factor=False)
    with pytest.raises(td.TdError) as e:
        gapped.gs_prepare()
    assert e.value.code == td.TD_ERR_UNSUPPORTED
    for m in (32769, 1023):
        other = td.Segment(inputs.acf_from_psd(m, 2048.0), factor=False)
        with pytest.raises(td.TdError) as e:
            other.gs_prepare()
        assert e.value.code == td.TD_ERR_UNSUPPORTED, m
    seg = td.Segment(acf, factor=False)
    R = torch_cuda.from_numpy(inputs.noise_residuals(n, 2048.0, 3, 1)).cuda()
    with pytest.raises(td.TdError) as e:
        seg.loglike(R, td.options(path=td.TD_PATH_GSCE))
    assert e.value.code == td.TD_ERR_NOT_FACTORED
    seg.gs_prepare()
    with pytest.raises(td.TdError) as e:
        seg.loglike(R, td.options(path=td.TD_PATH_GSCE, refine=1))
    assert e.value.code == td.TD_ERR_INVALID
    bad = np.zeros(1024)
    bad[0], bad[1] = 1.0, 2.0
    nd = td.Segment(bad, factor=False)
    with pytest.raises(td.TdError) as e:
        nd.gs_prepare()
    assert e.value.code == td.TD_ERR_NOT_PD
    assert nd.last_pivot == 1


def test_gsce_and_refine_strided_and_host_buffers(torch_cuda, gpu_lib):
    """ldr > N' (residuals inside a wider buffer) and the host-buffer entry point
    (600 columns: two chunks) for GSCE and for the refinement step: the same
    values as a packed device batch, within the bar of the oracle."""
    from paper_2603_06010_b300 import td
    n, K, pad = 2500, 600, 37
    acf = inputs.acf_from_psd(n, 2048.0)
    o = oracle.OracleSegment(acf)
    R = inputs.noise_residuals(n, 2048.0, K, 31337)
    exp = oracle.loglike_from_chi2(o.chi2(R), o.logdet, o.n_kept)
    wide = np.zeros((K, n + pad), np.float32)
    wide[:, :n] = R
    seg = td.Segment(acf)
    seg.gs_prepare()
    for opt in (td.options(path=td.TD_PATH_GSCE), td.options(precision=td.TD_PREC_BF16X3, refine=1)):
        packed = seg.loglike(torch_cuda.from_numpy(R).cuda(), opt).cpu().numpy()
        Wd = torch_cuda.from_numpy(wide).cuda()
        out = torch_cuda.empty(K, dtype=torch_cuda.float64, device="cuda")
        seg.loglike_into(Wd, out, opt, ldr=n + pad)
        torch_cuda.cuda.synchronize()
        seg.check()
        strided = out.cpu().numpy()
        host = np.empty(K)
        seg.loglike_host_into(torch_cuda.from_numpy(wide).pin_memory(), host, opt)
        assert np.max(np.abs(packed - exp)) <= GS_DLOGL
        assert np.max(np.abs(strided - packed)) <= 1e-6 * np.max(np.abs(packed))
        assert np.max(np.abs(host - packed)) <= 1e-6 * np.max(np.abs(packed))
