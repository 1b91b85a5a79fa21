"""CUDA path (through the C ABI) against the CPU FP64 oracle.

Tolerances (the bar stated for the method): |delta logL| <= 1e-3 absolute and
chi2 relative error <= 1e-7 for the split-product tensor-core path; the
plain FP64 path is held to 1e-11 relative.  The 3xBF16 (two-slice) option
is checked against the error band its arithmetic gives (~1e-5 relative),
which is above the bar by design.
"""
import ctypes
import json
import os
import zlib

import numpy as np
import pytest

import oracle
from paper_2603_06010_b300 import inputs

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = {  # precision -> (chi2 rel, |dlogL| abs)
    "fp64": (1e-11, 1e-7),
    "bf16x6": (1e-7, 1e-3),
    "bf16x10": (1e-7, 1e-3),
    "bf16x3": (3e-4, 5.0),
}


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _opt(td, prec):
    p = {"fp64": td.TD_PREC_FP64, "bf16x6": td.TD_PREC_BF16X6, "bf16x10": td.TD_PREC_BF16X10,
         "bf16x3": td.TD_PREC_BF16X3}[prec]
    return td.options(precision=p)


def _run(torch, td, seg, R_kn, prec):
    R = torch.from_numpy(np.ascontiguousarray(R_kn)).cuda()
    logL, chi2 = seg.loglike(R, _opt(td, prec), with_chi2=True)
    torch.cuda.synchronize()
    seg.check()
    return logL.cpu().numpy(), chi2.cpu().numpy()


def _compare(prec, got_ll, got_chi, exp_ll, exp_chi, what=""):
    rel_tol, abs_tol = TOL[prec]
    rel = np.abs(got_chi - exp_chi) / np.abs(exp_chi)
    dll = np.abs(got_ll - exp_ll)
    assert np.all(np.isfinite(got_ll)), what
    assert rel.max() <= rel_tol, f"{what} {prec}: chi2 rel {rel.max():.3e} > {rel_tol}"
    assert dll.max() <= abs_tol, f"{what} {prec}: |dlogL| {dll.max():.3e} > {abs_tol}"
    return rel.max(), dll.max()


def _mask(n, spans):
    m = np.ones(n, np.uint8)
    for a, b in spans:
        m[a:b] = 0
    return m


# (name, n, fs, mask spans, K) -- sizes span several 64/256-row tiles, ragged
# tails, ragged column tiles, gaps at the start/end/adjacent, a single kept
# sample and the one-sample segment.
CASES = [
    ("n1", 1, 1024.0, None, 3),
    ("n64_k1", 64, 1024.0, None, 1),
    ("n255_k3", 255, 1024.0, None, 3),
    ("n257_gaps_k129", 257, 1024.0, [(10, 30), (100, 120)], 129),
    ("n600_edges_adjacent_k127", 600, 2048.0, [(0, 7), (200, 260), (261, 300), (590, 600)], 127),
    ("one_kept_k5", 700, 2048.0, [(0, 350), (351, 700)], 5),
    ("n2048_gaps_k300", 2048, 2048.0, [(500, 1012), (1500, 1600)], 300),
    ("n1100_k257", 1100, 4096.0, None, 257),
]


@pytest.mark.parametrize("prec", ["fp64", "bf16x6", "bf16x10", "bf16x3"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_parity_small(torch_cuda, gpu_lib, case, prec):
    from paper_2603_06010_b300 import td
    name, n, fs, spans, K = case
    mask = None if spans is None else _mask(n, spans)
    acf = inputs.acf_from_psd(n, fs) if n > 1 else np.array([2.5])
    seg_o = oracle.OracleSegment(acf, mask)
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    R = inputs.noise_residuals(n, fs, K, 17, mask=mask) if n > 1 else \
        rng.standard_normal((K, 1)).astype(np.float32)
    R = (R + 0.5 * rng.standard_normal(R.shape)).astype(np.float32)
    exp_chi = seg_o.chi2(R)
    exp_ll = oracle.loglike_from_chi2(exp_chi, seg_o.logdet, seg_o.n_kept)
    seg = td.Segment(acf, mask)
    assert seg.n_kept == seg_o.n_kept
    assert abs(seg.logdet - seg_o.logdet) <= 1e-10 * max(1.0, abs(seg_o.logdet))
    got_ll, got_chi = _run(torch_cuda, td, seg, R, prec)
    _compare(prec, got_ll, got_chi, exp_ll, exp_chi, name)


def test_white_noise_closed_form(torch_cuda, gpu_lib):
    """C = s2 I with gaps: logL = -|r|^2/(2 s2) - (N'/2) log(2 pi s2) exactly."""
    from paper_2603_06010_b300 import td
    n, s2 = 777, 3.5
    mask = _mask(n, [(5, 9), (300, 420)])
    nk = int(mask.sum())
    R = np.random.default_rng(5).standard_normal((40, nk)).astype(np.float32)
    R64 = R.astype(np.float64)
    exp_ll = -np.sum(R64 * R64, 1) / (2 * s2) - 0.5 * nk * np.log(2 * np.pi * s2)
    seg = td.Segment(inputs.white_acf(n, s2), mask)
    for prec in ("fp64", "bf16x6", "bf16x10"):
        ll, _ = _run(torch_cuda, td, seg, R, prec)
        assert np.max(np.abs(ll - exp_ll)) < 1e-6, prec


def test_column_alone_equals_in_batch(torch_cuda, gpu_lib):
    """With the tile shape fixed, a column's logL does not depend on the batch
    it is evaluated in (bitwise); with automatic shapes (which depend on K) it
    agrees within the bar."""
    from paper_2603_06010_b300 import td
    n = 1500
    mask = _mask(n, [(700, 800)])
    seg = td.Segment(inputs.acf_from_psd(n, 2048.0), mask)
    R = inputs.noise_residuals(n, 2048.0, 300, 23, mask=mask)
    Rd = torch_cuda.from_numpy(R).cuda()

    def run(Rsub, opt):
        ll = seg.loglike(Rsub.contiguous(), opt)
        torch_cuda.cuda.synchronize()
        seg.check()
        return ll.cpu().numpy()

    for prec in (td.TD_PREC_FP64, td.TD_PREC_BF16X6, td.TD_PREC_BF16X10):
        for path in ((td.TD_PATH_FP64,) if prec == td.TD_PREC_FP64 else
                     (td.TD_PATH_TENSOR, td.TD_PATH_STREAM, td.TD_PATH_STREAM64, td.TD_PATH_TENSOR128,
                      td.TD_PATH_STREAM128, td.TD_PATH_SMALLK)):
            opt = td.options(precision=prec, path=path)
            # the small-batch kernel takes up to 256 columns: its widths 16 ... 256
            # (whole rows reduced in the kernel below 128 columns, all rows by
            # the chunk reduction from 128; up to 4 columns split rows and the
            # final sums reduced inside the product kernel too) give the same bits
            last = 255 if path == td.TD_PATH_SMALLK else 299
            full = run(Rd[:last + 1], opt)
            for k in (0, 1, 127, 128, last):
                assert run(Rd[k:k + 1], opt)[0] == full[k], (prec, path, k)
            for k0, k1 in ((10, 12), (30, 34), (200, 205)):
                assert np.array_equal(run(Rd[k0:k1], opt), full[k0:k1]), (prec, path, k0, k1)
            assert np.array_equal(run(Rd[100:229], opt), full[100:229]), (prec, path)
            assert np.array_equal(run(Rd[60:100], opt), full[60:100]), (prec, path)
            assert np.array_equal(run(Rd[20:120], opt), full[20:120]), (prec, path)
    auto_full = run(Rd, td.options())
    for k in (0, 5, 299):
        assert abs(run(Rd[k:k + 1], td.options())[0] - auto_full[k]) <= 1e-3


def test_repeatable_bits(torch_cuda, gpu_lib):
    from paper_2603_06010_b300 import td
    n = 1024
    seg = td.Segment(inputs.acf_from_psd(n, 1024.0))
    R = inputs.noise_residuals(n, 1024.0, 200, 29)
    a, _ = _run(torch_cuda, td, seg, R, "bf16x6")
    b, _ = _run(torch_cuda, td, seg, R, "bf16x6")
    assert np.array_equal(a, b)


def test_not_positive_definite(torch_cuda, gpu_lib):
    from paper_2603_06010_b300 import td
    acf = np.zeros(100)
    acf[0], acf[1] = 1.0, 2.0
    with pytest.raises(td.TdError) as e:
        td.Segment(acf)
    assert e.value.code == td.TD_ERR_NOT_PD
    seg = td.Segment(acf, factor=False)
    with pytest.raises(td.TdError):
        seg.factor()
    assert seg.last_pivot == 1
    o = oracle
    with pytest.raises(o.NotPositiveDefinite) as e2:
        o.OracleSegment(acf)
    assert e2.value.pivot == seg.last_pivot


def test_not_factored_and_bad_args(torch_cuda, gpu_lib):
    from paper_2603_06010_b300 import td
    seg = td.Segment(inputs.acf_from_psd(128, 1024.0), factor=False)
    R = torch_cuda.zeros((2, 128), dtype=torch_cuda.float32, device="cuda")
    with pytest.raises(td.TdError) as e:
        seg.loglike(R)
    assert e.value.code == td.TD_ERR_NOT_FACTORED
    seg.factor()
    with pytest.raises(td.TdError) as e:
        seg.loglike_into(R, torch_cuda.empty(2, dtype=torch_cuda.float64, device="cuda"), ldr=100)
    assert e.value.code == td.TD_ERR_INVALID
    # more columns than the entry point takes: refused on the host, nothing launched
    out = torch_cuda.empty(2, dtype=torch_cuda.float64, device="cuda")
    assert td.lib().td_loglike_batch(seg.handle, R.data_ptr(), 128, (1 << 30) + 1, out.data_ptr(), None, None,
                                     None) == td.TD_ERR_INVALID


def test_bounded_wait_times_out_and_context_survives(torch_cuda, gpu_lib):
    from paper_2603_06010_b300 import td
    assert td.debug_bounded_wait(20_000_000) == td.TD_ERR_TIMEOUT
    # the context is still usable
    seg = td.Segment(inputs.white_acf(64, 1.0))
    R = torch_cuda.ones((3, 64), dtype=torch_cuda.float32, device="cuda")
    ll = seg.loglike(R).cpu().numpy()
    assert np.allclose(ll, -32.0 - 32.0 * np.log(2 * np.pi))


# ---------------------------------------------------------------------------
# full-size workloads, sampled columns against stored oracle values
# ---------------------------------------------------------------------------
def _golden():
    with open(os.path.join(HERE, "golden", "full_size.json")) as f:
        return json.load(f)


def _full_case(torch, td, g, prec):
    seg_in = inputs.make_segment(g["n"], g["fs"], g["seed"], n_gaps=g["n_gaps"], gap_len=g["gap_len"],
                                 scale=g["scale"])
    R = inputs.residual_batch(seg_in, g["K"], g["rseed"])
    cols = g["columns"]
    chk = [float(np.sum(R[c].astype(np.float64))) for c in cols]
    assert np.allclose(chk, g["r_checksum"], rtol=1e-6, atol=1e-3), "input generator drifted"
    seg = td.Segment(seg_in.acf, seg_in.mask)
    assert abs(seg.logdet - g["logdet"]) <= 1e-9 * abs(g["logdet"])
    ll, chi = _run(torch, td, seg, R, prec)   # the whole batch, as the benchmark launches it
    seg.close()
    return ll[cols], chi[cols]


@pytest.mark.parametrize("prec", ["bf16x6", "bf16x10", "fp64"])
def test_full_single_n1024(torch_cuda, gpu_lib, prec):
    from paper_2603_06010_b300 import td
    g = _golden()["single_n1024"]
    ll, chi = _full_case(torch_cuda, td, g, prec)
    _compare(prec, ll, chi, np.array(g["logL"]), np.array(g["chi2"]), "single_n1024")


@pytest.mark.parametrize("prec", ["bf16x6", "bf16x10"])
def test_full_gapfree_n8192_k4096(torch_cuda, gpu_lib, prec):
    from paper_2603_06010_b300 import td
    g = _golden()["gapfree_n8192_k4096"]
    ll, chi = _full_case(torch_cuda, td, g, prec)
    _compare(prec, ll, chi, np.array(g["logL"]), np.array(g["chi2"]), "gapfree_n8192_k4096")


@pytest.mark.parametrize("prec", ["bf16x6", "bf16x10"])
def test_full_gapped_n16384_three_detectors(torch_cuda, gpu_lib, prec):
    from paper_2603_06010_b300 import td
    gg = _golden()["gapped_n16384_3det"]
    joint = None
    for g in gg["detectors"]:
        ll, chi = _full_case(torch_cuda, td, g, prec)
        _compare(prec, ll, chi, np.array(g["logL"]), np.array(g["chi2"]), "gapped N=16384 detector")
        joint = ll if joint is None else joint + ll
    assert np.max(np.abs(joint - np.array(gg["joint_logL"]))) <= 1e-3


@pytest.mark.parametrize("K", [100, 256])
def test_full_gapfree_n8192_mid_batches(torch_cuda, gpu_lib, K):
    """Mid-size batches of the N = 8192 workload on the small-batch kernel with
    128- and 256-column tiles (and on the automatic choice): the stored oracle
    columns, placed at the start, the middle and the end of the batch."""
    from paper_2603_06010_b300 import td
    g = _golden()["gapfree_n8192_k4096"]
    seg_in = inputs.make_segment(g["n"], g["fs"], g["seed"], n_gaps=g["n_gaps"], gap_len=g["gap_len"],
                                 scale=g["scale"])
    R = inputs.residual_batch(seg_in, g["K"], g["rseed"])
    cols = list(g["columns"])
    fill = [c for c in range(g["K"]) if c not in cols][:K - len(cols)]
    order = fill[:K // 2 - 5] + cols[:6] + fill[K // 2 - 5:] + cols[6:]
    assert len(order) == K
    pos = [order.index(c) for c in cols]
    seg = td.Segment(seg_in.acf, seg_in.mask, factor=False)
    td.factor_many([seg])
    Rd = torch_cuda.from_numpy(np.ascontiguousarray(R[order])).cuda()
    for path in (td.TD_PATH_SMALLK, td.TD_PATH_AUTO):
        ll, chi = seg.loglike(Rd, td.options(path=path), with_chi2=True)
        torch_cuda.cuda.synchronize()
        seg.check()
        _compare("bf16x6", ll.cpu().numpy()[pos], chi.cpu().numpy()[pos], np.array(g["logL"]),
                 np.array(g["chi2"]), f"N=8192 K={K} path {path}")
    seg.close()


def test_small_batch_path_width_limit(torch_cuda, gpu_lib):
    """The small-batch kernel takes up to 256 columns; wider batches are refused."""
    from paper_2603_06010_b300 import td
    n = 600
    seg = td.Segment(inputs.acf_from_psd(n, 2048.0))
    R = torch_cuda.zeros((257, n), dtype=torch_cuda.float32, device="cuda")
    out = torch_cuda.empty(257, dtype=torch_cuda.float64, device="cuda")
    opt = td.options(path=td.TD_PATH_SMALLK)
    assert td.lib().td_loglike_batch(seg.handle, R.data_ptr(), n, 257, out.data_ptr(), ctypes.byref(opt),
                                     None, None) == td.TD_ERR_UNSUPPORTED
    assert td.lib().td_loglike_batch(seg.handle, R.data_ptr(), n, 256, out.data_ptr(), ctypes.byref(opt),
                                     None, None) == td.TD_OK
    torch_cuda.cuda.synchronize()
    seg.check()
    seg.close()


@pytest.mark.parametrize("K", [1, 5, 17, 32, 48, 64, 100, 130, 256, 300])
def test_tile_shapes_agree(torch_cuda, gpu_lib, K):
    """256- and 128-row whole-row tiles, 256/128/64-row split tiles and the
    small-batch kernel agree within the bar (their correction sums round
    differently), and each matches the oracle."""
    from paper_2603_06010_b300 import td
    n = 2000
    mask = _mask(n, [(900, 1000)])
    seg = td.Segment(inputs.acf_from_psd(n, 2048.0), mask)
    R = torch_cuda.from_numpy(inputs.noise_residuals(n, 2048.0, K, 31, mask=mask)).cuda()
    out = {}
    paths = [td.TD_PATH_TENSOR, td.TD_PATH_STREAM, td.TD_PATH_STREAM64, td.TD_PATH_TENSOR128,
             td.TD_PATH_STREAM128] + ([td.TD_PATH_SMALLK] if K <= 256 else [])
    for path in paths:
        ll, chi = seg.loglike(R, td.options(path=path), with_chi2=True)
        torch_cuda.cuda.synchronize()
        seg.check()
        out[path] = (ll.cpu().numpy(), chi.cpu().numpy())
    o = oracle.OracleSegment(inputs.acf_from_psd(n, 2048.0), mask)
    exp_chi = o.chi2(R.cpu().numpy())
    exp_ll = oracle.loglike_from_chi2(exp_chi, o.logdet, o.n_kept)
    for path, (ll, chi) in out.items():
        _compare("bf16x6", ll, chi, exp_ll, exp_chi, f"path {path}")
    a = out[td.TD_PATH_TENSOR][1]
    for path in paths[1:]:
        b = out[path][1]
        assert np.max(np.abs(a - b) / b) <= 1e-7


def test_host_buffers_match_device_path(torch_cuda, gpu_lib):
    """td_loglike_batch_host (chunked, double-buffered copies) gives the device
    path's bits, for pinned and pageable host memory and a ragged last chunk."""
    from paper_2603_06010_b300 import td
    n = 1500
    mask = _mask(n, [(200, 260)])
    seg = td.Segment(inputs.acf_from_psd(n, 2048.0), mask)
    K = 1300
    R = inputs.noise_residuals(n, 2048.0, K, 77, mask=mask)
    Rd = torch_cuda.from_numpy(R).cuda()
    opt = td.options(path=td.TD_PATH_STREAM)    # one fixed path: bits comparable across batch sizes
    ll_d, chi_d = seg.loglike(Rd, opt, with_chi2=True)
    torch_cuda.cuda.synchronize()
    for pinned in (True, False):
        Rh = torch_cuda.from_numpy(R)
        ll = torch_cuda.empty(K, dtype=torch_cuda.float64)
        chi = torch_cuda.empty(K, dtype=torch_cuda.float64)
        if pinned:
            Rh, ll, chi = Rh.pin_memory(), ll.pin_memory(), chi.pin_memory()
        seg.loglike_host_into(Rh, ll, opt, chi2=chi)
        assert np.array_equal(ll.numpy(), ll_d.cpu().numpy()), pinned
        assert np.array_equal(chi.numpy(), chi_d.cpu().numpy()), pinned
    o = oracle.OracleSegment(inputs.acf_from_psd(n, 2048.0), mask)
    exp = oracle.loglike_from_chi2(o.chi2(R[:64]), o.logdet, o.n_kept)
    assert np.max(np.abs(ll.numpy()[:64] - exp)) <= 1e-3
    seg.close()


@pytest.mark.parametrize("n,K", [(1, 1000), (40, 70000), (2000, 33), (2000, 129), (2000, 257), (2000, 513),
                                 (4096, 300), (4096, 384), (3500, 512)])
def test_extreme_and_transition_shapes(torch_cuda, gpu_lib, n, K):
    """Very wide batches on tiny segments and the batch sizes where the automatic
    tile shape changes (the last three: whole 128-row tiles whose rows above an
    SM's mean share are cut into chunks): every column finite, sampled columns
    against the oracle."""
    from paper_2603_06010_b300 import td
    mask = _mask(n, [(700, 780)]) if n > 1000 else None
    acf = inputs.acf_from_psd(n, 2048.0) if n > 1 else np.array([1.7])
    seg = td.Segment(acf, mask)
    nk = seg.n_kept
    rng = np.random.default_rng(K + n)
    R = (rng.standard_normal((K, nk)) * np.sqrt(acf[0])).astype(np.float32)
    ll, chi = seg.loglike(torch_cuda.from_numpy(R).cuda(), td.options(), with_chi2=True)
    torch_cuda.cuda.synchronize()
    seg.check()
    ll, chi = ll.cpu().numpy(), chi.cpu().numpy()
    assert np.all(np.isfinite(ll))
    cols = np.unique(np.r_[0, K - 1, rng.integers(0, K, 40)])
    o = oracle.OracleSegment(acf, mask)
    exp_chi = o.chi2(R[cols])
    _compare("bf16x6", ll[cols], chi[cols], oracle.loglike_from_chi2(exp_chi, o.logdet, o.n_kept), exp_chi,
             f"n={n} K={K}")
    seg.close()


def test_empty_batch_every_form(torch_cuda, gpu_lib):
    """K = 0 is a no-op on every form of the call: status OK, outputs untouched."""
    from paper_2603_06010_b300 import td
    n = 1500
    acf = inputs.acf_from_psd(n, 2048.0)
    seg = td.Segment(acf)
    seg.gs_prepare()
    R = torch_cuda.zeros((0, n), dtype=torch_cuda.float32, device="cuda")
    out = torch_cuda.full((4,), 7.0, dtype=torch_cuda.float64, device="cuda")
    for opt in (td.options(), td.options(precision=td.TD_PREC_FP64), td.options(path=td.TD_PATH_GSCE),
                td.options(precision=td.TD_PREC_BF16X3, refine=1), td.options(path=td.TD_PATH_SMALLK)):
        assert td.lib().td_loglike_batch(seg.handle, R.data_ptr(), n, 0, out.data_ptr(), ctypes.byref(opt),
                                         None, None) == td.TD_OK
    host = np.full(4, 7.0)
    seg.loglike_host_into(np.zeros((0, n), np.float32), host)
    torch_cuda.cuda.synchronize()
    seg.check()
    assert np.all(out.cpu().numpy() == 7.0) and np.all(host == 7.0)


def test_many_column_tiles(torch_cuda, gpu_lib):
    """K = 20000 on a small gapped segment: 157 column tiles, a ragged last one."""
    from paper_2603_06010_b300 import td
    n = 300
    mask = _mask(n, [(40, 70)])
    acf = inputs.acf_from_psd(n, 1024.0)
    o = oracle.OracleSegment(acf, mask)
    R = inputs.noise_residuals(n, 1024.0, 20000, 99, mask=mask)
    seg = td.Segment(acf, mask)
    ll, chi = _run(torch_cuda, td, seg, R, "bf16x10")
    exp_chi = o.chi2(R)
    _compare("bf16x10", ll, chi, oracle.loglike_from_chi2(exp_chi, o.logdet, o.n_kept), exp_chi, "K=20000")


@pytest.mark.parametrize("gaps", [0, 3])
def test_gather_entry_point_equals_kept_rows(torch_cuda, gpu_lib, gaps):
    """td_loglike_batch_gather on full-length residuals (gap samples included)
    gives the bits of td_loglike_batch on their kept rows, and the oracle's
    values within the bar; bad leading dimensions are refused."""
    from paper_2603_06010_b300 import td
    n, K = 1800, 45
    seg_in = inputs.make_segment(n, 2048.0, 9100 + gaps, n_gaps=gaps, gap_len=150)
    rng = np.random.default_rng(9101)
    Rfull = (rng.standard_normal((K, n + 7)) * np.sqrt(seg_in.acf[0])).astype(np.float32)   # ldr = n + 7
    Rkept = np.ascontiguousarray(Rfull[:, seg_in.kept])
    seg = td.Segment(seg_in.acf, seg_in.mask)
    a = torch_cuda.empty(K, dtype=torch_cuda.float64, device="cuda")
    c = torch_cuda.empty(K, dtype=torch_cuda.float64, device="cuda")
    seg.loglike_gather_into(torch_cuda.from_numpy(Rfull).cuda(), a, chi2=c)
    b = seg.loglike(torch_cuda.from_numpy(Rkept).cuda(), td.options())
    torch_cuda.cuda.synchronize()
    seg.check()
    assert torch_cuda.equal(a, b)
    o = oracle.OracleSegment(seg_in.acf, seg_in.mask)
    exp = o.chi2(Rkept)
    _compare("bf16x6", a.cpu().numpy(), c.cpu().numpy(), oracle.loglike_from_chi2(exp, o.logdet, o.n_kept), exp,
             f"gather gaps={gaps}")
    out = torch_cuda.full((K,), 7.0, dtype=torch_cuda.float64, device="cuda")
    Rd = torch_cuda.from_numpy(Rfull).cuda()
    L = td.lib()
    assert L.td_loglike_batch_gather(seg.handle, Rd.data_ptr(), n - 1, K, out.data_ptr(), None, None,
                                     None) == td.TD_ERR_INVALID
    assert L.td_loglike_batch_gather(seg.handle, Rd.data_ptr(), n, 0, out.data_ptr(), None, None, None) == td.TD_OK
    torch_cuda.cuda.synchronize()
    assert np.all(out.cpu().numpy() == 7.0)
    seg.close()
