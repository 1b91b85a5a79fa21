"""Grouped launches (many uneven segments, one persistent launch) against the
CPU oracle; CUDA-graph replay and autotuned shapes give the same results."""
import numpy as np
import pytest

import oracle
from paper_2603_06010_b300 import inputs

pytestmark = pytest.mark.gpu

CHI2_REL, DLOGL_ABS = 1e-7, 1e-3

SEGS = [  # (n, fs, a, floor, gaps, K)
    (300, 4096.0, -4.2, 1.5, [], 16),
    (777, 4096.0, -3.6, 2.8, [(100, 140)], 33),
    (1024, 4096.0, -4.0, 2.0, [], 130),
    (1500, 4096.0, -4.4, 1.1, [(200, 300), (900, 950)], 257),
    (2048, 4096.0, -3.9, 2.4, [(0, 64)], 1),
    (640, 4096.0, -4.0, 2.0, [], 0),
]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _build(torch, td):
    segs, Rs, outs, chis, exp_ll, exp_chi = [], [], [], [], [], []
    for i, (n, fs, a, fl, gaps, K) in enumerate(SEGS):
        mask = None
        if gaps:
            mask = np.ones(n, np.uint8)
            for s0, s1 in gaps:
                mask[s0:s1] = 0
        acf = inputs.acf_from_psd(n, fs, a=a, floor=fl)
        seg = td.Segment(acf, mask)
        R = inputs.noise_residuals(n, fs, max(K, 1), 100 + i, mask=mask, a=a, floor=fl)[:K]
        o = oracle.OracleSegment(acf, mask)
        c = o.chi2(R) if K else np.zeros(0)
        exp_chi.append(c)
        exp_ll.append(oracle.loglike_from_chi2(c, o.logdet, o.n_kept) if K else np.zeros(0))
        segs.append(seg)
        Rs.append(torch.from_numpy(np.ascontiguousarray(R)).cuda() if K else
                  torch.zeros((0, o.n_kept), dtype=torch.float32, device="cuda"))
        outs.append(torch.full((K,), np.nan, dtype=torch.float64, device="cuda"))
        chis.append(torch.full((K,), np.nan, dtype=torch.float64, device="cuda"))
    return segs, Rs, outs, chis, exp_ll, exp_chi


def _check_all(outs, chis, exp_ll, exp_chi):
    for ll, ch, el, ec in zip(outs, chis, exp_ll, exp_chi):
        ll = ll.cpu().numpy()
        ch = ch.cpu().numpy()
        if el.size == 0:
            continue
        assert np.max(np.abs(ch - ec) / ec) <= CHI2_REL
        assert np.max(np.abs(ll - el)) <= DLOGL_ABS


def test_grouped_plan_graph_and_tune(torch_cuda, gpu_lib):
    from paper_2603_06010_b300 import td
    segs, Rs, outs, chis, exp_ll, exp_chi = _build(torch_cuda, td)
    g = td.Group(segs, Rs, outs, chis)
    g.launch()
    torch_cuda.cuda.synchronize()
    g.check()
    _check_all(outs, chis, exp_ll, exp_chi)
    first = [x.cpu().numpy().copy() for x in outs]
    # graph replay: same kernels, same plan -> same bits
    for x in outs:
        x.fill_(np.nan)
    g.graph_launch()
    g.graph_launch()
    torch_cuda.cuda.synchronize()
    g.check()
    for a, b in zip(first, outs):
        assert np.array_equal(a, b.cpu().numpy())
    # autotuned shape: still within the bar
    ms = g.tune()
    assert ms > 0
    bn, sf, ni = g.shape()
    assert bn in (0, 64, 128, 256) and sf >= 1 and ni > 0
    for x in outs:
        x.fill_(np.nan)
    g.launch()
    torch_cuda.cuda.synchronize()
    g.check()
    _check_all(outs, chis, exp_ll, exp_chi)
    g.close()


def test_grouped_small_orientation(torch_cuda, gpu_lib):
    """The small-batch kernel's orientation in a grouped launch (operator rows as
    the MMA M, up to 256 residual columns as N, each segment's last column tile
    only as wide as its columns): oracle parity, and graph replay bit for bit."""
    from paper_2603_06010_b300 import td
    segs, Rs, outs, chis, exp_ll, exp_chi = _build(torch_cuda, td)
    g = td.Group(segs, Rs, outs, chis, opt=td.options(path=td.TD_PATH_SMALLK))
    assert g.shape()[0] == 0
    g.launch()
    torch_cuda.cuda.synchronize()
    g.check()
    _check_all(outs, chis, exp_ll, exp_chi)
    first = [x.cpu().numpy().copy() for x in outs]
    for x in outs:
        x.fill_(np.nan)
    g.graph_launch()
    torch_cuda.cuda.synchronize()
    g.check()
    for a, b in zip(first, outs):
        assert np.array_equal(a, b.cpu().numpy())
    g.close()


def test_grouped_mixed_slice_counts(torch_cuda, gpu_lib):
    """Under the default precision each segment takes the slice count one
    segment alone would (ten products below 2048 kept samples, six from 2048):
    a group of both kinds runs one product launch per count and meets the bar
    on every segment."""
    from paper_2603_06010_b300 import td
    specs = [(300, [], 20), (2600, [(500, 700)], 37), (3000, [], 129), (1200, [(0, 50)], 5)]
    segs, Rs, outs, chis, exp_ll, exp_chi = [], [], [], [], [], []
    for i, (n, gaps, K) in enumerate(specs):
        mask = None
        if gaps:
            mask = np.ones(n, np.uint8)
            for s0, s1 in gaps:
                mask[s0:s1] = 0
        acf = inputs.acf_from_psd(n, 4096.0)
        R = inputs.noise_residuals(n, 4096.0, K, 300 + i, mask=mask)
        o = oracle.OracleSegment(acf, mask)
        c = o.chi2(R)
        exp_chi.append(c)
        exp_ll.append(oracle.loglike_from_chi2(c, o.logdet, o.n_kept))
        segs.append(td.Segment(acf, mask))
        Rs.append(torch_cuda.from_numpy(np.ascontiguousarray(R)).cuda())
        outs.append(torch_cuda.full((K,), np.nan, dtype=torch_cuda.float64, device="cuda"))
        chis.append(torch_cuda.full((K,), np.nan, dtype=torch_cuda.float64, device="cuda"))
    g = td.Group(segs, Rs, outs, chis)
    g.graph_launch()
    torch_cuda.cuda.synchronize()
    g.check()
    _check_all(outs, chis, exp_ll, exp_chi)
    g.close()


def test_grouped_one_shot_matches_per_segment(torch_cuda, gpu_lib):
    from paper_2603_06010_b300 import td
    segs, Rs, outs, chis, exp_ll, exp_chi = _build(torch_cuda, td)
    td.loglike_grouped(segs, Rs, outs)
    torch_cuda.cuda.synchronize()
    for seg, R, out in zip(segs, Rs, outs):
        if R.shape[0] == 0:
            continue
        single = seg.loglike(R)
        torch_cuda.cuda.synchronize()
        assert np.max(np.abs(single.cpu().numpy() - out.cpu().numpy())) <= DLOGL_ABS


def test_grouped_joint_three_detectors(torch_cuda, gpu_lib):
    """Multi-detector logL (Sec. II.B item 3): one group over three gapped
    detectors with a common K, the joint sum written by the group launch."""
    from paper_2603_06010_b300 import td
    n, K = 1800, 70
    segs, Rs, outs, exp = [], [], [], []
    joint_exp = np.zeros(K)
    for d, scale in enumerate((1.0, 1.3, 2.1)):
        si = inputs.make_segment(n, 2048.0, 9100 + d, n_gaps=2, gap_len=128, scale=scale)
        R = inputs.residual_batch(si, K, 9200 + d)
        o = oracle.OracleSegment(si.acf, si.mask)
        joint_exp += oracle.loglike_from_chi2(o.chi2(R), o.logdet, o.n_kept)
        segs.append(td.Segment(si.acf, si.mask))
        Rs.append(torch_cuda.from_numpy(R).cuda())
        outs.append(torch_cuda.empty(K, dtype=torch_cuda.float64, device="cuda"))
    g = td.Group(segs, Rs, outs)
    joint = torch_cuda.full((K,), np.nan, dtype=torch_cuda.float64, device="cuda")
    g.set_joint(joint)
    g.graph_launch()
    torch_cuda.cuda.synchronize()
    g.check()
    per = [x.cpu().numpy() for x in outs]
    j = joint.cpu().numpy()
    assert np.array_equal(j, (per[0] + per[1]) + per[2])
    assert np.max(np.abs(j - joint_exp)) <= 3e-3
    g.close()


@pytest.mark.parametrize("case", range(8))
def test_grouped_random_case(torch_cuda, gpu_lib, case):
    """Seeded random groups: 1-6 segments (N' 40 ... 4500, gaps or none, K from 0
    to 300, two sample rates), a random tile family and precision, one captured
    launch, every segment against the oracle at the bar."""
    from paper_2603_06010_b300 import td
    rng = np.random.default_rng(777000 + case)
    segs, Rs, outs, chis, exp_ll, exp_chi = [], [], [], [], [], []
    for i in range(int(rng.integers(1, 7))):
        n = int(rng.integers(40, 4500))
        mask = None
        if n > 200 and rng.random() < 0.5:
            mask = np.ones(n, np.uint8)
            a = int(rng.integers(0, n - 50))
            mask[a:a + int(rng.integers(1, n // 6))] = 0
        K = int(rng.choice([0, 1, 3, 16, 40, 127, 128, 129, 300]))
        fs = float(rng.choice([1024.0, 4096.0]))
        acf = inputs.acf_from_psd(n, fs)
        o = oracle.OracleSegment(acf, mask)
        R = inputs.noise_residuals(n, fs, max(K, 1), 5000 + 10 * case + i, mask=mask)[:K]
        c = o.chi2(R) if K else np.zeros(0)
        exp_chi.append(c)
        exp_ll.append(oracle.loglike_from_chi2(c, o.logdet, o.n_kept) if K else np.zeros(0))
        segs.append(td.Segment(acf, mask))
        Rs.append(torch_cuda.from_numpy(np.ascontiguousarray(R)).cuda() if K else
                  torch_cuda.zeros((0, o.n_kept), dtype=torch_cuda.float32, device="cuda"))
        outs.append(torch_cuda.full((K,), np.nan, dtype=torch_cuda.float64, device="cuda"))
        chis.append(torch_cuda.full((K,), np.nan, dtype=torch_cuda.float64, device="cuda"))
    path = int(rng.choice([td.TD_PATH_AUTO, td.TD_PATH_STREAM, td.TD_PATH_SMALLK, td.TD_PATH_STREAM64]))
    prec = int(rng.choice([td.TD_PREC_AUTO, td.TD_PREC_BF16X10]))
    g = td.Group(segs, Rs, outs, chis, opt=td.options(precision=prec, path=path))
    g.graph_launch()
    torch_cuda.cuda.synchronize()
    g.check()
    _check_all(outs, chis, exp_ll, exp_chi)
    g.close()


@pytest.mark.parametrize("path_name", ["STREAM", "STREAM64"])
def test_grouped_many_segments(torch_cuda, gpu_lib, path_name):
    """36 seeded segments of uneven size (N' 40 ... 3000, gaps, K from 0 to 300)
    in one launch: many items per CTA, taken from the work counter segment by
    segment; every segment against the oracle, graph replay equal to a direct
    launch bit for bit."""
    from paper_2603_06010_b300 import td
    rng = np.random.default_rng(424242)
    segs, Rs, outs, chis, exp_ll, exp_chi = [], [], [], [], [], []
    for i in range(36):
        n = int(rng.integers(40, 3000))
        mask = None
        if n > 300 and rng.random() < 0.4:
            mask = np.ones(n, np.uint8)
            a = int(rng.integers(0, n - 100))
            mask[a:a + int(rng.integers(1, n // 5))] = 0
        K = int(rng.choice([0, 1, 7, 64, 128, 129, 200, 300]))
        acf = inputs.acf_from_psd(n, 4096.0, a=float(rng.uniform(-4.5, -3.5)), floor=float(rng.uniform(1, 3)))
        o = oracle.OracleSegment(acf, mask)
        R = inputs.noise_residuals(n, 4096.0, max(K, 1), 9100 + i, mask=mask)[:K]
        c = o.chi2(R) if K else np.zeros(0)
        exp_chi.append(c)
        exp_ll.append(oracle.loglike_from_chi2(c, o.logdet, o.n_kept) if K else np.zeros(0))
        segs.append(td.Segment(acf, mask))
        Rs.append(torch_cuda.from_numpy(np.ascontiguousarray(R)).cuda() if K else
                  torch_cuda.zeros((0, o.n_kept), dtype=torch_cuda.float32, device="cuda"))
        outs.append(torch_cuda.full((K,), np.nan, dtype=torch_cuda.float64, device="cuda"))
        chis.append(torch_cuda.full((K,), np.nan, dtype=torch_cuda.float64, device="cuda"))
    g = td.Group(segs, Rs, outs, chis, opt=td.options(path=getattr(td, "TD_PATH_" + path_name)))
    g.launch()
    torch_cuda.cuda.synchronize()
    g.check()
    _check_all(outs, chis, exp_ll, exp_chi)
    first = [o.clone() for o in outs]
    for o in outs:
        o.fill_(np.nan)
    g.graph_launch()
    g.graph_launch()
    torch_cuda.cuda.synchronize()
    g.check()
    for a, b in zip(first, outs):
        assert torch_cuda.equal(a, b)
    g.close()
