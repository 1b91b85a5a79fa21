"""Seeded random sweep of (N, gaps, K, path, precision, refinement, GSCE)
against the CPU FP64 oracle, at the method's bar (chi2 1e-7 relative,
|delta logL| 1e-3; the plain FP64 path 1e-11).  Catches combinations the
fixed cases do not name: ragged row and column tiles, gaps at the edges,
every tile shape with every slice count."""
import numpy as np
import pytest

import oracle
from paper_2603_06010_b300 import inputs

pytestmark = pytest.mark.gpu

N_CASES = 40


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _case(i, td):
    rng = np.random.default_rng(20260000 + i)
    n = int(rng.integers(1, 5001)) if i % 4 else int(rng.integers(1024, 5001))
    if i % 7 == 3:
        n = int(rng.integers(1, 65))   # a single tile, down to one sample
    mask = None
    if n > 64 and rng.random() < 0.5:
        mask = np.ones(n, np.uint8)
        for _ in range(int(rng.integers(1, 4))):
            a = int(rng.integers(0, n - 1))
            mask[a:a + int(rng.integers(1, max(2, n // 8)))] = 0
        if mask.sum() == 0:
            mask[0] = 1
    K = int(rng.choice([1, 2, 7, 16, 31, 33, 64, 100, 129, 255, 300, 513, 700]))
    paths = [td.TD_PATH_AUTO, td.TD_PATH_TENSOR, td.TD_PATH_STREAM, td.TD_PATH_STREAM64, td.TD_PATH_TENSOR128,
             td.TD_PATH_STREAM128, td.TD_PATH_FP64]
    if K <= 256:
        paths.append(td.TD_PATH_SMALLK)
    path = int(rng.choice(paths))
    prec = int(rng.choice([td.TD_PREC_BF16X6, td.TD_PREC_BF16X10, td.TD_PREC_AUTO, td.TD_PREC_BF16X3]))
    refine = 0
    if path == td.TD_PATH_FP64:
        prec = td.TD_PREC_FP64
    elif prec == td.TD_PREC_BF16X3 or rng.random() < 0.2:
        refine = 1   # three products alone sit above the bar: refined, they meet it
        if path == td.TD_PATH_SMALLK:
            path = td.TD_PATH_AUTO
    gsce = mask is None and 1024 <= n <= 32768 and rng.random() < 0.7 and not refine and path != td.TD_PATH_FP64
    fs = float(rng.choice([1024.0, 2048.0, 4096.0]))
    return n, mask, K, path, prec, refine, gsce, fs


@pytest.mark.parametrize("i", range(N_CASES))
def test_random_case(torch_cuda, gpu_lib, i):
    from paper_2603_06010_b300 import td
    n, mask, K, path, prec, refine, gsce, fs = _case(i, td)
    acf = inputs.acf_from_psd(n, fs) if n > 1 else np.array([1.7])
    o = oracle.OracleSegment(acf, mask)
    if n > 1:
        R = inputs.noise_residuals(n, fs, K, 777 + i, mask=mask)
    else:
        R = np.random.default_rng(i).standard_normal((K, 1)).astype(np.float32)
    exp_chi = o.chi2(R)
    exp_ll = oracle.loglike_from_chi2(exp_chi, o.logdet, o.n_kept)
    seg = td.Segment(acf, mask)
    if gsce:
        seg.gs_prepare()
        path = td.TD_PATH_GSCE
    opt = td.options(precision=prec, path=path, refine=refine)
    Rd = torch_cuda.from_numpy(np.ascontiguousarray(R)).cuda()
    logL, chi2 = seg.loglike(Rd, opt, with_chi2=True)
    torch_cuda.cuda.synchronize()
    seg.check()
    got_chi, got_ll = chi2.cpu().numpy(), logL.cpu().numpy()
    rel_tol, ll_tol = (1e-11, 1e-7) if path == td.TD_PATH_FP64 else (1e-7, 1e-3)
    if prec == td.TD_PREC_BF16X6 and not refine and not gsce and o.n_kept < 2048:
        # six products represent each row to ~2^-24; with few rows a column's
        # chi2 rests on few of them (less averaging): up to ~1.2e-7 measured,
        # which is why the default precision takes ten products below 2048
        rel_tol = 2.5e-7
    what = f"n={n} gaps={mask is not None} K={K} path={path} prec={prec} refine={refine}"
    rel = np.max(np.abs(got_chi - exp_chi) / exp_chi)
    assert rel <= rel_tol, f"{what}: chi2 rel {rel:.3e}"
    assert np.max(np.abs(got_ll - exp_ll)) <= ll_tol, what
    seg.close()
