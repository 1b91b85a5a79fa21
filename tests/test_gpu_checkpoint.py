"""Factor checkpoint and resume: a segment saved to a file and loaded back
gives the same bits on every path it had, and a damaged file is refused."""
import ctypes
import os

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


def _status(td, seg, R, opt):
    import torch
    out = torch.empty(R.shape[0], dtype=torch.float64, device="cuda")
    st = td.lib().td_loglike_batch(seg.handle, R.data_ptr(), R.stride(0), R.shape[0], out.data_ptr(),
                                   ctypes.byref(opt), None, None)
    torch.cuda.synchronize()
    return st, (out.cpu().numpy() if st == td.TD_OK else None)


def _same_everywhere(td, a, b, R, opts):
    for opt in opts:
        sa, ra = _status(td, a, R, opt)
        sb, rb = _status(td, b, R, opt)
        assert sa == sb, (opt.path, opt.precision, opt.refine, sa, sb)
        if sa == td.TD_OK:
            assert np.array_equal(ra, rb), (opt.path, opt.precision, opt.refine)


def _opts(td):
    return [td.options(), td.options(path=td.TD_PATH_SMALLK), td.options(path=td.TD_PATH_TENSOR128),
            td.options(precision=td.TD_PREC_BF16X10), td.options(precision=td.TD_PREC_FP64),
            td.options(precision=td.TD_PREC_BF16X3, refine=1), td.options(path=td.TD_PATH_GSCE)]


def test_cholesky_factor_round_trip(torch_cuda, gpu_lib, tmp_path):
    from paper_2603_06010_b300 import td
    n = 2500
    seg_in = inputs.make_segment(n, 2048.0, 8100, n_gaps=2, gap_len=200)
    R = torch_cuda.from_numpy(inputs.residual_batch(seg_in, 70, 8101)).cuda()
    a = td.Segment(seg_in.acf, seg_in.mask)
    path = tmp_path / "gapped.ckpt"
    a.save(path)
    assert path.exists() and not os.path.exists(str(path) + ".tmp")
    b = td.Segment.load(path)
    assert b.logdet == a.logdet and b.n_kept == a.n_kept and b.resident_bytes == a.resident_bytes
    _same_everywhere(td, a, b, R, _opts(td))
    o = oracle.OracleSegment(seg_in.acf, seg_in.mask)
    ll = b.loglike(R, td.options())
    torch_cuda.cuda.synchronize()
    exp = o.loglike(R.cpu().numpy())
    assert np.max(np.abs(ll.cpu().numpy() - exp)) <= 1e-3
    # released FP64 factor: the file has no L, and the loaded segment refuses
    # the FP64 path exactly as the saved one does
    a.release_fp64()
    a.save(path)
    c = td.Segment.load(path)
    assert c.resident_bytes == a.resident_bytes < b.resident_bytes
    _same_everywhere(td, a, c, R, _opts(td))
    for s in (a, b, c):
        s.close()


def test_levinson_and_gsce_round_trip(torch_cuda, gpu_lib, tmp_path):
    from paper_2603_06010_b300 import td
    n = 4096
    acf = inputs.acf_from_psd(n, 2048.0)
    a = td.Segment(acf, factor=False)
    td.factor_many([a])
    a.gs_prepare()
    R = torch_cuda.from_numpy(inputs.noise_residuals(n, 2048.0, 33, 8201)).cuda()
    path = tmp_path / "gapfree.ckpt"
    a.save(path)
    b = td.Segment.load(path)
    assert b.logdet == a.logdet
    _same_everywhere(td, a, b, R, _opts(td))
    # GSCE alone (never factored)
    g = td.Segment(acf, factor=False)
    g.gs_prepare()
    g.save(path)
    h = td.Segment.load(path)
    assert h.logdet == g.logdet
    _same_everywhere(td, g, h, R, [td.options(path=td.TD_PATH_GSCE), td.options()])
    for s in (a, b, g, h):
        s.close()


def test_damaged_and_refused_files(torch_cuda, gpu_lib, tmp_path):
    from paper_2603_06010_b300 import td
    n = 1200
    a = td.Segment(inputs.acf_from_psd(n, 2048.0))
    path = tmp_path / "seg.ckpt"
    a.save(path)
    raw = bytearray(path.read_bytes())
    raw[len(raw) // 2] ^= 0x40            # one bit in the operator payload
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(bytes(raw))
    h = ctypes.c_void_p()
    assert td.lib().td_segment_load(str(bad).encode(), None, ctypes.byref(h)) == td.TD_ERR_INVALID
    assert h.value is None
    assert b"checksum" in td.lib().td_last_error()
    # an unfactored segment has nothing to save; an unwritable path writes nothing
    u = td.Segment(inputs.acf_from_psd(n, 2048.0), factor=False)
    assert td.lib().td_segment_save(u.handle, str(tmp_path / "u.ckpt").encode(), None) == td.TD_ERR_NOT_FACTORED
    nowhere = tmp_path / "no_such_dir" / "x.ckpt"
    assert td.lib().td_segment_save(a.handle, str(nowhere).encode(), None) == td.TD_ERR_INVALID
    assert not (tmp_path / "u.ckpt").exists() and not nowhere.parent.exists()
    # the good file still loads after all that
    b = td.Segment.load(path)
    R = torch_cuda.from_numpy(inputs.noise_residuals(n, 2048.0, 5, 8301)).cuda()
    _same_everywhere(td, a, b, R, [td.options()])
    for s in (a, b, u):
        s.close()
