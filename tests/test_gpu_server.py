"""The continuous-batching server (td_server) through the C ABI."""
import threading

import numpy as np
import pytest

import oracle
from paper_2603_06010_b300 import inputs

pytestmark = pytest.mark.gpu

DLOGL_ABS = 1e-3


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _segments():
    out = []
    for i, (n, gaps) in enumerate([(1024, []), (1500, [(300, 420)]), (2048, [(0, 50), (1900, 2048)])]):
        mask = None
        if gaps:
            mask = np.ones(n, np.uint8)
            for a, b in gaps:
                mask[a:b] = 0
        acf = inputs.acf_from_psd(n, 2048.0)
        out.append((acf, mask, oracle.OracleSegment(acf, mask)))
    return out


def _request(torch, o, K, seed):
    R = inputs.noise_residuals(o.n, 2048.0, K, seed, mask=o.mask)
    exp = oracle.loglike_from_chi2(o.chi2(R), o.logdet, o.n_kept)
    return torch.from_numpy(R).cuda(), torch.full((K,), np.nan, dtype=torch.float64, device="cuda"), exp


def test_server_results_match_oracle(torch_cuda, gpu_lib):
    from paper_2603_06010_b300 import td
    segs = _segments()
    srv = td.Server(max_batch_cols=1024, n_streams=3, max_kept=4096)
    ids = [srv.add_segment(a, m) for a, m, _ in segs]
    for i in ids:
        srv.prefetch(i)
    rng = np.random.default_rng(1)
    reqs = []
    for q in range(30):
        s = int(rng.integers(0, len(ids)))
        K = int(rng.choice([1, 8, 64, 200]))
        R, out, exp = _request(torch_cuda, segs[s][2], K, 500 + q)
        reqs.append((srv.submit(ids[s], R, out), R, out, exp))
    srv.drain()
    for t, R, out, exp in reqs:
        assert srv.poll(t) == td.Server.DONE
        assert np.max(np.abs(out.cpu().numpy() - exp)) <= DLOGL_ABS
    st = srv.stats()
    assert st["requests_done"] == 30 and st["failed"] == 0 and st["batches"] >= 3
    assert st["p99_us"] >= st["p50_us"] > 0
    srv.close()


def test_same_alone_and_in_the_mix(torch_cuda, gpu_lib):
    """A request gives the same logL, bit for bit, when it runs alone and when
    it is batched with other requests arriving at the same time (deterministic
    server: one fixed path per segment, whatever the batch width)."""
    from paper_2603_06010_b300 import td
    segs = _segments()
    acf, mask, o = segs[1]
    srv = td.Server(max_batch_cols=2048, n_streams=2, max_kept=4096, deterministic=True)
    sid = srv.add_segment(acf, mask)
    srv.prefetch(sid)
    R, alone, exp = _request(torch_cuda, o, 8, 77)
    srv.wait(srv.submit(sid, R, alone))
    mixed = torch_cuda.full((8,), np.nan, dtype=torch_cuda.float64, device="cuda")
    others = [_request(torch_cuda, o, k, 900 + k) for k in (1, 64, 200, 3)]
    srv.pause(True)
    ts = [srv.submit(sid, r, out) for r, out, _ in others[:2]]
    t_mix = srv.submit(sid, R, mixed)
    ts += [srv.submit(sid, r, out) for r, out, _ in others[2:]]
    srv.pause(False)
    srv.drain()
    a, b = alone.cpu().numpy(), mixed.cpu().numpy()
    assert srv.poll(t_mix) == td.Server.DONE
    assert np.array_equal(a, b)
    assert np.max(np.abs(a - exp)) <= DLOGL_ABS
    for (r, out, e), t in zip(others, ts):
        assert np.max(np.abs(out.cpu().numpy() - e)) <= DLOGL_ABS
    srv.close()


def test_cancel_before_batching(torch_cuda, gpu_lib):
    from paper_2603_06010_b300 import td
    acf, mask, o = _segments()[0]
    srv = td.Server(max_kept=4096)
    sid = srv.add_segment(acf, mask)
    srv.prefetch(sid)
    srv.pause(True)
    reqs = [_request(torch_cuda, o, 4, 30 + i) for i in range(5)]
    ts = [srv.submit(sid, R, out) for R, out, _ in reqs]
    srv.cancel(ts[1])
    srv.cancel(ts[3])
    srv.pause(False)
    srv.drain()
    for i, (t, (R, out, exp)) in enumerate(zip(ts, reqs)):
        if i in (1, 3):
            assert srv.poll(t) == td.Server.CANCELLED
            assert np.all(np.isnan(out.cpu().numpy()))
        else:
            assert srv.poll(t) == td.Server.DONE
            assert np.max(np.abs(out.cpu().numpy() - exp)) <= DLOGL_ABS
    with pytest.raises(td.TdError):
        srv.cancel(ts[0])          # already finished
    srv.close()


def test_lru_eviction_and_reload(torch_cuda, gpu_lib):
    from paper_2603_06010_b300 import td
    segs = _segments()
    probe = td.Segment(segs[2][0], segs[2][1])
    budget = probe.resident_bytes // 2     # room for about one operator
    probe.close()
    srv = td.Server(resident_bytes_budget=budget, n_streams=1, max_kept=4096)
    ids = [srv.add_segment(a, m) for a, m, _ in segs]
    for i in ids:
        srv.prefetch(i)
    results = []
    for q in range(6):
        s = q % 3
        R, out, exp = _request(torch_cuda, segs[s][2], 16, 60 + q)
        srv.wait(srv.submit(ids[s], R, out))
        results.append((out, exp))
    for out, exp in results:
        assert np.max(np.abs(out.cpu().numpy() - exp)) <= DLOGL_ABS
    st = srv.stats()
    assert st["evictions"] > 0 and st["misses"] > 0 and st["reloads"] > 0
    srv.close()


def test_deterministic_mix_over_batch_widths(torch_cuda, gpu_lib):
    """Deterministic server: requests of 1 .. 300 columns on one segment, each
    submitted alone and then all together (one batch of more than 256 columns,
    run in chunks), give identical bits; and the automatic server agrees with
    them within the bar."""
    torch = torch_cuda
    from paper_2603_06010_b300 import td
    acf, mask, o = _segments()[2]
    reqs = [_request(torch, o, k, 1300 + k) for k in (1, 5, 40, 130, 300)]
    srv = td.Server(max_batch_cols=1024, n_streams=3, max_kept=4096, deterministic=True)
    sid = srv.add_segment(acf, mask)
    srv.prefetch(sid)
    alone = []
    for R, _, _ in reqs:
        out = torch.full((R.shape[0],), np.nan, dtype=torch.float64, device="cuda")
        srv.wait(srv.submit(sid, R, out))
        alone.append(out.cpu().numpy())
    srv.pause(True)
    mixed = [torch.full((R.shape[0],), np.nan, dtype=torch.float64, device="cuda") for R, _, _ in reqs]
    ts = [srv.submit(sid, R, out) for (R, _, _), out in zip(reqs, mixed)]
    srv.pause(False)
    srv.drain()
    assert all(srv.poll(t) == td.Server.DONE for t in ts)
    for a, m, (_, _, exp) in zip(alone, mixed, reqs):
        assert np.array_equal(a, m.cpu().numpy())
        assert np.max(np.abs(a - exp)) <= DLOGL_ABS
    srv.close()


def test_admission_refused_when_full(torch_cuda, gpu_lib):
    from paper_2603_06010_b300 import td
    acf, mask, o = _segments()[0]
    srv = td.Server(max_pending_cols=100, max_batch_cols=64, max_kept=4096)
    sid = srv.add_segment(acf, mask)
    srv.prefetch(sid)
    srv.pause(True)
    R1, out1, e1 = _request(torch_cuda, o, 64, 1)
    R2, out2, _ = _request(torch_cuda, o, 64, 2)
    t1 = srv.submit(sid, R1, out1)
    with pytest.raises(td.TdError) as e:
        srv.submit(sid, R2, out2)
    assert e.value.code == td.TD_ERR_BUSY
    srv.pause(False)
    srv.wait(t1)
    assert np.max(np.abs(out1.cpu().numpy() - e1)) <= DLOGL_ABS
    assert srv.stats()["refused"] == 1
    t2 = srv.submit(sid, R2, out2)   # room again once the first has finished
    srv.wait(t2)
    srv.close()


def test_concurrent_submitters(torch_cuda, gpu_lib):
    from paper_2603_06010_b300 import td
    segs = _segments()
    srv = td.Server(max_batch_cols=512, n_streams=4, max_kept=4096)
    ids = [srv.add_segment(a, m) for a, m, _ in segs]
    for i in ids:
        srv.prefetch(i)
    work = []
    for q in range(24):
        s = q % 3
        R, out, exp = _request(torch_cuda, segs[s][2], [1, 8, 64][q % 3], 700 + q)
        work.append((ids[s], R, out, exp))
    torch_cuda.cuda.synchronize()
    errors = []

    def client(chunk):
        try:
            for sid, R, out, _ in chunk:
                srv.wait(srv.submit(sid, R, out))
        except Exception as ex:   # pragma: no cover - reported below
            errors.append(ex)

    th = [threading.Thread(target=client, args=(work[i::4],)) for i in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors
    for _, R, out, exp in work:
        assert np.max(np.abs(out.cpu().numpy() - exp)) <= DLOGL_ABS
    srv.close()


def test_gapfree_segment_served_through_gsce(torch_cuda, gpu_lib):
    """gs_gapfree: batches that TD_PATH_AUTO sends to GSCE run on the segment's
    Gohberg-Semencul data without loading its dense operator; results match
    the oracle."""
    from paper_2603_06010_b300 import td
    n = 3000
    acf = inputs.acf_from_psd(n, 2048.0)
    o = oracle.OracleSegment(acf)
    srv = td.Server(max_batch_cols=256, n_streams=2, max_kept=4096, gs_gapfree=True)
    sid = srv.add_segment(acf)
    reqs = []
    for q in range(12):
        R, out, exp = _request(torch_cuda, o, [1, 8, 64][q % 3], 900 + q)
        reqs.append((srv.submit(sid, R, out), out, exp))
    srv.drain()
    for t, out, exp in reqs:
        assert srv.poll(t) == td.Server.DONE
        assert np.max(np.abs(out.cpu().numpy() - exp)) <= DLOGL_ABS
    assert srv.stats()["resident_bytes"] == 0


def test_spill_pool_and_runtime_budget(torch_cuda, gpu_lib):
    """Operators spilled to the pinned pool reserved at creation, after the budget
    is lowered at run time; reloaded operators give the same bits as before."""
    torch = torch_cuda
    from paper_2603_06010_b300 import td
    segs = _segments()
    srv = td.Server(n_streams=2, max_kept=4096, host_spill_bytes=64 << 20)
    ids = [srv.add_segment(a, m) for a, m, _ in segs]
    for i in ids:
        srv.prefetch(i)
    reqs = [_request(torch, segs[i][2], 24, 1700 + i) for i in range(3)]
    first = []
    for i, (R, out, exp) in enumerate(reqs):
        srv.wait(srv.submit(ids[i], R, out))
        first.append(out.cpu().numpy().copy())
        assert np.max(np.abs(first[-1] - exp)) <= DLOGL_ABS
    srv.stats(reset=True)
    srv.set_budget(1)            # nothing fits: every new segment evicts the others
    for q in range(6):
        i = q % 3
        R, out, _ = reqs[i]
        out.fill_(np.nan)
        srv.wait(srv.submit(ids[i], R, out))
        assert np.array_equal(out.cpu().numpy(), first[i])
    st = srv.stats()
    assert st["evictions"] >= 4 and st["reloads"] >= 4 and st["failed"] == 0
    srv.close()

