"""Multi-rank host path on CPU (gloo, world_size 2): sharded oracle
evaluations reassemble to the single-process result, and the timing
aggregation is a max over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2603_06010_b300 import dist as tddist


def test_shard_columns_cover_exactly():
    for K in (0, 1, 7, 4096):
        for world in (1, 2, 3, 8):
            spans = [tddist.shard_columns(K, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == K
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1


def test_shard_segments_balanced():
    work = [float(n * n * k) for n, k in [(512, 16), (32768, 400), (8192, 64), (4096, 512), (1024, 100),
                                          (16384, 20), (2048, 300)]]
    parts = tddist.shard_segments(work, 2)
    assert sorted(sum(parts, [])) == list(range(len(work)))
    loads = [sum(work[i] for i in p) for p in parts]
    assert max(loads) <= sum(work)          # trivially, and the LPT bound:
    assert max(loads) <= sum(work) / 2 + max(work)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_q):
    import torch
    import torch.distributed as dist
    import oracle
    from paper_2603_06010_b300 import inputs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n, K = 400, 10
    mask = np.ones(n, np.uint8)
    mask[100:150] = 0
    R = inputs.noise_residuals(n, 1024.0, K, 5, mask=mask)
    seg = oracle.OracleSegment(inputs.acf_from_psd(n, 1024.0), mask)
    a, b = tddist.shard_columns(K, world, rank)
    ll = seg.loglike(R[a:b])
    parts = [None] * world
    dist.all_gather_object(parts, (a, b, ll.tolist()))
    t_max, evals = tddist.aggregate(0.1 * (rank + 1), b - a)
    if rank == 0:
        full = np.zeros(K)
        for a2, b2, v in parts:
            full[a2:b2] = v
        out_q.put((full.tolist(), seg.loglike(R).tolist(), t_max, evals))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_sharded_evaluation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    full, single, t_max, evals = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert np.array_equal(np.array(full), np.array(single))
    assert t_max == pytest.approx(0.2) and evals == 10
