"""Multi-rank partition of the imaging work, on CPU with gloo (world size 2).

Each rank images its own chunks with the CPU oracle (the GPU kernels are not needed to check the
bookkeeping); the union over ranks must equal the single-process result, every chunk must be imaged
exactly once, and the job time must be the max over ranks.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2505_15204_gb300.shard import chunks_for_rank, job_rate, max_over_ranks


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _images_of_chunk(chunk):
    import blinksynth as bs
    import oracle
    w = bs.build_workload("fullband", chunk=chunk, n_samples=10)
    v = np.ascontiguousarray(w["volt"][:, :8])
    out = oracle.pipeline(v, w["enu"], w["freqs"][:8], 10, 4, 64)
    return out["images"]


def _worker(rank, world, port, n_chunks, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = chunks_for_rank(n_chunks, rank, world)
    imgs = {c: _images_of_chunk(c) for c in mine}
    t = max_over_ranks(1.0 + rank, dist)
    q.put((rank, mine, imgs, t))
    dist.barrier()
    dist.destroy_process_group()


def test_partition_covers_every_chunk_once():
    for world in (1, 2, 3, 8):
        seen = []
        for r in range(world):
            seen += chunks_for_rank(20, r, world, first=4)
        assert sorted(seen) == list(range(20))
    with pytest.raises(ValueError):
        chunks_for_rank(4, 2, 2)
    # more ranks than chunks: every rank still images one chunk (replicas of the single-chunk workloads)
    assert [chunks_for_rank(1, r, 4) for r in range(4)] == [[0], [0], [0], [0]]
    assert [chunks_for_rank(3, r, 4, first=1) for r in range(4)] == [[1], [2], [0], [1]]
    assert job_rate(100, 4, 2.0) == 200.0


def test_two_gloo_ranks_reproduce_the_single_process_images():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world, n_chunks = 2, 3
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_chunks, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = {}
    for rank, mine, imgs, t in res:
        assert t == 2.0                       # max over ranks of (1 + rank)
        for c in mine:
            assert c not in got
            got[c] = imgs[c]
    assert sorted(got) == list(range(n_chunks))
    for c in range(n_chunks):
        assert np.array_equal(got[c], _images_of_chunk(c))
