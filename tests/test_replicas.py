"""Multi-rank host logic on CPU (gloo, world size 2): disjoint quadruple slices, the
max-over-ranks job time and the whole-job throughput."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import coulomb_inputs as ci
from paper_1502_08043_gb300 import replicas


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 500
        first, cnt = replicas.quad_slice(rank, n)
        q = torch.from_numpy(ci.quads(5, first, cnt)).contiguous()
        gathered = [torch.empty_like(q) for _ in range(world)]
        dist.all_gather(gathered, q)
        ms = 1.0 + 2.5 * rank
        job = replicas.max_over_ranks(ms)
        if rank == 0:
            out.put((torch.cat(gathered).numpy(), job,
                     replicas.job_throughput(n, world, job)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    allq, job, thr = out.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    # rank r owns quadruples r*500 .. r*500+499 of the stream: together the first 1000
    assert np.array_equal(allq, ci.quads(5, 0, 1000))
    assert job == 3.5
    assert thr == pytest.approx(2 * 500 / 3.5e-3)


def test_slice_arguments():
    assert replicas.quad_slice(3, 10) == (30, 10)
    with pytest.raises(ValueError):
        replicas.quad_slice(-1, 10)
    assert replicas.max_over_ranks(4.0) == 4.0   # no process group: identity
