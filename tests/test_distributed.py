"""The multi-process path of the benchmark on CPU (gloo, two ranks): the
render path does not shard, so N GPUs run N replicas; each timing is the
maximum over the ranks, the value counts the units of all ranks, and the
reference arm runs on rank 0 alone."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, loc = bench.dist_env()
    # rank r measured (r + 1) ms for the frame and (10 - r) ms for the training step
    fwd, train = bench.max_over_ranks([r + 1.0, 10.0 - r])
    dist.barrier()
    ref = bench.run_reference(type("A", (), {"warmup": 3, "steps": 1, "cpu_budget": 1.0})()) if r != 0 else None
    out.put((r, w, loc, fwd, train, bench.whole_job_rate(w, fwd), ref))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, world, local, fwd, train, rate, ref) in enumerate(res):
        assert (rank, world, local) == (r, 2, r)
        assert (fwd, train) == (2.0, 10.0)       # the slowest rank's times on every rank
        assert rate == 2 * 1000.0 / 2.0          # frames of both replicas per second
    assert res[1][6] is None                     # rank 1 does no reference work


def test_single_process_values_pass_through():
    import bench
    assert bench.max_over_ranks([3.5, 1.25]) == [3.5, 1.25]
    assert bench.whole_job_rate(1, 4.0) == 250.0
