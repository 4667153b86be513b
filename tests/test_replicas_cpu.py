"""The multi-GPU path (replicas) on CPU: two gloo ranks, the slowest rank's time and the whole-job rate."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    from paper_1209_6038_gb300 import replicas
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    env = replicas.dist_env()
    t = replicas.max_over_ranks(1.5 + rank)  # rank 1 is slower
    rate = replicas.whole_job_rate(1000.0, t, env[0])
    out.put((rank, env, t, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, env, t, rate in res:
        assert env == (2, rank, rank)
        assert t == 2.5
        assert rate == pytest.approx(2 * 1000.0 / 2.5)


def test_single_process_needs_no_group():
    from paper_1209_6038_gb300 import replicas
    assert replicas.max_over_ranks(3.25) == 3.25
    assert replicas.whole_job_rate(10.0, 2.0, 1) == 5.0
