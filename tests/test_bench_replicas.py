"""The replica path of bench.py (``--gpus N`` under torchrun: N independent
solves, timed intervals reduced to the slowest rank) on CPU: two gloo ranks
on 127.0.0.1 call the same reduction the bench applies to its timed
interval and to its end-to-end time, and both get the larger value."""
import importlib.util
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, values, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        assert b.dist_env()[:2] == (rank, world)
        out.put((rank, b.max_over_ranks(values[rank], world, device="cpu")))
    finally:
        dist.destroy_process_group()


def test_single_process_keeps_its_value():
    assert _bench().max_over_ranks(0.25, 1) == 0.25


@pytest.mark.parametrize("values", [(0.31, 0.27), (1.0, 2.5)])
def test_two_gloo_ranks_agree_on_the_slowest(values):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, values, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: max(values), 1: max(values)}
