"""The multi-GPU path of the benchmark runs independent replicas (no
collective on the data path); its one collective is the MAX over ranks of the
timed seconds.  Two gloo ranks on the CPU check the whole-job throughput:
every rank reports the units of all ranks over the slowest rank's time."""
import importlib.util
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, seconds, q):
    import torch
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, _bench().replica_throughput(seconds[rank], 10, world, "cpu")))
    finally:
        torch.distributed.destroy_process_group()


def test_replica_throughput_single_rank():
    assert _bench().replica_throughput(2.0, 10, 1, "cpu") == (5.0, 2.0)


def test_replica_throughput_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    seconds = [0.5, 0.8]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, seconds, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    for r in range(2):
        value, slowest = got[r]
        assert slowest == pytest.approx(0.8)
        assert value == pytest.approx(2 * 10 / 0.8)
