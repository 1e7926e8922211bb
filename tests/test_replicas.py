"""The multi-GPU path is replicas only: every rank runs its own step, and the job's time is the
slowest rank's.  The host logic of that path (max over ranks, whole-job value, a distinct probe
stream per rank) runs here as two gloo ranks on the CPU."""
import importlib.util
import multiprocessing as mp
import os
import socket

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as td
    td.init_process_group("gloo", rank=rank, world_size=world)
    bench = _bench()
    # rank r took 10 + r ms per step and 30 - r ms end to end
    ms, e2e = bench.replica_times(10.0 + rank, 30.0 - rank)
    seed = bench.make_workload("fcc1k", rank).probe_seed
    out.put((rank, ms, e2e, seed, bench.job_rate(1000.0, world, ms)))
    td.barrier()
    td.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_take_the_slowest_time_and_their_own_probes():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [11.0, 11.0]          # step time: the slower rank's
    assert [r[2] for r in res] == [30.0, 30.0]          # end to end: the slower rank's
    assert res[0][3] != res[1][3]                       # independent probe streams
    assert res[0][4] == res[1][4] == 1000.0 * 2 / 11e-3  # every rank's units over that time


def test_one_process_keeps_its_own_times():
    bench = _bench()
    assert bench.replica_times(4.0, 5.0) == [4.0, 5.0]
    assert bench.job_rate(10.0, 1, 2.0) == 5000.0
