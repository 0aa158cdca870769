"""Multi-replica host logic of the benchmark, on CPU with two gloo ranks: both
ranks get the slowest rank's time (max over ranks), the whole-job throughput
counts every replica's steps, and the reference arm leaves every rank but 0
without work."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, port):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)


def _max_worker(rank, port, q):
    _env(rank, port)
    import torch.distributed as dist
    import bench
    r, w, _ = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    ms = bench.max_over_ranks(1.0 + 2.0 * r, w)  # rank 0 took 1 ms per step, rank 1 3 ms
    bench.rank_barrier(w)
    q.put((r, w, ms, bench.job_iters_per_s(w, ms)))
    dist.destroy_process_group()


def _reference_worker(rank, port, q):
    _env(rank, port)
    import torch.distributed as dist
    import bench
    if rank == 0:
        # rank 0 only joins the group: its reference run is the CPU oracle
        # step, timed elsewhere
        dist.init_process_group("gloo", rank=0, world_size=2)
        dist.barrier()
        q.put((0, "joined"))
    else:
        sys.argv = ["bench.py", "--impl", "reference"]
        bench.main()  # joins the group, then returns before any work
        dist.barrier()
        q.put((1, "returned"))
    dist.destroy_process_group()


def _run(target):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=target, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=180) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in ps)
    return out


def test_two_ranks_take_the_slowest_time():
    out = _run(_max_worker)
    for rank, (r, w, ms, v) in enumerate(out):
        assert r == rank and w == 2
        assert ms == 3.0
        assert abs(v - 2 * 1e3 / 3.0) < 1e-9


def test_reference_arm_runs_on_rank_zero_only():
    assert _run(_reference_worker) == [(0, "joined"), (1, "returned")]


def test_single_rank_helpers_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, 1) == 2.5
    bench.rank_barrier(1)
    assert abs(bench.job_iters_per_s(1, 1.455) - 1e3 / 1.455) < 1e-9
