"""Host-side logic of the multi-process benchmark (one process per GPU, each advancing its own
replica; no data exchange): rank discovery from the launcher's environment, the slowest rank's
time, the whole-job aggregate, and the reference arm's rank-0-only rule.  Two gloo ranks on the
CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    r, w, lr = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        ms = [120.0, 250.0][r]  # this rank's timed milliseconds
        ms_max = bench.max_over_ranks(ms, w, "cpu")
        value = bench.aggregate_mlups(w, 1024 * 1024, 1000, 10, ms_max / 1e3)
        dist.barrier()
        q.put((r, lr, w, ms_max, value))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_aggregate_all_cells():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
    for p in procs:
        if p.is_alive():
            p.kill()
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get() for _ in range(2))
    for r, (rank, local, world, ms_max, value) in enumerate(res):
        assert (rank, local, world) == (r, r, 2)
        assert ms_max == 250.0
        # 2 replicas x 2^20 cells x 10^4 time steps in 0.25 s
        assert value == pytest.approx(2 * 1024 * 1024 * 1000 * 10 / 0.25 / 1e6, rel=1e-12)


def test_single_rank_defaults(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (0, 1, 0)
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.aggregate_mlups(1, 100, 10, 2, 0.5) == pytest.approx(100 * 10 * 2 / 0.5 / 1e6)


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench
    # ranks other than 0 return without touching the oracle (args are not even read)
    assert bench.run_reference(None, bench.WORKLOADS["c0"], 1, 2) is None
    assert bench.run_batch_reference(None, 1) is None
