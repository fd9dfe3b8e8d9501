"""Host logic of the multi-replica benchmark on CPU: two gloo ranks.

Rays, frames and renders are independent, so N GPUs run N replicas with no collective on
the data path; the only cross-rank steps are the barrier and the reductions of the timing
(max over ranks) and of the work (sum over ranks).  These run here with the gloo backend.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, samples, ms, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        steps = 5
        value, ms_per_step = bench.replica_throughput(samples[rank], steps, ms[rank], world)
        mx = bench.max_over_ranks(float(rank + 1), world)
        sm = bench.sum_over_ranks(float(rank + 1), world)
        out[rank] = (value, ms_per_step, mx, sm)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replica_throughput_takes_total_work_over_slowest_rank(world):
    samples = [1_000_000, 3_000_000]  # per step
    ms = [10.0, 25.0]  # total of the timed steps on each rank
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, samples, ms, out))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    steps = 5
    want_value = sum(samples) * steps / (max(ms) / 1e3) / 1e9
    for r in range(world):
        value, ms_per_step, mx, sm = out[r]
        assert value == pytest.approx(want_value, rel=1e-12)
        assert ms_per_step == pytest.approx(max(ms) / steps, rel=1e-12)
        assert mx == float(world)
        assert sm == float(world * (world + 1) // 2)


def test_single_rank_needs_no_process_group():
    import bench

    value, ms_per_step = bench.replica_throughput(2_000_000, 4, 8.0, 1)
    assert value == pytest.approx(2_000_000 * 4 / 8e-3 / 1e9)
    assert ms_per_step == 2.0
