"""The bench's multi-rank logic (one process per GPU under torchrun) on CPU: two gloo ranks.

On a GPU machine every rank projects its own batch (weak scaling, no data-path collective); the only
cross-rank steps are the barrier around the timed region and the max of the ranks' times.  These
tests run those steps with the gloo backend, and check that the reference arm works on rank 0
only.
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
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = bench.max_over_ranks(times[rank], world, "cpu")
        value = bench.job_throughput(1024 * 65536, world, ms * 1e-3)
        dist.barrier()
        results[rank] = (ms, value)
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    times = [0.81, 0.93]          # the second rank is slower
    with mp.Manager() as m:
        results = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), times, results), nprocs=world, join=True)
        res = dict(results)
    for rank in range(world):
        ms, value = res[rank]
        assert ms == max(times)                                   # every rank sees the job's time
        assert value == pytest.approx(2 * 1024 * 65536 / (max(times) * 1e-3))


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(1.25, 1, "cpu") == 1.25
    assert bench.job_throughput(100, 1, 2.0) == 50.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    class Args:
        workload = "c65k"
        steps = 1
        warmup = 1
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(Args())          # other ranks: no work, no output
    assert capsys.readouterr().out == ""


def test_ncu_traffic_lookup_scales_to_the_launch():
    # profiles/ncu_traffic.txt: DRAM bytes of one captured launch, the pairs it covered and the
    # FFT length of the captured workload (another length has no figure)
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    rows = {}
    with open(path) as f:
        for line in f:
            parts = line.split()
            if len(parts) == 4 and not line.startswith("#"):
                rows[parts[0]] = (float(parts[1]), float(parts[2]), int(parts[3]))
    assert "k_fastB4096" in rows
    b, pairs, M = rows["k_fastB4096"]
    assert bench.ncu_traffic("k_fastB4096", pairs, M) == b
    assert bench.ncu_traffic("k_fastB4096", 2 * pairs, M) == 2 * b
    assert bench.ncu_traffic("k_fastB4096", pairs, 2 * M) is None
    assert bench.ncu_traffic("no_such_kernel", 1, M) is None
