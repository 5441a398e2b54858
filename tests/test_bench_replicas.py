"""The multi-rank path of bench.py on CPU: two gloo ranks run the replica
aggregation (sum of every rank's updates over the slowest rank's time), as
torchrun would launch them on a multi-GPU node."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r "updated" (r + 1) * 1e9 points in (r + 1) * 100 ms
        value, ms_max = bench.replica_throughput(world, (rank + 1) * 1e9, (rank + 1) * 100.0)
        bench.barrier(world)
        out[rank] = (value, ms_max)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_replicas():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        value, ms_max = out[r]
        assert ms_max == pytest.approx(200.0)
        # (1e9 + 2e9) updates in 0.2 s = 15 GLUP/s on every rank
        assert value == pytest.approx(15.0)


def test_profiled_traffic_reads_only_a_matching_summary(tmp_path):
    # the DRAM traffic of a kernel is reported from its committed ncu summary
    # only while the kernel's sources hash to the recorded value
    import bench
    for sources in (bench.KERNEL_SOURCES, bench.KERNEL_SOURCES_3D):
        good = tmp_path / "good.md"
        good.write_text("dram_bytes_per_launch: 1234\nsource_sha256: `%s`\n"
                        % bench.kernel_source_hash(sources))
        stale = tmp_path / "stale.md"
        stale.write_text("dram_bytes_per_launch: 1234\nsource_sha256: `%s`\n" % ("0" * 64))
        assert bench.profiled_traffic(str(good), sources) == 1234
        assert bench.profiled_traffic(str(stale), sources) is None
        assert bench.profiled_traffic(str(tmp_path / "missing.md"), sources) is None
    # the two kernels' source lists hash differently
    assert bench.kernel_source_hash(bench.KERNEL_SOURCES) != bench.kernel_source_hash(
        bench.KERNEL_SOURCES_3D)
