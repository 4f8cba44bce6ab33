"""Multi-rank host path of bench.py on CPU (gloo, world size 2): every rank
reports its own time, the job time is the maximum over ranks and the job
throughput counts the node updates of all ranks."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms_local = 100.0 + 50.0 * rank  # rank 1 is slower
    value, ms = bench.job_value(ms_local, 1_000_000, 10, world, dist, "cpu")
    out[rank] = (value, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_job_value_uses_slowest_rank():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    for r in range(world):
        value, ms = out[r]
        assert ms == 150.0
        assert value == pytest.approx(world * 1_000_000 * 10 / 0.150 / 1e6)


def test_job_value_single_rank():
    import bench

    v, ms = bench.job_value(200.0, 2_000_000, 5, 1)
    assert ms == 200.0 and v == pytest.approx(2_000_000 * 5 / 0.2 / 1e6)


def test_collide_kernel_names_and_traffic():
    """The bench names the kernel a collision form launches and takes the
    DRAM traffic measured for that form."""
    import bench
    assert bench.collide_kernel_name("f64", 3, 5).startswith("collide_prefetch_kernel")
    assert bench.collide_kernel_name("f64", 3, 9).startswith("collide_kernel")
    assert bench.collide_kernel_name("f32dev", 3, 9).startswith("collide_pair_kernel")
    assert "covered" in bench.collide_kernel_name("dfdev", 3, 6)
    # measured forms only: the FP64 pulled-ahead form above its algorithmic
    # 309.7 B per node, an uncaptured form without a figure
    assert 309.7 < bench.traffic_per_node("f64", 3, 5) < 400.0
    assert bench.traffic_per_node("f64", 3, 0) is None
    assert bench.traffic_per_node("f64", 2, 0) is None


def test_result_line_fits_the_record():
    """The printed result line stays within the characters the record keeps:
    optional summaries go first, the contract's keys stay."""
    import json
    import bench

    line = {"metric": "m", "value": 1.0, "unit": "MLUPS", "roofline": {"frac": 0.9}, "e2e": {"value": 1.0},
            "valid": {"x": "y" * 600}, "closure": {"x": "y" * 600}, "batch32": [1, 2, 3]}
    out = bench.fit_line(line, limit=400)
    assert len(json.dumps(out, separators=(",", ":"))) <= 400
    assert {"metric", "value", "unit", "roofline", "e2e"} <= set(out)
    assert "valid" not in out and "closure" not in out and out["batch32"] == [1, 2, 3]
    assert bench.fit_line({"metric": "m"}, limit=400) == {"metric": "m"}
