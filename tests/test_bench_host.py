"""Host logic of bench.py's multi-replica form (replicas only: each rank codes
its own copy of the workload, and the only exchange is the max of the timed
regions).  Two gloo ranks on the CPU stand in for two GPUs."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def test_one_rank_keeps_its_time_and_scales_by_its_pixels():
    assert bench.max_over_ranks(2.5, None, "cpu") == 2.5
    # 3 qualities x 2048 x 1536 pixels per step, 20 steps in 200 ms
    assert bench.job_mpx_per_s(1, 3 * 2048 * 1536, 20, 200.0) == pytest.approx(943.7184)


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = bench.max_over_ranks(times[rank], dist, "cpu")
        out.put((rank, ms, bench.job_mpx_per_s(world, 1000, 4, ms)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_report_the_slowest_time_and_the_whole_job_throughput(world):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    times = [5.0 + 1.5 * r for r in range(world)][::-1]   # rank 0 is the slowest
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, times, out)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slowest = max(times)
    assert [g[0] for g in got] == list(range(world))
    for _, ms, value in got:
        assert ms == slowest
        # all ranks' pixels over the slowest rank's time
        assert value == pytest.approx(world * 1000 * 4 / (slowest / 1e3) / 1e6)



def _run_bench(*argv, env=None):
    import json
    import subprocess
    import sys
    e = dict(os.environ)
    e.update(env or {})
    p = subprocess.run([sys.executable, os.path.join(os.path.dirname(bench.__file__), "bench.py"), *argv],
                       capture_output=True, text=True, timeout=600, env=e)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    return [json.loads(ln) for ln in lines]


@pytest.mark.slow
def test_reference_arm_prints_one_line_of_the_contract():
    """`--impl reference` times the CPU oracle on the bench workload (the
    7680x4320 image, one band per host core): one JSON line with the same
    metric and unit, its own cpu_baseline and an e2e object without
    host-device copies."""
    (line,) = _run_bench("--impl", "reference", "--steps", "1", "--warmup", "0")
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["higher_is_better"] is True and line["bit_exact"] is True and line["value"] > 0
    assert line["config"]["pixels_per_step"] == 7680 * 4320
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == min(bench.host_cores(), 540) and cb["value"] == line["value"]
    assert cb["sample"] and cb["cpu_model"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_runs_on_rank_zero_only():
    assert _run_bench("--impl", "reference", "--steps", "1", "--warmup", "0", env={"RANK": "1"}) == []


def test_image_bands_cover_every_row_once():
    import numpy as np
    img = np.arange(4320 * 16, dtype=np.uint32).reshape(4320, 16)
    for parts in (1, 7, 16, 72):
        bands = bench.image_bands(img, parts)
        assert len(bands) == parts
        assert all(b.shape[0] >= 8 and b.flags["C_CONTIGUOUS"] for b in bands)
        assert np.array_equal(np.concatenate(bands), img)
    # never a band under 8 rows
    assert len(bench.image_bands(img[:20], 16)) == 2
    assert len(bench.image_bands(img[:5], 16)) == 1


def test_cpu_model_and_cores_are_reported():
    assert isinstance(bench.cpu_model(), str) and bench.cpu_model()
    assert bench.host_cores() >= 1
