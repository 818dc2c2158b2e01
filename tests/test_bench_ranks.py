"""The multi-rank logic of bench.py, on CPU: the job time is the slowest
rank's (max over a world_size-2 gloo group), the job value counts every
rank's units, and every rank renders its own camera of the same scene
(weak scaling, no collective on the data path)."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 * (rank + 1) + 0.25
        m = bench.max_over_ranks(local_ms, dist, "cpu")
        v = bench.job_throughput(world, 4, 1.696, m)
        dist.barrier()
        q.put((rank, m, v))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        r, m, v = q.get(timeout=120)
        res[r] = (m, v)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1]
    m, v = res[0]
    assert m == 20.25
    assert abs(v - 2 * 4 * 1.696 / 0.02025) < 1e-9


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_throughput(1, 20, 1.696, 1000.0) == 20 * 1.696


def test_each_rank_renders_its_own_camera_of_the_same_scene():
    w0, w1 = bench.workload(0, 2000), bench.workload(1, 2000)
    assert np.array_equal(w0.scenes[0].params, w1.scenes[0].params)
    v0, v1 = w0.views[0], w1.views[0]
    assert (v0.width, v0.height) == (v1.width, v1.height) == (1600, 1060)
    assert not np.allclose(v0.R, v1.R)  # another camera on the same radius-8 sphere


def test_reference_arm_prints_one_line_on_rank_zero_only():
    """``bench.py --impl reference`` times the oracle on the host cores and
    prints the bench line with ``impl: reference``; under torchrun the other
    ranks return without work."""
    import json
    import subprocess
    import sys

    assert bench.bench_reference(None, 1, 2) is None
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1",
                        "--primitives", "20000"], cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["metric"] == bench.METRIC and out["unit"] == "MP/s"
    assert out["value"] > 0 and out["steps"] == 1 and out["warmup"] == 1 and out["higher_is_better"] is True
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["value"] == out["value"]
    assert out["e2e"] == {"value": out["value"], "unit": "MP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert out["config"]["workload"] == "static_n3_1m_1600x1060"


def test_our_arm_fails_loudly_without_a_gpu():
    """No CPU fallback: without a CUDA device the bench exits non-zero and
    prints no result line."""
    import subprocess
    import sys

    import pytest
    import torch

    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--no-cpu-baseline", "--no-batched", "--steps", "1", "--warmup", "3"],
                       cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0
    assert '"value"' not in r.stdout


def test_traffic_figures_come_from_the_committed_profiles(monkeypatch):
    """The roofline's DRAM traffic is read from the committed ncu summaries,
    and only while the kernel's source is the one that was captured."""
    for kernel in ("render_bwd_blend", "render_fwd"):
        b = bench.traffic_record(kernel)
        assert b is None or b > 0
    assert bench.traffic_record("no_such_kernel") is None
    monkeypatch.setattr(bench, "source_sha", lambda path: "0" * 16)
    assert bench.traffic_record("render_bwd_blend") is None
