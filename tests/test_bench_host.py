"""Host-side pieces of bench.py: the replica aggregation over a 2-rank gloo group, the
kernel-hash gate of the profiled traffic, and the reference arm's JSON line."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench

    dist = bench._init_dist(world)
    bench._barrier(dist)
    m = bench._max_over_ranks(dist, 10.0 + 5.0 * rank)
    q.put((rank, m))
    dist.destroy_process_group()


def test_replica_timing_takes_the_max_over_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 15.0), (1, 15.0)]


def test_traffic_gate_follows_the_kernel_source(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    h = bench.kernel_source_hash()
    monkeypatch.setattr(bench, "STEP_TRAFFIC", {"kernel_source_sha256": h,
                                                "dram_bytes_per_launch": 123})
    assert bench.profiled_traffic() == 123
    monkeypatch.setattr(bench, "STEP_TRAFFIC", {"kernel_source_sha256": "0000",
                                                "dram_bytes_per_launch": 123})
    assert bench.profiled_traffic() is None


def test_bench_reads_no_profile_files():
    """The emitted line is built from measurements and constants, never from profiles/."""
    with open(os.path.join(ROOT, "bench.py")) as fh:
        src = fh.read()
    assert "profiles/" not in src


def test_window_count_covers_a_second_and_five_windows():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.window_count(1000.0) == bench.MIN_WINDOWS  # long windows: five of them
    assert bench.window_count(0.78) == 1283                  # 20 channel steps: >= 1 s in all
    assert bench.window_count(1e-9) == bench.MAX_WINDOWS


def test_reference_arm_prints_one_json_line():
    env = dict(os.environ, OMP_NUM_THREADS="4")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "3"], capture_output=True, text=True,
                       env=env, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["higher_is_better"] is True
