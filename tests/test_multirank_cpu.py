"""The benchmark's multi-rank logic on CPU: world-size-2 gloo ranks.

The path has no exchange step (pairs are independent), so ranks are
replicas: each works on its own seeded pairs and the ranks meet only to take
the slowest rank's time. No GPU is used here.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank  # rank 1 is slower
    mx = bench.reduce_max_ms(ms, "cpu", world)
    value = bench.whole_job_pairs_per_s(128, 10, world, mx)
    first = bench.rank_first_pair(rank, 16)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, mx, value, first))


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [150.0, 150.0]
    assert res[0][2] == res[1][2] == pytest.approx(2 * 128 * 10 / 0.150)
    firsts = [r[3] for r in res]
    assert firsts == [0, 16]  # disjoint seeded pairs per rank


def test_reference_arm_runs_on_rank0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_recorded_traffic_only_for_the_source_it_was_taken_on(monkeypatch):
    """bench.py reports the search class's DRAM traffic from the committed
    counters only while csrc/search.cu is the source they were taken on;
    for any other source the roofline's traffic is null."""
    sys.path.insert(0, ROOT)
    import bench
    rec = json.load(open(os.path.join(ROOT, "profiles", "search_traffic.json")))["ps8"]
    monkeypatch.setattr(bench, "search_src_sha", lambda: rec["search_cu_sha256_16"])
    assert bench.recorded_traffic(8) == rec["dram_bytes_per_pair"]
    assert bench.recorded_traffic(12) is None  # no record for patch 12
    monkeypatch.setattr(bench, "search_src_sha", lambda: "0" * 16)
    assert bench.recorded_traffic(8) is None
