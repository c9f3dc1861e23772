"""The multi-GPU path is replicas only (tiles and images are independent; no
data-path collective).  What it adds on the host is tested here with two
`gloo` ranks on CPU: disjoint inputs per rank, the slowest replica's time as
the job's time, whole-job throughput, and the reference arm running on rank 0
only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as d
    import bench
    d.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                         world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank
        job_ms = bench.max_over_ranks(local_ms, d, "cpu")
        value = bench.whole_job_value(1_000_000, 4, world, job_ms)
        out.put((rank, job_ms, value, bench.rank_seed(rank)))
        d.barrier()
    finally:
        d.destroy_process_group()


def test_two_replicas_take_the_slowest_time_and_sum_the_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (r0, ms0, v0, s0), (r1, ms1, v1, s1) = res
    assert ms0 == ms1 == 15.0                      # the slower replica
    assert v0 == v1 == pytest.approx(2 * 4 * 1e6 / 15e-3 / 1e6)
    assert s0 != s1 and s0 == 2                    # disjoint inputs, rank 0 = benchmark scene


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    args = argparse.Namespace(steps=1, warmup=3)
    bench.run_reference(args, rank=1, world=2)
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_rank_zero(capsys, monkeypatch):
    """Rank 0 prints one JSON line with the base contract's keys, the oracle
    as the reference implementation, and zero host-device bytes."""
    import argparse
    import json
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("MHFD_REF_SIDE", "128")
    bench.run_reference(argparse.Namespace(steps=2, warmup=1), rank=0, world=1)
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == d["unit"] == bench.METRIC
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 2
    assert d["n_gpus"] == 1 and d["config"]["workload"] == bench.WORKLOAD
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": bench.METRIC, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
