"""The N > 1 path of bench.py (replicas): two gloo ranks on CPU agree on
the slowest rank's time, the whole-job rate counts every rank's work, ranks
draw distinct seeds, and only rank 0 prints the reference arm's line."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank            # rank 1 is the slower one
        ms = bench.max_over_ranks(local_ms, world)
        out[rank] = (ms, bench.job_rate(world, 3, 300, ms), bench.rank_seed(rank))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest():
    world, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    assert res[0][1] == res[1][1] == pytest.approx(2 * 3 * 300 / 0.015)
    assert res[0][2] != res[1][2]


def test_one_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_rate(1, 2, 100, 20.0) == pytest.approx(10000.0)


def test_reference_arm_prints_on_rank_0_only(capsys):
    import bench
    saved = sys.argv
    sys.argv = ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"]
    try:
        args = bench.parse()
    finally:
        sys.argv = saved
    assert bench.run_reference(args, rank=1, world=2) is None
    assert capsys.readouterr().out == ""


def test_reference_arm_line_keeps_the_contract(capsys):
    """rank 0 of --impl reference times the FP64 oracle on the host (here the
    small line-scan workload, about a second of work) and prints one JSON line
    with the contract's keys: the oracle as cpu_baseline, an e2e with no
    copies, and the same metric and unit as the GPU arm."""
    import json
    import bench
    saved = sys.argv
    sys.argv = ["bench.py", "--impl", "reference", "--workload", "line2d", "--steps", "2",
                "--warmup", "1", "--cpu-seconds", "1"]
    try:
        args = bench.parse()
    finally:
        sys.argv = saved
    bench.run_reference(args, rank=0, world=1)
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and "unavailable" not in d
    assert d["metric"] == "FISTA iterations/s" and d["unit"] == "it/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1
    assert d["ms_per_step"] > 0 and d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["config"]["workload"].startswith("line2d")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "it/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
