"""bench.py's multi-process path on CPU (gloo, world size 2). The analysis does
not shard: `bench.py --gpus N` runs N independent replicas, each on its own
synthetic instance, and reports the whole-job throughput N * steps / (slowest
rank's time). These tests run that host logic in two processes without a GPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, steps, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        agg = bench.combine(times[rank], steps, world, bench.make_reduce_max(world, "cpu"))
        w = bench.workload(rank)
        # every rank sees the same aggregate; the seeds of its instance are its own
        got = torch.tensor([agg["value"], agg["max_total_s"], float(w.seeds[0])],
                           dtype=torch.float64)
        gathered = [torch.zeros(3, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(gathered, got)
        if rank == 0:
            out.put([g.tolist() for g in gathered])
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_job_throughput_over_the_slowest_rank():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    times, steps = [0.40, 0.55], 100
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, steps, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = out.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for value, tmax, _ in res:
        assert tmax == max(times)
        assert value == pytest.approx(2 * steps / max(times), rel=1e-12)
    assert res[0][2] != res[1][2]          # distinct instances per replica


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    agg = bench.combine(0.25, 50, 1, bench.make_reduce_max(1, "cpu"))
    assert agg["value"] == pytest.approx(200.0)
    assert agg["ms_per_step"] == pytest.approx(5.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"]) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_prints_the_contract_line(monkeypatch, capsys):
    """`bench.py --impl reference` (the oracle timed on the host cores) prints
    one JSON line with the keys the bench contract names."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.delenv("RANK", raising=False)
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"]) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "frames/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("elt-80x80")
