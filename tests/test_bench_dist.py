"""Host logic of the multi-GPU bench path, run as two gloo ranks on the CPU.

Every rank labels its own copy of the workload (replicas: no collective on the
data path); the only collectives are the timing barrier and the maximum over
ranks of the timed region, from which rank 0 reports the whole-job rate.  The
reference arm runs on rank 0 alone.
"""
import contextlib
import io
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got_ws, got_rank, got_local = bench._dist()
        dist.barrier()
        own_ms = 10.0 + 7.5 * rank            # the slower rank sets the job's time
        total = bench._max_over_ranks(dist, own_ms, "cpu")
        dist.barrier()
        rate = bench._job_rate(ws, 1_000_000, 4, total)
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump(dict(ws=got_ws, rank=got_rank, local=got_local, own=own_ms,
                           total=total, rate=rate), f)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    ws = 2
    mp.start_processes(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws,
                       join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(ws)]
    slowest = max(r["own"] for r in res)
    for r, x in enumerate(res):
        assert (x["ws"], x["rank"], x["local"]) == (ws, r, r)
        assert x["total"] == slowest                       # every rank sees the max
        # whole job: voxels of all ranks over the slowest rank's time
        assert x["rate"] == pytest.approx(ws * 1_000_000 * 4 / (slowest * 1e-3) / 1e9)


def test_single_process_needs_no_collective():
    assert bench._max_over_ranks(None, 12.5, "cpu") == 12.5
    assert bench._job_rate(1, 2_000_000, 10, 20.0) == pytest.approx(1.0)


def test_reference_arm_runs_on_rank_zero_only():
    class A:
        steps, warmup, workload = 1, 0, "voronoi-64^3-periodic-100"
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(A, bench._workloads()[A.workload](), ws=2, rank=1)
    assert buf.getvalue() == ""                            # other ranks exit without work


def test_reference_arm_line_on_rank_zero():
    """Rank 0 prints the contract's line for the oracle arm: the metric, a
    positive rate, and a cpu_baseline naming its kind, cores and CPU model."""
    class A:
        steps, warmup, workload = 1, 0, "voronoi-64^3-periodic-100"
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(A, bench._workloads()[A.workload](), ws=1, rank=0)
    line = json.loads(buf.getvalue())
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["value"] > 0 and line["unit"] == "Gvoxel/s" and line["steps"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["cpu_model"] and cb["sample"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
