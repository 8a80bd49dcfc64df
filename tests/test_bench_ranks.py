"""The benchmark's multi-rank path on CPU: two gloo ranks (spawned processes)
combine their timings by the slowest rank, report the whole job's rate, and
only rank 0 runs and prints the oracle reference arm."""
import contextlib
import io
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world)})
    sys.path.insert(0, ROOT)
    import argparse

    import bench
    r, ws, local, dist = bench.dist_setup()
    res = {"rank": r, "world": ws, "backend": dist.get_backend()}
    # every rank brings its own time; the job is as fast as its slowest rank
    mine = 1.0 + rank
    slowest = bench.max_over_ranks(mine, dist)
    res["slowest"] = slowest
    res["rate"] = bench.whole_job_rate(1000, 10, ws, slowest)
    dist.barrier()
    dist.destroy_process_group()
    # the reference arm: rank 0 alone runs the oracle and prints one line
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        rc = bench.run_reference(argparse.Namespace(steps=1, warmup=0, gpus=ws))
    res["ref_rc"] = rc
    res["ref_out"] = buf.getvalue()
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump(res, f)


def test_two_gloo_ranks_combine_by_the_slowest_rank(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(2)]
    for r, d in enumerate(res):
        assert d["rank"] == r and d["world"] == 2 and d["backend"] == "gloo"
        assert d["slowest"] == 2.0  # rank 1's time
        assert d["rate"] == pytest.approx(1000 * 10 * 2 / 2.0)
        assert d["ref_rc"] == 0
    # one JSON line from rank 0, nothing from rank 1
    lines = [l for l in res[0]["ref_out"].splitlines() if l.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert res[1]["ref_out"] == ""


def test_tissue_partition_balances_and_covers_every_tissue():
    sys.path.insert(0, ROOT)
    import bench
    from paper_1605_06015_gb300 import workloads as wl
    cells = [w.n_cells for w in wl.tissue_batch()]
    for n in (1, 2, 3, 8):
        parts = bench.partition_tissues(cells, n)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(cells)))  # every tissue on exactly one rank
        loads = [sum(cells[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(cells)  # greedy bound: within one tissue
