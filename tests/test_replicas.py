"""Host logic of bench.py's multi-replica path (one process per GPU under
torchrun, independent problems, no data-path collective), run as two gloo
ranks on the CPU: the whole-job totals (slowest rank's time, sum of the units)
and the reference arm, which rank 0 alone runs and prints."""
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str) -> None:
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    w, r, loc, pg = bench.dist_setup()
    assert (w, r, loc) == (world, rank, rank) and pg is not None
    # rank r processes 100 (r + 1) units in 2 + r seconds
    t, u = bench.job_totals(pg, 2.0 + rank, 100 * (rank + 1))
    m = bench.max_over_ranks(pg, float(10 - rank))
    bench.barrier(pg)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"time": t, "units": u, "max": m}, f)
    pg.destroy_process_group()


def test_job_totals_one_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_totals(None, 1.5, 7) == (1.5, 7)
    assert bench.max_over_ranks(None, 3.0) == 3.0


def test_job_totals_two_gloo_ranks(tmp_path):
    mp.start_processes(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    for rank in range(2):
        with open(tmp_path / f"rank{rank}.json") as f:
            d = json.load(f)
        # every rank sees the slowest rank's time and the units of both
        assert d == {"time": 3.0, "units": 300.0, "max": 10.0}


def test_reference_arm_under_torchrun():
    """The launch the two-GPU bench uses, with the reference arm on the 12^3
    cell: exactly one JSON line (rank 0's), and rank 1 exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference", "--gpus", "2",
           "--steps", "2", "--warmup", "1", "--workload", "tiny_cubic"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
