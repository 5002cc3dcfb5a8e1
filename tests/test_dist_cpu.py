"""Host logic of bench.py's multi-process path, on CPU with gloo, world size 2:
the max-over-ranks timing and sum-over-ranks work behind the whole-job
value, and the reference arm under torchrun (rank 0 alone prints one line,
the other rank exits 0 without work)."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist, w, r, _ = bench.dist_setup("gloo")
    # per-rank step time and work of a weak-scaling run
    ms = 10.0 + 5.0 * r
    pairs = 1000.0 * (r + 1)
    t_max = bench.max_over_ranks(dist, w, ms)
    p_sum = bench.sum_over_ranks(dist, w, pairs)
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump({"world": w, "t_max": t_max, "p_sum": p_sum, "value": p_sum / (t_max * 1e-3)}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_rank_reductions_gloo(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for d in res:
        assert d["world"] == 2
        assert d["t_max"] == 15.0          # the slowest rank sets the time
        assert d["p_sum"] == 3000.0        # the work of all ranks
        assert d["value"] == pytest.approx(3000.0 / 0.015)


def test_reference_arm_under_torchrun():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "pair-evals/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
