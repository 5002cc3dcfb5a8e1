"""Host logic of the X-row shards of one registration, on CPU with gloo at
world size 2 (no GPU): the row partition covers every row of X exactly once,
and the shard loop of register_sharded sums every iteration's statistics
over the ranks before the step, so that both ranks take the same steps and
stop together.  The library's four shard calls are replaced by CPU stand-ins
here (the GPU test of the same loop is tests/test_gpu_shard.py)."""
import json
import os
import socket
import sys

import numpy as np
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


def test_shard_rows_partition_single_process():
    import paper_2012_03683_gb300 as cvo
    for n in (0, 1, 7, 64, 200000, 200003):
        for world in (1, 2, 3, 8):
            rows = [cvo.shard_rows(n, world, r) for r in range(world)]
            assert rows[0][0] == 0 and rows[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))
            sizes = [hi - lo for lo, hi in rows]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        cvo.shard_rows(10, 2, 2)


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import paper_2012_03683_gb300 as cvo
    dist.init_process_group("gloo")
    n = 1001
    lo, hi = cvo.shard_rows(n, world, rank)
    # every row exactly once over the ranks
    mine = torch.zeros(n, dtype=torch.int64)
    mine[lo:hi] = 1
    dist.all_reduce(mine)
    # per-row statistics of a stand-in sweep: row i contributes f_k(i, it)
    rows = np.arange(n, dtype=np.float64)

    def contrib(idx, it):
        k = np.arange(cvo.SHARD_STATS, dtype=np.float64)
        return (np.cos(0.01 * np.outer(idx, k + 1) + it) * (1 + idx[:, None] % 7)).sum(axis=0)

    seen = []
    state = {"it": 0, "begun": None}

    def fake_begin(h, X_rows, Z, n_total, T_init, FX_rows=None, FZ=None):
        state["begun"] = (len(X_rows), n_total)

    def fake_sweep(h, stats):
        stats.copy_(torch.from_numpy(contrib(rows[lo:hi], state["it"])))

    def fake_step(h, stats, wait=False):
        seen.append(stats.numpy().copy())
        state["it"] += 1
        done = stats[0].item() > 0.0 and state["it"] >= 5   # a decision taken from the summed statistics
        return done if wait else None

    def fake_end(h):
        return np.eye(4), {"iters": state["it"]}

    cvo.cvo_shard_begin, cvo.cvo_shard_sweep, cvo.cvo_shard_step, cvo.cvo_shard_end = (
        fake_begin, fake_sweep, fake_step, fake_end)
    stats = torch.zeros(cvo.SHARD_STATS, dtype=torch.float64)
    X_rows = np.zeros((hi - lo, 3), dtype=np.float32)
    T, info = cvo.register_sharded(None, X_rows, np.zeros((5, 3), np.float32), n, np.eye(4),
                                   allreduce=lambda t: dist.all_reduce(t), max_iters=12, check_every=1, stats=stats)
    full = [contrib(rows, it).tolist() for it in range(len(seen))]
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"cover": mine.tolist(), "rows": [lo, hi], "begun": state["begun"], "iters": info["iters"],
                   "seen": [s.tolist() for s in seen], "full": full}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_shard_loop_sums_statistics_over_ranks_gloo(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for d in res:
        assert d["cover"] == [1] * 1001                      # every row exactly once
        assert d["begun"][1] == 1001 and d["begun"][0] == d["rows"][1] - d["rows"][0]
        assert d["iters"] >= 5
        # what each step saw is the statistics of all rows, not the shard's
        np.testing.assert_allclose(d["seen"], d["full"], rtol=1e-12, atol=1e-9)
    # both ranks saw the same bits and stopped at the same iteration
    assert res[0]["seen"] == res[1]["seen"] and res[0]["iters"] == res[1]["iters"]
