"""The replica path of bench.py under several ranks, on CPU with gloo.

Every rank factors its own matrix (weak scaling, no collective on the data
path); the only cross-rank steps are the timing barrier and the max-over-
ranks of the measured time.  These run here with world_size 2 on the gloo
backend; the reference arm prints from rank 0 only.
"""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = 100.0 + 50.0 * rank          # rank 1 is the slow one
    t = bench.max_over_ranks(mine, device="cpu")
    dist.barrier()
    v = bench.job_throughput(8.0e9, 4, t, world)
    q.put((rank, t, v))
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo():
    world, port = 2, 29517
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    out = sorted(q.get(timeout=10) for _ in range(world))
    for rank, t, v in out:
        assert t == 150.0                     # slowest rank's time on every rank
        assert abs(v - 2 * 8.0e9 * 4 / 0.150 / 1e9) < 1e-9
    assert out[0][2] == out[1][2]


def test_single_process_identity():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_throughput(1e9, 2, 1000.0, 1) == 2.0


def test_reference_arm_only_rank0_prints():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], capture_output=True, text=True, env=env,
                       timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_reference_arm_prints_one_contract_line():
    # rank 0 alone: the oracle timed on the host cores, one JSON line whose
    # value is the 2 m n^2 model of the four factorizations of the row
    # sample divided by the mean step time
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], capture_output=True, text=True, env=env,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3
    assert d["higher_is_better"] is True and d["unit"] == "GFLOP/s" and d["dtype"] == "f64"
    assert d["config"]["workload"] and d["config"]["m"] == 1 << 20 and d["config"]["n"] == 128
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == d["value"] == d["e2e"]["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    model = 4 * 2.0 * 32768 * 128 ** 2  # four factorizations of the 32768-row sample
    assert abs(d["value"] * 1e9 * d["ms_per_step"] * 1e-3 - model) <= 1e-9 * model
