"""The benchmark's multi-process path on CPU (gloo, world size 2): rank
set-up from the launcher's environment, the max over ranks of the step time,
the barrier, and the reference arm under torchrun (rank 0 alone runs and
prints; the other rank exits 0 without work)."""
import json
import os
import socket
import subprocess
import sys
import types

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    w, r, local = bench.dist_setup(types.SimpleNamespace(impl="reference"))
    step_ms = 1.0 + 0.5 * r  # rank 1 is the slow one
    worst = bench.max_over_ranks(step_ms, w)
    bench.barrier(w)
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump({"world": w, "rank": r, "local": local, "backend": dist.get_backend(), "max": worst}, f)
    dist.destroy_process_group()


def test_rank_helpers_gloo(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r, g in enumerate(got):
        assert g["world"] == world and g["rank"] == r and g["local"] == r
        assert g["backend"] == "gloo"
        assert g["max"] == pytest.approx(1.5)  # every rank reports the slowest rank's time


def test_reference_arm_under_torchrun():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0",  # the driver's own form of the call,
           "--gaussians", "30000"]  # a smaller scene: every oracle step is a whole step
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout  # rank 0 alone prints
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2
    assert out["value"] > 0 and out["e2e"]["value"] == out["value"]
    assert out["cpu_baseline"]["kind"] == "oracle-binned" and out["cpu_baseline"]["extrapolated"] is False
    assert out["steps"] == out["measured_steps"] == 1
