"""The benchmark's multi-GPU launcher on CPU: `bench.py --gpus 2` with no
WORLD_SIZE in the environment spawns two ranks itself; with the gloo backend
(no GPU here) they take their channel blocks through the shard helper, reduce
the step time to the slowest rank's, and rank 0 alone prints the line.  The
same code path (spawn_ranks -> rank_setup -> max_over_ranks) runs the NCCL
ranks on a GPU node; torchrun-launched ranks skip the spawn."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env_extra=None):
    env = {k: v for k, v in os.environ.items()
           if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT")}
    env["CUDA_VISIBLE_DEVICES"] = ""
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True,
                       text=True, timeout=240, env=env, cwd=ROOT)
    return r


@pytest.mark.parametrize("n", [2, 3])
def test_spawned_ranks_report_the_slowest_and_cover_the_channels(n):
    r = _run(["--launcher-selftest", "--gpus", str(n)])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(s) for s in r.stdout.splitlines() if s.startswith("{")]
    assert len(lines) == 1, r.stdout  # rank 0 only
    line = lines[0]
    assert line["n_gpus"] == n and line["launcher"] == "spawn" and line["scaling"] == "weak"
    assert line["ms_per_step"] == 10.0 + (n - 1)      # rank r reports 10 + r ms
    blocks = [tuple(b) for b in line["shards"]]
    assert blocks == [(64 * r, 64 * (r + 1)) for r in range(n)]


def test_world_size_must_match_gpus():
    r = _run(["--launcher-selftest", "--gpus", "2"], {"WORLD_SIZE": "1", "RANK": "0"})
    assert r.returncode != 0 and "WORLD_SIZE" in r.stderr
