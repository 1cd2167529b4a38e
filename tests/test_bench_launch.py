"""bench.py's multi-rank launch on the CPU: `--gpus 2` outside a launcher starts
two ranks (torch.distributed.run on 127.0.0.1), each with its own pairs (weak
scaling), and rank 0 prints one line for the whole job.  `--dry-run` uses gloo
and does no GPU work."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*argv):
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *argv], cwd=ROOT, env=env,
                         capture_output=True, text=True, timeout=240)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, res.stdout
    return json.loads(lines[0])


@pytest.mark.timeout(300)
def test_two_ranks_each_with_own_pairs():
    out = _run("--gpus", "2", "--dry-run", "--pairs-per-class", "1")
    assert out["n_gpus"] == 2 and out["backend"] == "gloo"
    assert out["pairs_per_rank"] == [4, 4]
    assert out["first_pair_digest"][0] != out["first_pair_digest"][1]


@pytest.mark.timeout(300)
def test_one_rank_default():
    out = _run("--dry-run", "--pairs-per-class", "1")
    assert out["n_gpus"] == 1 and out["pairs_per_rank"] == [4]
