"""bench.py --gpus N starts N ranks itself (torch.distributed.run) and splits
the batched workload over them; checked with the CPU dry run (gloo, no GPU
work), where the JSON line must report n_gpus == N and shares that cover
every batch image exactly once."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_dry(n):
    env = dict(os.environ)
    env.pop("WORLD_SIZE", None)
    env.pop("RANK", None)
    env.pop("LOCAL_RANK", None)
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", str(n), "--dry-run"],
                       capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, p.stdout
    return json.loads(lines[0])


def test_two_rank_dry_run_reports_both_ranks_and_a_full_split():
    d = run_dry(2)
    assert d["dry_run"] and d["n_gpus"] == 2 == d["gpus_requested"]
    flat = sorted(i for share in d["batch_shares"] for i in share)
    assert flat == list(range(64))
    assert all(len(s) > 0 for s in d["batch_shares"])


def test_engine_traffic_is_read_from_the_committed_capture():
    sys.path.insert(0, ROOT)
    import bench

    traffic, note = bench.engine_traffic()
    with open(bench.ENGINE_PROFILE) as f:
        text = f.read()
    assert "traffic_bytes_per_launch:" in text and "sources_digest:" in text
    if "sources" in note and "changed" not in note:
        assert traffic and traffic > 0
    else:
        assert traffic is None  # stale capture: reported as null, with the reason
