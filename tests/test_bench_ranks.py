"""bench.py is single-GPU only: a multi-GPU request (--gpus N > 1 or a
torchrun environment with WORLD_SIZE > 1) prints one "unavailable" line and
does no GPU work. Runs on the CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env_extra):
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, env=env,
                       capture_output=True, text=True, timeout=120)
    return r


def test_gpus_flag_above_one_is_refused():
    r = _run(["--gpus", "2"], {"RANK": "0", "WORLD_SIZE": "1"})
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["n_gpus"] == 2 and "single-GPU" in d["unavailable"]


def test_torchrun_world_above_one_is_refused_and_only_rank0_prints():
    r0 = _run([], {"RANK": "0", "WORLD_SIZE": "4", "LOCAL_RANK": "0"})
    r1 = _run([], {"RANK": "1", "WORLD_SIZE": "4", "LOCAL_RANK": "1"})
    assert r0.returncode == 0 and r1.returncode == 0
    assert json.loads(r0.stdout.strip())["n_gpus"] == 4
    assert r1.stdout.strip() == ""


def test_single_gpu_is_not_refused():
    sys.path.insert(0, ROOT)
    import bench

    class A:
        gpus = 1
    old = {k: os.environ.pop(k, None) for k in ("WORLD_SIZE", "RANK")}
    try:
        assert not bench.multi_gpu_requested(A())
    finally:
        for k, v in old.items():
            if v is not None:
                os.environ[k] = v
