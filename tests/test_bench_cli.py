"""bench.py's command line on the host: the reference arm's other ranks exit
0 without work, and workloads that run on one GPU, or that the reference arm
does not time, are refused instead of silently running something else."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, **env):
    e = dict(os.environ)
    e.update(env)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=e,
                          capture_output=True, text=True, timeout=120)


def test_reference_arm_other_ranks_exit_without_work():
    r = _run(["--impl", "reference", "--gpus", "2"], RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_refuses_other_workloads():
    r = _run(["--impl", "reference", "--workload", "ising10"])
    assert r.returncode != 0 and "cpu_baseline" in r.stderr


def test_single_gpu_workloads_refuse_torchrun():
    r = _run(["--workload", "smesolve_jc", "--gpus", "2"], RANK="0", LOCAL_RANK="0", WORLD_SIZE="2")
    assert r.returncode != 0 and "one GPU" in r.stderr


@pytest.mark.parametrize("workload", ["steadystate", "dsf", "dsf_mc"])
def test_newer_workloads_are_accepted_and_routed(workload):
    """The stationary-state and DSF workloads parse, refuse torchrun (one
    GPU each) and refuse the reference arm (their lines carry the oracle's
    timing in cpu_baseline)."""
    r = _run(["--workload", workload, "--gpus", "2"], RANK="0", LOCAL_RANK="0", WORLD_SIZE="2")
    assert r.returncode != 0 and "one GPU" in r.stderr
    r = _run(["--impl", "reference", "--workload", workload])
    assert r.returncode != 0 and "cpu_baseline" in r.stderr
