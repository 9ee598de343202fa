"""The benchmark's reference arm (the oracle timed on the host cores) runs without a GPU and
prints one JSON line with the keys of the bench contract: metric, unit and direction of the
GPU arm, the per-step sample it timed, the cores it used, and an end-to-end entry with no
host-device traffic."""
import json
import os
import subprocess
import sys

from conftest import ROOT


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["unit"] == "Gsamples/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["vs_baseline"] is None and d["data"] == "synthetic"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_reference_arm_under_torchrun_prints_from_rank_0_only():
    """Launched as the multi-GPU bench is (torchrun, two ranks on 127.0.0.1), the reference arm
    runs on rank 0 alone: exactly one JSON line, every rank exits 0."""
    import socket

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                          "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
                          "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2


def test_clock_sampler_child_never_outlives_the_bench(monkeypatch, tmp_path):
    """The clock sampler's child process (nvidia-smi on a GPU machine; a stand-in here) is ended by
    stop(), and by the exit handler start() registers if stop() is never reached."""
    import atexit

    import bench

    real_popen = subprocess.Popen
    monkeypatch.setattr(bench.subprocess, "Popen",
                        lambda args, **kw: real_popen(["sleep", "60"], **kw))
    monkeypatch.setenv("PRNGD_CLOCKS_DIR", str(tmp_path))
    registered = []
    monkeypatch.setattr(atexit, "register", lambda f: registered.append(f))
    monkeypatch.setattr(atexit, "unregister", lambda f: None)
    a = bench.ClockSampler(0)
    a.start()
    assert a.proc.poll() is None and len(registered) == 1
    registered[0]()  # what interpreter exit would run after an exception in the timed region
    assert a.proc.poll() is not None
    b = bench.ClockSampler(0)
    b.start()
    res = b.stop()
    assert b.proc.poll() is not None and res["samples"] == 0
