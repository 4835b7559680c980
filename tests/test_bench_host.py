"""Host-side pieces of bench.py: the multi-rank (replica) plumbing on gloo, the
reference arm's JSON line, and the parsers of clocks and committed ncu figures."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    r, w, _ = bench.dist_setup(world)
    bench.barrier(w)
    q.put((r, bench.max_over_ranks(1.5 + r, w)))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 2.5), (1, 2.5)]


def test_reference_arm_single_rank_json():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "3",
                          "--warmup", "1"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["value"] > 0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == cores
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["higher_is_better"] is True
    # the same metric and workload as the GPU arm, so that the two lines compare
    sys.path.insert(0, ROOT)
    import bench
    assert d["metric"] == bench.METRIC
    assert d["config"]["workload"] == bench.workload("tgv8192", 0)["desc"]


def test_reference_arm_under_torchrun_world2():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "1"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1                         # rank 0 alone prints
    assert json.loads(lines[0])["n_gpus"] == 2


def test_clock_sampler_parses_nvidia_smi_lines():
    s = bench.ClockSampler(0)

    class Fake:
        def terminate(self):
            pass

        def communicate(self, timeout=None):
            return ("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                    "0, 1980, 2070, 1300.5, 0x4, Not Active, Not Active, Not Active, Active\n"
                    "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active\n", "")

    s.proc = Fake()
    c = s.stop()
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"] and c["samples"] == 3


def test_committed_traffic_requires_current_sources(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (tmp_path / "paper_2409_01076_gb300").symlink_to(os.path.join(ROOT, "paper_2409_01076_gb300"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_source_hash()
    (prof / "step_kernel_traffic.md").write_text(
        "source_hash: %s\ntraffic_bytes_per_node[f32-ab-smrt]: 72.9\n" % h)
    assert bench.committed_traffic("f32", "ab", "smrt")[0] == 72.9
    assert bench.committed_traffic("f16", "ab", "smrt")[0] is None
    (prof / "step_kernel_traffic.md").write_text(
        "source_hash: deadbeef\ntraffic_bytes_per_node[f32-ab-smrt]: 72.9\n")
    assert bench.committed_traffic("f32", "ab", "smrt")[0] is None


def test_workloads_match_the_stated_configs():
    t = bench.workload("tgv8192")
    assert (t["nx"], t["ny"], t["tau"], t["u0"]) == (8192, 8192, 0.51, 0.05)
    c = bench.workload("cavity4096")
    assert c["nx"] == 4096 and abs(c["tau"] - (3 * 0.1 * 4096 / 1e4 + 0.5)) < 1e-15
