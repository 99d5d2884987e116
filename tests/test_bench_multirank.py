"""Host logic of the multi-process benchmark on the CPU: the max-over-ranks reduction with
two gloo ranks, and the reference arm under torchrun (rank 0 alone prints one line)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    got = bench.reduce_max(10.0 + 3.0 * rank, "cpu")
    with open(f"{out_path}.{rank}", "w") as f:
        f.write(repr(got))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "r")
    mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    assert [float(open(f"{out}.{r}").read()) for r in range(2)] == [13.0, 13.0]


def test_reference_arm_under_torchrun():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3", "--mesh-m", "3"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["cores"] == max(1, min(64, len(os.sched_getaffinity(0))))


def test_kernel_hash_ignores_comments_not_code():
    """The traffic record is tied to the residual kernel's code: comment and layout edits
    keep the hash, code edits change it."""
    import bench
    src = {f: open(os.path.join(ROOT, "paper_2312_07874_gb300", "csrc", f)).read() for f in bench.KERNEL_SOURCES}
    base = bench._kernel_hash(lambda f: src[f])
    commented = dict(src)
    commented["device.cuh"] = "// a new comment\n" + src["device.cuh"].replace("\n", "  \n", 3) + "\n/* end\n */\n"
    assert bench._kernel_hash(lambda f: commented[f]) == base
    edited = dict(src)
    edited["device.cuh"] = src["device.cuh"].replace("0.5", "0.25", 1)
    assert edited["device.cuh"] != src["device.cuh"]
    assert bench._kernel_hash(lambda f: edited[f]) != base


def test_cpu_baseline_all_cores_small_mesh(monkeypatch):
    """The all-core oracle baseline forks one worker per core on distinct element blocks
    (a 162-tetrahedron mesh here) and reports the cores it used."""
    import bench
    monkeypatch.setitem(bench.WORKLOAD, "M", 3)
    monkeypatch.setattr(bench, "_ORACLE", {})
    out = bench.cpu_baseline_all_cores(n_el=4)
    cores = max(1, min(64, len(os.sched_getaffinity(0))))
    assert out["cores"] == cores and out["kind"] == "oracle" and out["value"] > 0
    assert out["unit"] == bench.UNIT
    assert f"{cores} forked workers x {max(1, min(4, 162 // cores))} distinct elements" in out["sample"]
