"""The benchmark's multi-rank logic on CPU ranks (gloo, world size 2): the
max-over-ranks time and the rank environment."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, l = bench.dist_env()
    t = bench.aggregate_max(1.5 + rank, w)
    bench.barrier(w)
    q.put((r, w, l, t))
    dist.destroy_process_group()


def test_aggregate_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 2, 0, 2.5), (1, 2, 1, 2.5)]


def test_single_rank_identity():
    import bench
    assert bench.aggregate_max(3.25, 1) == 3.25


def test_traffic_records_follow_kernel_sources(tmp_path, monkeypatch):
    """The roofline's DRAM traffic comes from committed ncu summaries only while
    the kernel's sources still hash to the recorded value, and a record is
    picked by kernel and workload."""
    import hashlib
    import json
    import shutil

    import bench
    root = tmp_path / "tree"
    csrc = root / "paper_1908_07847_gb300" / "csrc"
    shutil.copytree(os.path.join(bench.ROOT, "paper_1908_07847_gb300", "csrc"), csrc)
    (root / "profiles").mkdir()

    def record(kernel, workload, sources, nbytes):
        h = hashlib.sha256()
        for f in sources:
            h.update(open(csrc / f, "rb").read())
        return "traffic-record: " + json.dumps({"kernel": kernel, "workload": workload, "sources": sources,
                                                 "source_sha256_16": h.hexdigest()[:16],
                                                 "dram_bytes_per_launch": nbytes})

    src = ["fused_kernels.cu", "row_engine.cuh", "mlp_internal.cuh"]
    (root / "profiles" / "a.md").write_text("\n".join([
        "# summary", record("k_fused_train", "w1", src, 111), record("k_fused_train", "w2", src, 222),
        record("k_batched_train", "w3", ["batched_kernels.cu", "row_engine.cuh"], 333)]) + "\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.traffic_record("k_fused_train", "w1")["dram_bytes_per_launch"] == 111
    assert bench.traffic_record("k_fused_train", "w2")["dram_bytes_per_launch"] == 222
    assert bench.traffic_record("k_fused_train", "no such workload") is None
    assert bench.traffic_record("k_batched_train")["dram_bytes_per_launch"] == 333
    # the fused kernel's source changes by one byte: its records lapse, the
    # other kernel's stays
    with open(csrc / "fused_kernels.cu", "a") as f:
        f.write("\n")
    assert bench.traffic_record("k_fused_train", "w1") is None
    assert bench.traffic_record("k_batched_train") is not None


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the FP64 oracle on the host cores) runs
    without a GPU and prints one JSON line with the keys the benchmark
    contract asks of the reference arm."""
    import json
    import subprocess
    import sys

    import bench
    out = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=bench.ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "sample-steps/s"
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["gpu_launches"] == 0 and d["n_gpus"] == 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["config"] == bench.c2_config(1)


def test_reference_arm_under_torchrun_prints_once():
    """Launched the way the multi-GPU runs launch it (torchrun, two ranks),
    the reference arm runs on rank 0 only and prints one line; the other rank
    exits 0 without work."""
    import json
    import subprocess
    import sys

    import bench
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(_free_port()), os.path.join(bench.ROOT, "bench.py"), "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "1"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=bench.ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
