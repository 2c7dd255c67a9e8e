"""Training throughput of the one-hidden-layer sigmoid network (arXiv 1908.07847)
on one or more GB300s: train sample-steps/s (forward + backward + update).

Default workload (one line of JSON on rank 0): 4096 independent 33-H-1 sigmoid
networks, H ~ U{4..128} and n ~ U{50..120} rows each (the sex-split and
bootstrap sweeps of the paper's cohort, scaled up), 33 synthetic standardised
markers per row with teacher-net labels, trained by full-batch gradient descent
(lr 0.1, mean squared error, FP32) for 500 epochs.  One step is the whole
500-epoch run of all 4096 nets: one persistent kernel launch, captured once in
a CUDA graph and replayed.  Inputs stay resident in device memory; L2 is
flushed (256 MiB write) between timed steps, outside the timed intervals;
every step is timed with CUDA events on the launching stream.  `e2e` is the
same run through the host-buffer entry point (mlp_batch_run_host): rows,
labels and initial weights copied in, trained weights and loss histories
copied out, inside the timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload c0|c1|c2|c3|c4]

--impl reference times the FP64 CPU oracle on the host cores (the reference
arm of this benchmark: a plain serial program written from the paper) on a
bounded subset of the same workload.  With --gpus N > 1 (under torchrun) the
4096 x N nets are partitioned across the ranks by cost (longest processing
time first), every rank trains its share in one launch, and the trained
weights and loss histories are gathered to rank 0 inside the timed step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_ROWS, D_IN, H_HID, LR = 4096, 33, 64, 0.1
WORKLOAD = "33-64-1 sigmoid MLP, full-batch GD lr 0.1, 4096 rows x 33 features, FP32"
METRIC = "train sample-steps/s (fwd+bwd+update) vs plain FP32 path on 1 GB300; % roofline"
FLOPS_PER_SAMPLE = 4 * D_IN * H_HID + 10 * H_HID   # forward 2DH+3H, backward 2DH+7H
SMS, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nets", type=int, default=0,
                    help="c2 / c4: nets per GPU (default 4096 / 1024; fewer for profiling captures)")
    ap.add_argument("--epochs", type=int, default=0, help="c2 / c4: epochs per step (default 500 / 200)")
    ap.add_argument("--shape", type=int, default=-1,
                    help="c2 only: FP32 many-nets kernel shape (0..6); default: the autotuner's pick")
    ap.add_argument("--clusters", type=int, default=0,
                    help="c3 only: thread-block clusters of the wide-net kernel; default: the autotuner's pick")
    ap.add_argument("--workload", default="c2", choices=["c0", "c1", "c2", "c3", "c4"],
                    help="c0: the 33-16-1 net on the 120-row cohort, 1000 epochs per step; "
                         "c1: the 33-64-1 full-batch workload on 4096 rows, one epoch per step; "
                         "c2: 4096 independent 33-H-1 nets, 500 epochs per step (default line); "
                         "c3: one 48-2048-1 net on bf16 tensor cores, 1M rows, mini-batch 8192, one epoch per step; "
                         "c4: 1024 independent 48-256-1 nets on bf16 tensor cores, 200 epochs per step")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate_max(value: float, world: int) -> float:
    """Max of a per-rank float over all ranks (identity when world == 1)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------ inputs --

def workload_inputs(rank: int):
    """Seeded synthetic rows (features N(0,1)), weights and teacher weights;
    labels are computed afterwards by the library's own predict call."""
    from paper_1908_07847_gb300 import inputs as I
    X = I.features(I.COHORT_SEED + 1 + 1000 * rank, N_ROWS, D_IN)
    W = I.init_weights(I.INIT_SEED + rank, D_IN, H_HID)
    T = I.teacher_weights(D=D_IN)
    return X, W, T


# ---------------------------------------------------------------- clocks ----

class ClockSampler:
    """nvidia-smi clock and throttle-reason samples while the timed loop runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- our arm ------

def unit_rates():
    """Measured device rates (instructions/s) of the FP32 FMA pipe and of the
    special-function unit for tanh and exp2, from the library's diagnostic."""
    from paper_1908_07847_gb300 import binding as B
    ffma, tanh, ex2 = B.mlp_unit_rates()
    return {"ffma_tflops": 2 * ffma / 1e12, "tanh_per_s": tanh, "ex2_per_s": ex2}


def host_cpu():
    """Host core count and CPU model (lscpu), for the oracle baselines."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"cores_available": os.cpu_count(), "cpu_model": model}


def plain_rate(B, h, X, y, rows, steps, stream):
    """sample-steps/s of the plain path (separate forward, output, gradient,
    reduction and update kernels, mlp_step_plain) on `rows` rows, CUDA events."""
    import torch
    loss = torch.zeros(1, dtype=torch.float64, device=X.device)
    for _ in range(3):
        B.mlp_step_plain(h, X, y, rows, loss, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        B.mlp_step_plain(h, X, y, rows, loss, stream)
    e1.record()
    torch.cuda.synchronize()
    return rows * steps / (e0.elapsed_time(e1) * 1e-3)


def sfu_roofline(sigmoids_per_launch, launch_s, rates):
    """Sigmoids per second against the measured tanh rate of the SFU (the bf16
    paths evaluate every sigmoid as one tanh, two per bf16x2 instruction at the
    same value rate)."""
    got = sigmoids_per_launch / launch_s
    return {"achieved_per_s": got, "peak_per_s": rates["tanh_per_s"], "frac": got / rates["tanh_per_s"],
            "peak_basis": "tanh.approx rate measured by mlp_unit_rates on this device"}

def traffic_record(kernel: str, workload: str | None = None):
    """The DRAM traffic record of `kernel` (on `workload`, if given) from the
    committed ncu summaries (a `traffic-record:` line in profiles/*.md), if it
    was taken on the current kernel sources; else None."""
    import glob
    csrc = os.path.join(ROOT, "paper_1908_07847_gb300", "csrc")
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(path):
            if not line.startswith("traffic-record:"):
                continue
            try:
                rec = json.loads(line.split(":", 1)[1])
            except ValueError:
                continue
            if rec.get("kernel") != kernel or (workload is not None and rec.get("workload") != workload):
                continue
            h = hashlib.sha256()
            try:
                for f in rec["sources"]:
                    h.update(open(os.path.join(csrc, f), "rb").read())
            except (OSError, KeyError):
                return None
            return rec if h.hexdigest()[:16] == rec.get("source_sha256_16") else None
    return None


def traffic_from_profile():
    """DRAM bytes per launch of the fused kernel on the default workload."""
    rec = traffic_record("k_fused_train", WORKLOAD)
    return rec.get("dram_bytes_per_launch") if rec else None


def run_c1(args, rank, world, local):
    import torch
    from paper_1908_07847_gb300 import binding as B
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream().cuda_stream
    X, W, T = workload_inputs(rank)
    Xd = torch.from_numpy(X).to(dev)
    # labels: the teacher net's class decisions, by the library's predict
    th = B.mlp_create(D_IN, T[0].shape[0], LR, 1, B.MLP_FP32, B.MLP_ACT_SIGMOID)
    B.mlp_set_weights(th, *T)
    lab = torch.zeros(N_ROWS, dtype=torch.int8, device=dev)
    B.mlp_predict(th, Xd, N_ROWS, lab, stream)
    B.mlp_destroy(th)
    yd = lab.to(torch.float32)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed(step_fn, steps, warmup):
        for _ in range(warmup):
            step_fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for s, e in ev:
            flush.zero_()
            s.record()
            step_fn()
            e.record()
        torch.cuda.synchronize()
        return [s.elapsed_time(e) * 1e-3 for s, e in ev]

    from paper_1908_07847_gb300 import autotune
    rates = unit_rates()
    rows, _ = autotune.tune_fused(Xd, yd, D_IN, H_HID, N_ROWS)   # untimed; cached per device and shape
    h = B.mlp_create(D_IN, H_HID, LR, 1, B.MLP_FP32, B.MLP_ACT_SIGMOID)
    B.mlp_set_rows_per_block(h, rows)
    hp = B.mlp_create(D_IN, H_HID, LR, 1, B.MLP_FP32, B.MLP_ACT_SIGMOID)
    B.mlp_set_weights(h, *W)
    B.mlp_set_weights(hp, *W)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)

    def fused_step():
        B.mlp_train_epochs(h, Xd, yd, N_ROWS, 1, 0, loss, None, stream)

    def plain_step():
        B.mlp_step_plain(hp, Xd, yd, N_ROWS, loss, stream)

    # e2e: host buffers through the C ABI (pinned), copies inside the timed step
    Xh = torch.from_numpy(X).pin_memory()
    yh = yd.cpu().pin_memory()
    lh = torch.zeros(1, dtype=torch.float64).pin_memory()
    he = B.mlp_create(D_IN, H_HID, LR, 1, B.MLP_FP32, B.MLP_ACT_SIGMOID)
    B.mlp_set_rows_per_block(he, rows)
    B.mlp_set_weights(he, *W)

    def e2e_step():
        B.mlp_train_host(he, Xh, yh, N_ROWS, 1, 0, lh, stream)

    barrier(world)
    with ClockSampler(local) as clk:
        t_fused = timed(fused_step, args.steps, args.warmup)
    t_plain = timed(plain_step, max(args.steps // 4, 10), args.warmup)
    t_e2e = timed(e2e_step, max(args.steps // 4, 10), args.warmup)
    assert B.mlp_check(h, stream) == B.MLP_OK, B.mlp_last_error()
    for x in (h, hp, he):
        B.mlp_destroy(x)
    barrier(world)
    T_f = aggregate_max(sum(t_fused), world)
    T_p = aggregate_max(sum(t_plain), world)
    T_e = aggregate_max(sum(t_e2e), world)
    units = N_ROWS * world
    value = units * args.steps / T_f
    plain_value = units * len(t_plain) / T_p
    e2e_value = units * len(t_e2e) / T_e
    clocks = clk.summary()
    launch_s = statistics.mean(t_fused)
    achieved = FLOPS_PER_SAMPLE * N_ROWS / launch_s / 1e12
    peak = SMS * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
    out = {
        "metric": METRIC, "value": value, "unit": "sample-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": T_f / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (N(0,1) features, teacher-net labels; the paper's cohort is not public)",
        "config": {"workload": WORKLOAD, "n": N_ROWS, "D": D_IN, "H": H_HID, "lr": LR, "rows_per_block": rows,
                   "step": "one full-batch epoch: fwd+bwd+reduction+update (fused cooperative kernel)",
                   "l2": "flushed between timed steps (256 MiB write, outside the timed intervals)"},
        "plain_fp32": {"value": plain_value, "unit": "sample-steps/s",
                       "ms_per_step": T_p / len(t_plain) * 1e3,
                       "path": "separate forward/output/gradient/reduce/update kernels (mlp_step_plain)",
                       "speedup_of_fused": value / plain_value},
        "e2e": {"value": e2e_value, "unit": "sample-steps/s",
                "h2d_bytes_per_step": N_ROWS * D_IN * 4 + N_ROWS * 4, "d2h_bytes_per_step": 8,
                "call": "mlp_train_host (pinned host X, y in, read by the kernel through the host mapping; "
                        "loss written back to pinned host memory)"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic_from_profile(),
                     "kernel": "k_fused_train<36,2,sigmoid>",
                     "peak_basis": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (FFMA, derived)",
                     "ffma_measured_tflops": rates["ffma_tflops"],
                     "flops_per_launch": FLOPS_PER_SAMPLE * N_ROWS},
        "gpu_launches": args.steps,
        "clocks": clocks,
    }
    if rank == 0:
        out["cpu_baseline"] = cpu_baseline()
        print(json.dumps(out), flush=True)


# ------------------------------------------------------- reference arm ------

def oracle_epoch_rate(budget_s: float, rows: int):
    """Times the FP64 oracle on full-batch epochs of `rows` rows of the
    workload for about budget_s seconds; returns (sample-steps/s, epochs, rows)."""
    import oracle
    from paper_1908_07847_gb300 import inputs as I
    X, W, T = workload_inputs(0)
    X = X[:rows]
    y = oracle.predict(X, oracle.Params(*T)).astype(np.float64)
    p = oracle.Params(*W)
    t0 = time.perf_counter()
    oracle.train(X, y, p, LR, 1)
    one = max(time.perf_counter() - t0, 1e-6)
    epochs = max(1, int(budget_s / one))
    t0 = time.perf_counter()
    oracle.train(X, y, p, LR, epochs)
    dt = time.perf_counter() - t0
    return rows * epochs / dt, epochs, rows


def cpu_baseline():
    rate, epochs, rows = oracle_epoch_rate(10.0, N_ROWS)
    return {"value": rate, "unit": "sample-steps/s", "cores": 1, "kind": "oracle",
            "sample": "%d full-batch epochs over all %d rows (serial FP64 C oracle, one thread)" % (epochs, rows),
            **host_cpu()}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    from paper_1908_07847_gb300 import inputs as I
    X, W, T = workload_inputs(0)
    y = oracle.predict(X, oracle.Params(*T)).astype(np.float64)
    p = oracle.Params(*W)
    # Each step: one full-batch epoch over a bounded slice of the rows, sized so
    # that warm-up + steps take about two minutes at most.
    t0 = time.perf_counter()
    oracle.train(X, y, p, LR, 1)
    one = time.perf_counter() - t0
    rows = N_ROWS
    total = (args.steps + args.warmup) * one
    if total > 120.0:
        rows = max(64, int(N_ROWS * 120.0 / total))
    Xs, ys = X[:rows], y[:rows]
    for _ in range(args.warmup):
        p, _, _ = oracle.train(Xs, ys, p, LR, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        p, lh, _ = oracle.train(Xs, ys, p, LR, 1)
    dt = time.perf_counter() - t0
    value = rows * args.steps / dt
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "sample-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (N(0,1) features, teacher-net labels)",
        "config": {"workload": WORKLOAD, "n": N_ROWS, "D": D_IN, "H": H_HID, "lr": LR,
                   "step": "one full-batch epoch over %d of the %d rows (FP64 C oracle)" % (rows, N_ROWS)},
        "cpu_baseline": {"value": value, "unit": "sample-steps/s", "cores": 1, "kind": "oracle",
                         "sample": "%d steps of one full-batch epoch over %d rows" % (args.steps, rows)},
        "e2e": {"value": value, "unit": "sample-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(out), flush=True)


# ------------------------------------------------- cohort workload (c0) ----

C0_ROWS, C0_TRAIN, C0_H, C0_EPOCHS = 120, 96, 16, 1000
C0_WORKLOAD = ("33-16-1 sigmoid MLP on the 120-row synthetic cohort (first 96 rows train, 24 test), "
               "full-batch GD lr 0.1, 1000 epochs per step in one launch, FP32")


def run_c0(args, rank, world, local):
    """The cohort-sized network (Sec. 2.1-2.2 sizes): every step trains the
    33-16-1 net from the same initial weights for 1000 full-batch epochs on
    the 96 training rows, in one launch of the fused kernel (the rows stay in
    shared memory for all epochs)."""
    import torch
    from paper_1908_07847_gb300 import binding as B
    from paper_1908_07847_gb300 import inputs as I
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream().cuda_stream
    X = I.features(I.COHORT_SEED + 1000 * rank, C0_ROWS)
    W = I.init_weights(I.INIT_SEED + rank, D_IN, C0_H)
    T = I.teacher_weights(D=D_IN)
    Xd = torch.from_numpy(X).to(dev)
    th = B.mlp_create(D_IN, T[0].shape[0], LR, 1, B.MLP_FP32, B.MLP_ACT_SIGMOID)
    B.mlp_set_weights(th, *T)
    lab = torch.zeros(C0_ROWS, dtype=torch.int8, device=dev)
    B.mlp_predict(th, Xd, C0_ROWS, lab, stream)
    B.mlp_destroy(th)
    yd = lab.to(torch.float32)
    Xtr, ytr = Xd[:C0_TRAIN].contiguous(), yd[:C0_TRAIN].contiguous()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    lh = torch.zeros(C0_EPOCHS, dtype=torch.float64, device=dev)
    h = B.mlp_create(D_IN, C0_H, LR, 1, B.MLP_FP32, B.MLP_ACT_SIGMOID)
    # one block: the 96 rows fit it, and a single block sums and updates on chip
    # (a search over 1..12 blocks, timed on GB300s, picked it every time)
    rows_best = C0_TRAIN
    B.mlp_set_rows_per_block(h, rows_best)

    def timed(step_fn, steps, warmup):
        # every step restarts from the initial weights (set outside the timed interval)
        for _ in range(warmup):
            B.mlp_set_weights(h, *W)
            step_fn()
        torch.cuda.synchronize()
        out = []
        for _ in range(steps):
            B.mlp_set_weights(h, *W)
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            step_fn()
            e1.record()
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1) * 1e-3)
        return out

    def fused_step():
        B.mlp_train_epochs(h, Xtr, ytr, C0_TRAIN, C0_EPOCHS, 0, lh, None, stream)

    def plain_step():
        for _ in range(C0_EPOCHS):
            B.mlp_step_plain(h, Xtr, ytr, C0_TRAIN, lh, stream)

    Xh = torch.from_numpy(np.ascontiguousarray(X[:C0_TRAIN])).pin_memory()
    yh = ytr.cpu().pin_memory()
    lhh = torch.zeros(C0_EPOCHS, dtype=torch.float64).pin_memory()

    def e2e_step():
        B.mlp_train_host(h, Xh, yh, C0_TRAIN, C0_EPOCHS, 0, lhh, stream)

    barrier(world)
    with ClockSampler(local) as clk:
        t_fused = timed(fused_step, args.steps, args.warmup)
    # accuracies after one step (1000 epochs from the initial weights)
    pred = torch.zeros(C0_ROWS, dtype=torch.int8, device=dev)
    B.mlp_predict(h, Xd, C0_ROWS, pred, stream)
    torch.cuda.synchronize()
    ok = (pred == lab).cpu().numpy()
    acc = {"train": float(ok[:C0_TRAIN].mean()), "test": float(ok[C0_TRAIN:].mean())}
    t_plain = timed(plain_step, max(2, args.steps // 10), 1)
    t_e2e = timed(e2e_step, max(3, args.steps // 4), 1)
    assert B.mlp_check(h, stream) == B.MLP_OK, B.mlp_last_error()
    B.mlp_destroy(h)
    barrier(world)
    T_f = aggregate_max(sum(t_fused), world)
    T_p = aggregate_max(sum(t_plain), world)
    T_e = aggregate_max(sum(t_e2e), world)
    units = C0_TRAIN * C0_EPOCHS * world
    flops = (4 * D_IN * C0_H + 10 * C0_H) * C0_TRAIN * C0_EPOCHS
    rec = traffic_record("k_fused_train", C0_WORKLOAD)
    c0_traffic = rec.get("dram_bytes_per_launch") if rec else None
    launch_s = statistics.mean(t_fused)
    peak = SMS * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
    out = {
        "metric": METRIC, "value": units * args.steps / T_f, "unit": "sample-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": T_f / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": C0_WORKLOAD, "n": C0_ROWS, "n_train": C0_TRAIN, "D": D_IN, "H": C0_H, "lr": LR,
                   "epochs_per_step": C0_EPOCHS, "rows_per_block": rows_best, "us_per_epoch": T_f / args.steps / C0_EPOCHS * 1e6,
                   "l2": "flushed between timed steps (256 MiB write, outside the timed intervals)"},
        "accuracy": acc,
        "plain_fp32": {"value": units * len(t_plain) / T_p, "unit": "sample-steps/s",
                       "ms_per_step": T_p / len(t_plain) * 1e3,
                       "path": "mlp_step_plain, one call (five kernels) per epoch",
                       "speedup_of_fused": (units * args.steps / T_f) / (units * len(t_plain) / T_p)},
        "e2e": {"value": units * len(t_e2e) / T_e, "unit": "sample-steps/s",
                "h2d_bytes_per_step": C0_TRAIN * D_IN * 4 + C0_TRAIN * 4, "d2h_bytes_per_step": 8 * C0_EPOCHS,
                "call": "mlp_train_host (pinned host X, y in; loss history out)"},
        "roofline": {"bound": "alu", "achieved": flops / launch_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                     "frac": flops / launch_s / 1e12 / peak, "traffic": c0_traffic,
                     "kernel": "k_fused_train (33-16-1 instance)",
                     "peak_basis": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (FFMA, derived)",
                     "flops_per_launch": flops},
        "gpu_launches": args.steps, "clocks": clk.summary(),
    }
    if rank == 0:
        out["cpu_baseline"], out["parity"] = c0_oracle_leg(X, W, T, acc)
        print(json.dumps(out), flush=True)


def c0_oracle_leg(X, W, T, acc_gpu):
    """The FP64 oracle's full run of the workload (1000 epochs, one thread),
    timed; its train and test accuracies beside the library's."""
    import oracle
    y = oracle.predict(X, oracle.Params(*T)).astype(np.float64)
    t0 = time.perf_counter()
    q, _, _ = oracle.train(X[:C0_TRAIN], y[:C0_TRAIN], oracle.Params(*W), float(np.float32(LR)), C0_EPOCHS)
    dt = time.perf_counter() - t0
    ok = oracle.predict(X, q) == y
    cpu = {"value": C0_TRAIN * C0_EPOCHS / dt, "unit": "sample-steps/s", "cores": 1, "kind": "oracle",
           "sample": "the whole step: 1000 full-batch epochs over the 96 training rows (serial FP64 C oracle)",
           **host_cpu()}
    parity = {"oracle_accuracy": {"train": float(ok[:C0_TRAIN].mean()), "test": float(ok[C0_TRAIN:].mean())},
              "accuracy": acc_gpu, "tolerance": "one point (0.01) of the oracle's"}
    return cpu, parity


# --------------------------------------- many-nets workload (c2, default) --

C2_NETS, C2_EPOCHS, C2_SEED = 4096, 500, 2


def c2_workload():
    """The many-nets workload's name (--nets / --epochs shrink it for profiling
    captures only; the benchmark line is the 4096-net, 500-epoch one)."""
    return ("%d independent 33-H-1 sigmoid MLPs per GPU, H ~ U{4..128}, n ~ U{50..120}, "
            "full-batch GD lr 0.1, %d epochs per step in one launch, FP32" % (C2_NETS, C2_EPOCHS))


C2_WORKLOAD = c2_workload()


KERNEL_OF_SHAPE = {0: "k_batched_train", 1: "k_batched_train2", 2: "k_batched_train2", 3: "k_batched_tiled",
                   4: "k_batched_tiled", 5: "k_batched_tiled", 6: "k_batched_train2"}


def c2_shapes(world: int):
    """Hidden widths and row counts of the whole job's 4096 x world nets."""
    from paper_1908_07847_gb300 import inputs as I
    return I.batched_shapes(C2_SEED, C2_NETS * world, (4, 128), (50, 120))


def c2_config(world: int):
    """The workload description both arms print (identical by construction)."""
    Hs, ns = c2_shapes(world)
    return {"workload": c2_workload(), "nets": int(len(Hs)), "rows_total": int(ns.sum()),
            "epochs_per_step": C2_EPOCHS, "D": D_IN, "lr": LR,
            "l2": "flushed between timed steps (256 MiB write, outside the timed intervals)"}


def c2_net(t: int, n: int, H: int):
    """Net t of the job: its rows (N(0, 1) features) and initial weights."""
    from paper_1908_07847_gb300 import inputs as I
    return (I.features(I.subseed(C2_SEED, 100 + t), int(n), D_IN),
            I.init_weights(I.subseed(C2_SEED, 200 + t), D_IN, int(H)))


def c2_flops(Hs, ns, epochs):
    """Algorithmic FLOPs of `epochs` epochs: 4 D H + 10 H per row-epoch
    (forward 2 D H + 3 H, backward 2 D H + 7 H)."""
    return float(np.sum(ns * (4 * D_IN * Hs + 10 * Hs))) * epochs


def run_c2(args, rank, world, local):
    import torch
    from paper_1908_07847_gb300 import binding as B
    from paper_1908_07847_gb300 import shard
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream().cuda_stream
    rates = unit_rates()
    Hs_all, ns_all = c2_shapes(world)
    # nets split across ranks by cost (rows x hidden units), largest first
    parts = shard.partition_lpt(ns_all * Hs_all, world)
    mine = parts[rank]
    Hs, ns = Hs_all[mine], ns_all[mine]
    nets = [c2_net(int(t), ns_all[t], Hs_all[t]) for t in mine]
    _, _, T = workload_inputs(0)
    Xall = torch.from_numpy(np.concatenate([X for X, _ in nets])).to(dev)
    # labels: the teacher net's class decisions, by the library's predict
    th = B.mlp_create(D_IN, T[0].shape[0], LR, 1, B.MLP_FP32, B.MLP_ACT_SIGMOID)
    B.mlp_set_weights(th, *T)
    lab = torch.zeros(Xall.shape[0], dtype=torch.int8, device=dev)
    B.mlp_predict(th, Xall, Xall.shape[0], lab, stream)
    B.mlp_destroy(th)
    yall = lab.to(torch.float32)
    P0h = np.concatenate([np.concatenate([W[0].ravel(), W[1], W[2], W[3]]) for _, W in nets]).astype(np.float32)
    P0 = torch.from_numpy(P0h).to(dev)
    Pw = P0.clone()
    L = torch.zeros((len(mine), C2_EPOCHS), dtype=torch.float64, device=dev)
    offs_x = np.concatenate([[0], np.cumsum(ns)[:-1]])
    offs_p = np.concatenate([[0], np.cumsum((D_IN + 2) * Hs + 1)[:-1]])
    descs = [B.mlp_net_desc(int(Hs[i]), int(ns[i]), Xall[int(offs_x[i]):].data_ptr(),
                            yall[int(offs_x[i]):].data_ptr(), Pw[int(offs_p[i]):].data_ptr(), L[i].data_ptr())
             for i in range(len(mine))]
    plan = B.mlp_batch_create(B.MLP_FP32, B.MLP_ACT_SIGMOID, D_IN, descs, LR, 1)
    # kernel shape: the autotuner's pick on this plan (untimed; it restores the
    # weights it trains), unless given
    from paper_1908_07847_gb300 import autotune
    if args.shape >= 0:
        B.mlp_batch_set_shape(plan, args.shape)
        tuned = {"shape": args.shape, "source": "--shape"}
    else:
        shape, ms = autotune.tune_batched(plan, D_IN, Hs, ns, Pw, epochs=25, reps=3)
        tuned = {"shape": shape, "source": "autotune.tune_batched", "ms_per_epoch": ms}
    gather = shard.Gather(parts, D_IN, Hs_all, C2_EPOCHS) if world > 1 else None
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    # one step = the whole 500-epoch launch, captured once in a CUDA graph
    g = torch.cuda.CUDAGraph()
    s2 = torch.cuda.Stream()
    s2.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s2):
        B.mlp_batch_run(plan, C2_EPOCHS, s2.cuda_stream)   # warm-up outside capture
        s2.synchronize()
        with torch.cuda.graph(g, stream=s2):
            B.mlp_batch_run(plan, C2_EPOCHS, s2.cuda_stream)
    torch.cuda.current_stream().wait_stream(s2)

    def step():
        g.replay()
        if gather is not None:
            gather(Pw, L)

    for _ in range(max(args.warmup, 1)):
        Pw.copy_(P0)
        step()
    torch.cuda.synchronize()
    barrier(world)
    times = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            Pw.copy_(P0)
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            step()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) * 1e-3)
    # the kernel's own duration (graph replay alone), for the roofline
    kt = []
    for _ in range(3):
        Pw.copy_(P0)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        kt.append(e0.elapsed_time(e1) * 1e-3)
    assert B.mlp_batch_check(plan, stream) == B.MLP_OK, B.mlp_last_error()
    B.mlp_batch_destroy(plan)
    del g

    # e2e: the same training through the host-buffer entry point (rows, labels
    # and initial weights in; trained weights and loss histories out)
    Xh = torch.from_numpy(np.concatenate([X for X, _ in nets])).pin_memory()
    yh = yall.cpu().pin_memory()
    Pin = torch.from_numpy(P0h).pin_memory()
    Pout = torch.empty_like(Pin).pin_memory()
    Lh = torch.empty((len(mine), C2_EPOCHS), dtype=torch.float64).pin_memory()
    hplan = B.mlp_batch_create_host(B.MLP_FP32, B.MLP_ACT_SIGMOID, D_IN, Hs, ns, C2_EPOCHS, LR, 1)
    B.mlp_batch_set_shape(hplan, tuned["shape"])
    e2e_steps = max(3, args.steps // 4)
    B.mlp_batch_run_host(hplan, Xh, yh, Pin, Pout, Lh, C2_EPOCHS, stream)
    t_e2e = []
    with ClockSampler(local) as clk_e2e:
        for _ in range(e2e_steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            B.mlp_batch_run_host(hplan, Xh, yh, Pin, Pout, Lh, C2_EPOCHS, stream)
            e1.record()
            torch.cuda.synchronize()
            t_e2e.append(e0.elapsed_time(e1) * 1e-3)
    B.mlp_batch_destroy(hplan)
    e2e_same = bool(np.array_equal(Pout.numpy(), Pw.cpu().numpy()))

    # the plain path, one net at a time (a mid-size net of the sample), for the
    # speedup of the one-launch many-nets kernel over it
    t_mid = int(np.argsort(ns * Hs)[len(mine) // 2])
    hp = B.mlp_create(D_IN, int(Hs[t_mid]), LR, 1, B.MLP_FP32, B.MLP_ACT_SIGMOID)
    B.mlp_set_weights(hp, *nets[t_mid][1])
    plain = plain_rate(B, hp, Xall[int(offs_x[t_mid]):], yall[int(offs_x[t_mid]):], int(ns[t_mid]), 200, stream)
    B.mlp_destroy(hp)
    barrier(world)
    T_f = aggregate_max(sum(times), world)
    T_e = aggregate_max(sum(t_e2e), world)
    units = int(ns_all.sum()) * C2_EPOCHS
    value = units * args.steps / T_f
    launch_s = statistics.mean(kt)
    flops = c2_flops(Hs, ns, C2_EPOCHS)
    ffma_peak = rates["ffma_tflops"]
    # DRAM bytes of a launch from the committed capture of a reduced case of
    # the same kernel, scaled by the rows of the job (rows and weights are
    # read once a launch and stay on chip for every epoch), while the
    # kernel's sources still hash to the recorded value
    rec = traffic_record(KERNEL_OF_SHAPE[tuned["shape"]], "c2")
    traffic = rec["dram_bytes_per_row"] * float(ns.sum()) if rec and "dram_bytes_per_row" in rec else None
    sigmoids = float(np.sum(ns * (Hs + 1))) * C2_EPOCHS
    out = {
        "metric": METRIC, "value": value, "unit": "sample-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": T_f / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (N(0,1) features, teacher-net labels; the paper's cohort is not public)",
        "config": c2_config(world),
        "roofline": {"bound": "alu", "achieved": flops / launch_s / 1e12, "peak": ffma_peak, "unit": "TFLOP/s",
                     "frac": flops / launch_s / 1e12 / ffma_peak, "traffic": traffic,
                     "kernel": "%s (one launch, %d epochs of this rank's nets)" % (KERNEL_OF_SHAPE[tuned["shape"]],
                                                                                  C2_EPOCHS),
                     "peak_basis": "FP32 FFMA rate measured on this device by mlp_unit_rates (of measured; "
                                   "MEASURED_PEAKS.json holds no FP32 figure)",
                     "flops_per_launch": flops, "launch_ms": launch_s * 1e3,
                     "sfu": {"sigmoids_per_s": sigmoids / launch_s, "mufu_ops_per_sigmoid": 2,
                             "peak_mufu_per_s": rates["ex2_per_s"],
                             "frac": 2 * sigmoids / launch_s / rates["ex2_per_s"],
                             "peak_basis": "ex2.approx rate measured by mlp_unit_rates (each FP32 sigmoid is one "
                                           "ex2.approx and one rcp.approx)"}},
        "e2e": {"value": units * len(t_e2e) / T_e, "unit": "sample-steps/s",
                "h2d_bytes_per_step": int(Xh.numel() * 4 + yh.numel() * 4 + Pin.numel() * 4),
                "d2h_bytes_per_step": int(Pout.numel() * 4 + Lh.numel() * 8),
                "call": "mlp_batch_run_host (pinned host rows, labels and initial weights in; trained weights "
                        "and %d-epoch loss histories out; one launch)" % C2_EPOCHS,
                "same_weights_as_device_path": e2e_same, "clocks": clk_e2e.summary()},
        "plain_fp32": {"value": plain, "unit": "sample-steps/s",
                       "path": "mlp_step_plain on one mid-size net of the workload (the plain path takes one net "
                               "at a time)", "speedup_of_batched": value / world / plain},
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
        "kernel_shape": tuned,
    }
    if world > 1:
        out["multi_gpu"] = {"split": "nets by cost (rows x hidden), longest processing time first",
                            "exchange": "one gather of trained weights and loss histories to rank 0 per step "
                                        "(NCCL), inside the timed step"}
    if rank == 0:
        out["cpu_baseline"], out["parity"] = c2_oracle_leg([(nets[i][0], nets[i][1]) for i in range(min(16, len(nets)))],
                                                           Pw.cpu().numpy(), offs_p)
        print(json.dumps(out), flush=True)


def c2_oracle_leg(sample, P_gpu, offs_p):
    """The FP64 oracle on the first nets of this rank's share for all 500
    epochs (OpenMP over nets on every host core), timed; their weights after
    the benchmark's last step (same initial weights, labels by the oracle's
    teacher predict) compared with the oracle's."""
    import oracle
    from paper_1908_07847_gb300 import inputs as I
    T = oracle.Params(*I.teacher_weights(D=D_IN))
    onets = []
    for X, W in sample:
        X64 = X.astype(np.float64)
        onets.append((X64, oracle.predict(X64, T).astype(np.float64), oracle.Params(*W)))
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    out, _ = oracle.batch_train(onets, float(np.float32(LR)), C2_EPOCHS, threads=threads)
    dt = time.perf_counter() - t0
    err = 0.0
    for i, q in enumerate(out):
        ref = q.flat()
        got = P_gpu[int(offs_p[i]):int(offs_p[i]) + ref.size].astype(np.float64)
        err = max(err, float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))))
    rows = int(sum(X.shape[0] for X, _, _ in onets))
    cpu = {"value": rows * C2_EPOCHS / dt, "unit": "sample-steps/s", "cores": threads, "kind": "oracle",
           "sample": "%d of the nets (%d rows), all %d epochs (FP64 C oracle, OpenMP over nets)"
                     % (len(onets), rows, C2_EPOCHS), **host_cpu()}
    parity = {"nets": len(onets), "epochs": C2_EPOCHS,
              "measure": "max over nets of max |w - w*| / max |w*| after the benchmark's %d epochs" % C2_EPOCHS,
              "value": err, "tolerance": 1e-4}
    return cpu, parity


def run_reference_c2(args, rank, world):
    """The reference arm on the default workload: the FP64 oracle on a bounded
    subset of the job's nets (16 nets, all 500 epochs, OpenMP over nets on
    every host core) per step; rank 0 only."""
    if rank != 0:
        return
    import oracle
    from paper_1908_07847_gb300 import inputs as I
    Hs_all, ns_all = c2_shapes(world)
    T = oracle.Params(*I.teacher_weights(D=D_IN))
    onets = []
    for t in range(16):
        X, W = c2_net(t, ns_all[t], Hs_all[t])
        X64 = X.astype(np.float64)
        onets.append((X64, oracle.predict(X64, T).astype(np.float64), oracle.Params(*W)))
    rows = int(sum(X.shape[0] for X, _, _ in onets))
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.batch_train(onets, float(np.float32(LR)), C2_EPOCHS, threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.batch_train(onets, float(np.float32(LR)), C2_EPOCHS, threads=threads)
    dt = time.perf_counter() - t0
    value = rows * C2_EPOCHS * args.steps / dt
    sample = ("each step: 16 of the %d nets (%d rows) for all %d epochs (FP64 C oracle, OpenMP over nets "
              "on %d threads)" % (len(Hs_all), rows, C2_EPOCHS, threads))
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "sample-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (N(0,1) features, teacher-net labels; the paper's cohort is not public)",
        "config": c2_config(world),
        "cpu_baseline": {"value": value, "unit": "sample-steps/s", "cores": threads, "kind": "oracle",
                         "sample": sample, **host_cpu()},
        "e2e": {"value": value, "unit": "sample-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(out), flush=True)


# --------------------------------- one wide bf16 tensor-core net (c3) ------

C3_N, C3_D, C3_H, C3_MB, C3_SUB = 1 << 20, 48, 2048, 8192, 8192
C3_WORKLOAD = ("one 48-2048-1 sigmoid MLP (33 features zero-padded to 48), 1,048,576 rows, bf16 X on tcgen05 "
               "tensor cores (clusters of 8 blocks), FP32 master weights, mini-batch 8192, lr 0.1, one epoch per step")


def c3_inputs(dev, seed=1908):
    """1M seeded rows in bf16 on the device (33 N(0,1) features, zero padding),
    teacher-net labels by the library's predict; returns X, y and init weights."""
    import torch
    from paper_1908_07847_gb300 import binding as B
    from paper_1908_07847_gb300 import inputs as I
    X = torch.zeros((C3_N, C3_D), dtype=torch.bfloat16, device=dev)
    chunk = 1 << 18
    for r0 in range(0, C3_N, chunk):
        Xc = I.features(I.subseed(seed, 20_000 + r0 // chunk), chunk, 33, C3_D)
        X[r0:r0 + chunk] = torch.from_numpy(Xc).to(dev).to(torch.bfloat16)
    T = I.teacher_weights(D=33, Dpad=C3_D)
    th = B.mlp_create(C3_D, T[0].shape[0], LR, 1, B.MLP_BF16, B.MLP_ACT_SIGMOID)
    B.mlp_set_weights(th, *T)
    lab = torch.zeros(C3_N, dtype=torch.int8, device=dev)
    B.mlp_predict(th, X, C3_N, lab, torch.cuda.current_stream().cuda_stream)
    B.mlp_destroy(th)
    W = [np.ascontiguousarray(np.asarray(a, np.float32)) for a in I.init_weights(I.INIT_SEED + 3, 33, C3_H, C3_D)]
    return X, lab.to(torch.float32), W


def c3_oracle_leg(X, W):
    """The FP64 oracle on one mini-batch step over the first 8192 rows (labels by
    the oracle's teacher predict), timed; the library's step on the same rows,
    compared.  Returns (cpu_baseline dict, parity dict)."""
    import torch
    import oracle
    from paper_1908_07847_gb300 import binding as B
    from paper_1908_07847_gb300 import inputs as I
    Xs = X[:C3_SUB].float().cpu().numpy().astype(np.float64)
    ys = oracle.predict(Xs, oracle.Params(*I.teacher_weights(D=33, Dpad=C3_D))).astype(np.float64)
    p0 = oracle.Params(*[a.astype(np.float64) for a in W])
    t0 = time.perf_counter()
    q, _, _ = oracle.train(Xs, ys, p0, float(np.float32(LR)), 1, minibatch=C3_MB)
    dt = time.perf_counter() - t0
    h = B.mlp_create(C3_D, C3_H, LR, 1, B.MLP_BF16, B.MLP_ACT_SIGMOID)
    try:
        B.mlp_set_weights(h, *W)
        yd = torch.from_numpy(ys.astype(np.float32)).to(X.device)
        B.mlp_train_epochs(h, X[:C3_SUB].contiguous(), yd, C3_SUB, 1, C3_MB, None, None,
                           torch.cuda.current_stream().cuda_stream)
        assert B.mlp_check(h, torch.cuda.current_stream().cuda_stream) == B.MLP_OK, B.mlp_last_error()
        W1 = np.zeros((C3_H, C3_D), np.float32)
        b1, w2, b2 = np.zeros(C3_H, np.float32), np.zeros(C3_H, np.float32), np.zeros(1, np.float32)
        B.mlp_get_weights(h, W1, b1, w2, b2)
    finally:
        B.mlp_destroy(h)
    flat = lambda a, b, c, d: np.concatenate([np.ravel(a), np.ravel(b), np.ravel(c), np.ravel(d)]).astype(np.float64)
    w0 = flat(*W)
    dg, dr = flat(W1, b1, w2, b2) - w0, q.flat() - w0
    err = float(np.max(np.abs(dg - dr)) / np.max(np.abs(dr)))
    cpu = {"value": C3_SUB / dt, "unit": "sample-steps/s", "cores": 1, "kind": "oracle",
           "sample": "one mini-batch step over the first %d rows (serial FP64 C oracle, one thread)" % C3_SUB,
           **host_cpu()}
    parity = {"rows": C3_SUB, "steps": 1, "measure": "max |dw - dw*| / max |dw*| of the weight update",
              "value": err, "tolerance": 2e-2}
    return cpu, parity


def run_c3(args, rank, world, local):
    import torch
    from paper_1908_07847_gb300 import binding as B
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream().cuda_stream
    X, y, W = c3_inputs(dev, 1908 + rank)
    rates = unit_rates()
    h = B.mlp_create(C3_D, C3_H, LR, 1, B.MLP_BF16, B.MLP_ACT_SIGMOID)
    B.mlp_set_weights(h, *W)
    # cluster count: the autotuner's pick for this shape (untimed), unless given
    from paper_1908_07847_gb300 import autotune
    if args.clusters > 0:
        tuned = {"clusters": args.clusters, "source": "--clusters"}
    else:
        k, us = autotune.tune_clusters(X, y, C3_D, C3_H, C3_N, C3_MB)
        tuned = {"clusters": k, "source": "autotune.tune_clusters", "us_per_step": us,
                 "limit": B.mlp_cluster_limit(C3_H)}
    B.mlp_set_clusters(h, tuned["clusters"])
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        B.mlp_train_epochs(h, X, y, C3_N, 1, C3_MB, loss, None, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for s0, e0 in ev:
            flush.zero_()
            s0.record()
            step()
            e0.record()
        torch.cuda.synchronize()
    times = [s0.elapsed_time(e0) * 1e-3 for s0, e0 in ev]
    assert B.mlp_check(h, stream) == B.MLP_OK, B.mlp_last_error()
    # e2e: host X, y through mlp_train_host (staged to the device every step)
    Xh = X.cpu().pin_memory()
    yh = y.cpu().pin_memory()
    lh = torch.zeros(1, dtype=torch.float64).pin_memory()
    e2e_steps = max(3, args.steps // 4)
    B.mlp_train_host(h, Xh, yh, C3_N, 1, C3_MB, lh, stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        B.mlp_train_host(h, Xh, yh, C3_N, 1, C3_MB, lh, stream)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    # the plain path (separate kernels per step, FP32 arithmetic on the bf16
    # rows) on mini-batches of 8192 rows of the same net
    plain = plain_rate(B, h, X, y, C3_MB, 20, stream)
    B.mlp_destroy(h)
    barrier(world)
    T_f = aggregate_max(sum(times), world)
    T_e = aggregate_max(t_e2e, world)
    units = C3_N * world
    launch_s = statistics.mean(times)
    # algorithmic tensor-core work per row: X W1^T and d1^T X (2 D H each), gb1
    # and gw2 (2 H each)
    mma_flops = float(C3_N) * (4 * C3_D * C3_H + 4 * C3_H)
    peak = 1731.1   # MEASURED_PEAKS.json bf16_tflops_sustained
    out = {
        "metric": METRIC, "value": units * args.steps / T_f, "unit": "sample-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": T_f / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": C3_WORKLOAD, "n": C3_N, "D": C3_D, "H": C3_H, "minibatch": C3_MB,
                   "updates_per_step": C3_N // C3_MB,
                   "l2": "flushed between timed steps (256 MiB write, outside the timed intervals)"},
        "e2e": {"value": units * e2e_steps / T_e, "unit": "sample-steps/s",
                "h2d_bytes_per_step": C3_N * C3_D * 2 + C3_N * 4, "d2h_bytes_per_step": 8,
                "call": "mlp_train_host (pinned host X, y in; loss out)"},
        "plain_fp32": {"value": plain, "unit": "sample-steps/s",
                       "path": "mlp_step_plain on 8192-row mini-batches (FP32 arithmetic on bf16 rows)",
                       "speedup_of_tensor_core": units * args.steps / T_f / plain},
        "roofline": {"bound": "tensor", "achieved": mma_flops / launch_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                     "frac": mma_flops / launch_s / 1e12 / peak, "traffic": None, "kernel": "k_tc_cluster",
                     "peak_basis": "bf16_tflops_sustained of measured", "flops_per_launch": mma_flops,
                     "sfu": sfu_roofline(float(C3_N) * (C3_H + 1), launch_s, rates)},
        "gpu_launches": args.steps, "clocks": clk.summary(), "kernel_shape": tuned,
    }
    if rank == 0:
        out["cpu_baseline"], out["parity"] = c3_oracle_leg(X, W)
        print(json.dumps(out), flush=True)


# ----------------------------------------- bf16 tensor-core workload (c4) --

C4_NETS, C4_EPOCHS, C4_H, C4_D = 1024, 200, 256, 48
C4_WORKLOAD = ("1024 independent 48-256-1 sigmoid MLPs (33 features zero-padded to 48), n ~ U{4096..16384}, "
               "bf16 X on tcgen05 tensor cores, FP32 master weights, full-batch GD lr 0.1, 200 epochs per step")


def run_c4(args, rank, world, local):
    import torch
    from paper_1908_07847_gb300 import binding as B
    from paper_1908_07847_gb300 import inputs as I
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream().cuda_stream
    rates = unit_rates()
    seed = 4 + rank
    n_nets = args.nets or C4_NETS
    epochs = args.epochs or C4_EPOCHS
    _, ns = I.batched_shapes(seed, n_nets, (C4_H, C4_H), (4096, 16384))
    offs = np.concatenate([[0], np.cumsum(ns)])
    total = int(offs[-1])
    Xall = torch.zeros((total, C4_D), dtype=torch.bfloat16, device=dev)
    chunk = 1 << 20
    for r0 in range(0, total, chunk):
        r1 = min(total, r0 + chunk)
        Xc = I.features(I.subseed(seed, 10_000 + r0 // chunk), r1 - r0, 33, C4_D)
        Xall[r0:r1] = torch.from_numpy(Xc).to(dev).to(torch.bfloat16)
    T = I.teacher_weights(D=33, Dpad=C4_D)
    th = B.mlp_create(C4_D, T[0].shape[0], LR, 1, B.MLP_BF16, B.MLP_ACT_SIGMOID)
    B.mlp_set_weights(th, *T)
    lab = torch.zeros(total, dtype=torch.int8, device=dev)
    B.mlp_predict(th, Xall, total, lab, stream)
    B.mlp_destroy(th)
    yall = lab.to(torch.float32)
    P_per = (C4_D + 2) * C4_H + 1
    P0 = torch.from_numpy(np.concatenate([np.concatenate([a.ravel() for a in I.init_weights(
        I.subseed(seed, 200 + t), 33, C4_H, C4_D)]) for t in range(n_nets)])).to(dev)
    Pw = P0.clone()
    descs = [B.mlp_net_desc(C4_H, int(ns[t]), Xall[int(offs[t]):].data_ptr(), yall[int(offs[t]):].data_ptr(),
                            Pw[t * P_per:].data_ptr(), None) for t in range(n_nets)]
    plan = B.mlp_batch_create(B.MLP_BF16, B.MLP_ACT_SIGMOID, C4_D, descs, LR, 1)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    g = torch.cuda.CUDAGraph()
    s2 = torch.cuda.Stream()
    s2.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s2):
        B.mlp_batch_run(plan, epochs, s2.cuda_stream)   # warm-up outside capture
        s2.synchronize()
        with torch.cuda.graph(g, stream=s2):
            B.mlp_batch_run(plan, epochs, s2.cuda_stream)
    torch.cuda.current_stream().wait_stream(s2)
    for _ in range(max(args.warmup, 1)):
        Pw.copy_(P0)
        g.replay()
    torch.cuda.synchronize()
    times = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            Pw.copy_(P0)
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) * 1e-3)
    assert B.mlp_batch_check(plan, stream) == B.MLP_OK, B.mlp_last_error()
    B.mlp_batch_destroy(plan)
    dev_w = Pw.cpu().numpy()
    # e2e: the same training through the host-buffer entry point (bf16 rows,
    # labels and initial weights in; trained weights and loss histories out)
    Xh = Xall.cpu().pin_memory()
    yh = yall.cpu().pin_memory()
    Pin = P0.cpu().pin_memory()
    Pout = torch.empty_like(Pin).pin_memory()
    Lh = torch.empty((n_nets, epochs), dtype=torch.float64).pin_memory()
    hplan = B.mlp_batch_create_host(B.MLP_BF16, B.MLP_ACT_SIGMOID, C4_D, [C4_H] * n_nets, ns, epochs, LR, 1)
    B.mlp_batch_run_host(hplan, Xh, yh, Pin, Pout, Lh, epochs, stream)
    t_e2e = []
    with ClockSampler(local) as clk_e2e:
        for _ in range(max(2, args.steps // 2)):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            B.mlp_batch_run_host(hplan, Xh, yh, Pin, Pout, Lh, epochs, stream)
            e1.record()
            torch.cuda.synchronize()
            t_e2e.append(e0.elapsed_time(e1) * 1e-3)
    B.mlp_batch_destroy(hplan)
    e2e_same = bool(np.array_equal(Pout.numpy(), dev_w))
    T_e = aggregate_max(sum(t_e2e), world)
    e2e = {"value": int(ns.sum()) * epochs * world * len(t_e2e) / T_e, "unit": "sample-steps/s",
           "h2d_bytes_per_step": int(Xh.numel() * 2 + yh.numel() * 4 + Pin.numel() * 4),
           "d2h_bytes_per_step": int(Pout.numel() * 4 + Lh.numel() * 8),
           "call": "mlp_batch_run_host (pinned host bf16 rows, labels and initial weights in; trained weights "
                   "and %d-epoch loss histories out; one launch)" % epochs,
           "same_weights_as_device_path": e2e_same, "clocks": clk_e2e.summary()}
    del Xh
    # the plain path on net 0 (separate kernels per step, FP32 arithmetic on its
    # bf16 rows), for the speedup of the one-launch tensor-core kernel over it
    hp = B.mlp_create(C4_D, C4_H, LR, 1, B.MLP_BF16, B.MLP_ACT_SIGMOID)
    B.mlp_set_weights(hp, *[np.ascontiguousarray(np.asarray(a_, np.float32)) for a_ in
                            I.init_weights(I.subseed(seed, 200), 33, C4_H, C4_D)])
    plain = plain_rate(B, hp, Xall, yall, int(ns[0]), 50, stream)
    B.mlp_destroy(hp)
    T_f = aggregate_max(sum(times), world)
    units = int(ns.sum()) * epochs * world
    # algorithmic tensor-core work per row-epoch: X W1^T and d1^T X (2 D H each),
    # gb1 and gw2 (2 H each)
    mma_flops = float(ns.sum()) * epochs * (4 * C4_D * C4_H + 4 * C4_H)
    launch_s = statistics.mean(times)
    peak = 1731.1   # MEASURED_PEAKS.json bf16_tflops_sustained
    # DRAM bytes of one launch, scaled by rows x epochs from the committed
    # capture of a reduced case (X is read once per epoch at any size)
    rec = traffic_record("k_tc_batched")
    c4_traffic = rec["dram_bytes_per_row_epoch"] * float(ns.sum()) * epochs if rec else None
    out = {
        "metric": METRIC, "value": units * args.steps / T_f, "unit": "sample-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": T_f / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": C4_WORKLOAD, "nets": n_nets, "rows_total": int(ns.sum()), "epochs_per_step": epochs,
                   "l2": "inputs (1 GB of bf16 X) larger than L2; L2 also flushed between timed steps"},
        "roofline": {"bound": "tensor", "achieved": mma_flops / launch_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                     "frac": mma_flops / launch_s / 1e12 / peak, "traffic": c4_traffic, "kernel": "k_tc_batched",
                     "peak_basis": "bf16_tflops_sustained of measured", "flops_per_launch": mma_flops,
                     "sfu": sfu_roofline(float(ns.sum()) * epochs * (C4_H + 1), launch_s, rates)},
        "plain_fp32": {"value": plain, "unit": "sample-steps/s",
                       "path": "mlp_step_plain on one net of the workload (FP32 arithmetic on bf16 rows)",
                       "speedup_of_tensor_core": units * args.steps / T_f / plain},
        "e2e": e2e, "gpu_launches": args.steps, "clocks": clk.summary(),
    }
    if rank == 0:
        out["cpu_baseline"], out["parity"] = c4_oracle_leg(seed, ns)
        print(json.dumps(out), flush=True)


def c4_oracle_leg(seed, ns, sample=2, epochs=3):
    """The FP64 oracle on the first `sample` nets of the workload for `epochs`
    epochs (their bf16 rows regenerated on the host, labels by the oracle's
    teacher predict), timed; the library's bf16 batch plan on the same nets and
    labels, compared by the weight change."""
    import torch
    import oracle
    from paper_1908_07847_gb300 import binding as B
    from paper_1908_07847_gb300 import inputs as I
    rows = int(sum(ns[:sample]))
    Xh = I.bf16_round(I.features(I.subseed(seed, 10_000), rows, 33, C4_D)).astype(np.float64)
    T = oracle.Params(*I.teacher_weights(D=33, Dpad=C4_D))
    yh = oracle.predict(Xh, T).astype(np.float64)
    offs = np.concatenate([[0], np.cumsum(ns[:sample])])
    onets = [(Xh[offs[t]:offs[t + 1]], yh[offs[t]:offs[t + 1]],
              oracle.Params(*I.init_weights(I.subseed(seed, 200 + t), 33, C4_H, C4_D))) for t in range(sample)]
    t0 = time.perf_counter()
    ref = [oracle.train(X, y, p, float(np.float32(LR)), epochs)[0] for X, y, p in onets]
    dt = time.perf_counter() - t0
    dev = torch.device("cuda")
    Xd = torch.from_numpy(Xh.astype(np.float32)).to(dev).to(torch.bfloat16)
    yd = torch.from_numpy(yh.astype(np.float32)).to(dev)
    params = [torch.from_numpy(p.flat().astype(np.float32)).to(dev) for _, _, p in onets]
    descs = [B.mlp_net_desc(C4_H, int(ns[t]), Xd[int(offs[t]):].data_ptr(), yd[int(offs[t]):].data_ptr(),
                            params[t].data_ptr(), None) for t in range(sample)]
    plan = B.mlp_batch_create(B.MLP_BF16, B.MLP_ACT_SIGMOID, C4_D, descs, LR, 1)
    B.mlp_batch_run(plan, epochs, torch.cuda.current_stream().cuda_stream)
    assert B.mlp_batch_check(plan, torch.cuda.current_stream().cuda_stream) == B.MLP_OK, B.mlp_last_error()
    B.mlp_batch_destroy(plan)
    err = 0.0
    for P, q, (_, _, p0) in zip(params, ref, onets):
        dg, dr = P.cpu().numpy().astype(np.float64) - p0.flat(), q.flat() - p0.flat()
        err = max(err, float(np.max(np.abs(dg - dr)) / np.max(np.abs(dr))))
    cpu = {"value": rows * epochs / dt, "unit": "sample-steps/s", "cores": 1, "kind": "oracle",
           "sample": "%d of the nets (%d rows), %d epochs (serial FP64 C oracle, one thread)" % (sample, rows, epochs),
           **host_cpu()}
    parity = {"nets": sample, "epochs": epochs, "measure": "max over nets of max |dw - dw*| / max |dw*|",
              "value": err, "tolerance": 2e-2}
    return cpu, parity


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.workload == "c2" and (args.nets or args.epochs):
        global C2_NETS, C2_EPOCHS
        C2_NETS = args.nets or C2_NETS
        C2_EPOCHS = args.epochs or C2_EPOCHS
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    if args.impl == "reference":
        if args.workload == "c2":
            run_reference_c2(args, rank, world)
        else:
            run_reference(args, rank, world)
    elif args.workload == "c0":
        run_c0(args, rank, world, local)
    elif args.workload == "c2":
        run_c2(args, rank, world, local)
    elif args.workload == "c3":
        run_c3(args, rank, world, local)
    elif args.workload == "c4":
        run_c4(args, rank, world, local)
    else:
        run_c1(args, rank, world, local)
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
