#!/usr/bin/env python3
"""Benchmark: verified motion-point queries/s on the bin-picking workload.

Workload (one step = one svm_check_motions call over the whole batch):
64 linear joint motions x a 200 000-point depth-camera cloud of a bin with 30
objects, margin 0.03 m, 128 steps per motion, network 15 -> 256 x 4 ReLU -> 1
in the chosen precision.  Before timing, the network is trained on the GPU on
data the library generates and labels itself (1024 motions like the
workload's, 4096 samples each), and the gate is calibrated on 16 separate
motions.  Every (motion, point) pair covered by a verdict counts as one query.
The same step through the plain FP32 path (SIMT network, same verifier) is
timed too and reported beside the value.

Timing: W warm-up steps, then K steps each bracketed by CUDA events on the
launching stream; an L2 flush (a 256 MiB write) runs between steps, outside
the events.  Clocks are sampled with nvidia-smi during the timed region.
``e2e`` repeats the measurement through the same C ABI with the cloud and the
results in pinned host memory (copies inside the timed region).

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same
workload (the reference arm of this build).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2402_15281_gb300 import synth as S  # noqa: E402

EPS = 0.03
STEPS = 128
N_MOTIONS = 64
N_POINTS = 200_000
WIDTH, HIDDEN = 256, 4
PREC_NAMES = {"fp32": 0, "bf16": 1, "fp8": 2}
DTYPE_NAMES = {"fp32": "f32", "bf16": "bf16", "fp8": "e4m3"}
METRIC = "verified motion-point queries/s"
FLOP_PER_PAIR = 2 * (3 * WIDTH + HIDDEN * WIDTH * WIDTH + WIDTH)   # 526 336
FLOP_PER_CAPSULE_TEST = 20
# DRAM bytes (read + write) of one launch of the tensor-core network kernel on this workload, from
# one-pass ncu captures of a full-size launch; to be reset to None whenever that kernel changes.
TC_TRAFFIC_BYTES = {"bf16": 3.86e6, "fp8": 3.62e6}


def workload(seed=0):
    robot = S.make_robot(1)
    pts = S.bin_cloud(N_POINTS, seed=seed)
    q0, q1 = S.bin_motions(robot, N_MOTIONS, seed=seed)
    return robot, pts, q0, q1


def weights():
    return S.xavier_weights(WIDTH, HIDDEN, seed=2)


def workload_config(prec, weights="trained"):
    w = {"trained": "trained on GPU-generated, exactly labelled data (1024 motions x 4096 samples, 30 epochs), "
                    "gate calibrated on 16 separate motions",
         "random": "Glorot-uniform seed 2, gate calibrated on 16 separate motions",
         "open": "Glorot-uniform seed 2, gate open (every pair also checked exactly)"}[weights]
    return {"workload": "bin-picking: 64 linear motions x 200k-point bin cloud, margin 0.03 m, 128 steps, "
                        "MLP 15-256x4-1 ReLU",
            "motions": N_MOTIONS, "points": N_POINTS, "steps": STEPS, "margin_m": EPS,
            "precision": prec, "l2": "flushed between steps (256 MiB write)", "weights": w,
            **({"fp8_scales": "per-layer activation scales calibrated on the same 16 motions (2x headroom)"}
               if prec == "fp8" else {})}


# --------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        finally:
            os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------- oracle

def oracle_sample(robot, pts, q0, q1, layers, prec, gate, n_motions):
    """The FP64 oracle's combined check on the first n_motions motions."""
    import oracle
    P = oracle.quantized_params(layers, PREC_NAMES[prec])
    t = time.perf_counter()
    oracle.check_motions(P, WIDTH, HIDDEN, 0, robot, q0[:n_motions], q1[:n_motions], STEPS, pts, EPS, gate)
    dt = time.perf_counter() - t
    return n_motions * len(pts) / dt, dt, oracle.num_threads()


def run_reference(args):
    if world_info()[1] != 0:
        return
    robot, pts, q0, q1 = workload()
    layers = weights()
    gate = float("inf")    # random weights flag every pair (see the calibrated gate of the GPU arm)
    n_m = 1
    for _ in range(args.warmup):
        oracle_sample(robot, pts, q0, q1, layers, args.prec, gate, n_m)
    times = []
    for k in range(args.steps):
        _, dt, cores = oracle_sample(robot, pts, q0[k % N_MOTIONS:], q1[k % N_MOTIONS:], layers, args.prec, gate, n_m)
        times.append(dt)
    pairs = n_m * N_POINTS
    value = pairs * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.prec, "open"),
            "cpu_baseline": {"value": value, "unit": "queries/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n_m} motion x {N_POINTS} points per step (FP64 C oracle, OpenMP; "
                                       "Glorot weights with the gate open, so every pair is also checked "
                                       "exactly -- the FP64 network dominates the cost either way)"},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# --------------------------------------------------------------------- ranks

def world_info():
    """(world size, rank, local rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x, device=None):
    """The largest x over all ranks (x itself with one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(pairs_per_rank_step, steps, total_ms_max, world):
    """Whole-job queries/s: every rank checks its own batch (weak scaling), so
    the job checks world x pairs per step in the slowest rank's time."""
    return world * pairs_per_rank_step * steps / (total_ms_max / 1e3)


# --------------------------------------------------------------------- GPU arm

def run_gpu(args):
    import torch
    import paper_2402_15281_gb300 as svm

    world, rank, local = world_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    svm.build() if rank == 0 or world == 1 else None
    if world > 1:
        torch.distributed.barrier()
    from paper_2402_15281_gb300 import training
    robot, pts, q0, q1 = workload(seed=rank)
    prec = PREC_NAMES[args.prec]
    train_info = None
    if args.weights == "trained":
        tq0, tq1 = training.bin_training_motions(robot, 1024, seed=41)
        blob, hist = training.train_model(svm, robot, tq0, tq1, samples_per_motion=4096, steps=STEPS,
                                          batch=65536, epochs=30, patience=10, device=local)
        train_info = {"val_mae_m": hist["best_val_mae"], "train_samples": hist["train_samples"],
                      "train_samples_per_s": hist["samples_per_s"], "seconds": round(hist["seconds"], 2)}
    else:
        blob = svm.make_blob(weights())
    layers = svm.parse_blob(blob)
    pts_d = torch.from_numpy(pts).to(dev)
    cq0, cq1 = S.bin_motions(robot, 16, seed=1000)

    def make_model(p):
        h = svm.svm_create_model(robot, WIDTH, HIDDEN, svm.SVM_RELU, p, local)
        svm.svm_load_weights(h, blob)
        if p == svm.SVM_FP8_E4M3:
            # per-layer activation scales from the calibration motions (2x headroom)
            svm.svm_calibrate_act_scales(h, cq0, cq1, pts_d, 2.0)
        t = training.calibrate_tau(svm, h, robot, pts_d, EPS, STEPS, cq0, cq1)
        svm.svm_set_gate(h, t)
        return h, t

    model, tau = make_model(prec)
    svm.svm_profile_enable(model, True)
    res = svm.new_results(N_MOTIONS, dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    flags = 0

    def step():
        svm.svm_check_motions(model, q0, q1, pts_d, EPS, STEPS, flags, res, stream)

    for _ in range(args.warmup):
        step()
        flush.fill_(1.0)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    phases = np.zeros(4)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))
            starts[k].record(stream)
            step()
            ends[k].record(stream)
            phases += svm.svm_profile_read(model)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = np.array([s.elapsed_time(e) for s, e in zip(starts, ends)])
    total_ms = max_over_ranks(float(ms.sum()), dev)
    clocks = clk.summary()
    phases /= args.steps
    r = svm.results_to_numpy(res)[:N_MOTIONS]
    pairs_step = N_MOTIONS * N_POINTS
    value = job_throughput(pairs_step, args.steps, total_ms, world)

    # end to end through the C ABI with host buffers: H2D cloud, check, D2H results
    pts_h = torch.from_numpy(pts).pin_memory()
    res_h = torch.empty_like(res, device="cpu").pin_memory()
    pts_e = torch.empty_like(pts_d)
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pts_e.copy_(pts_h, non_blocking=True)
        svm.svm_check_motions(model, q0, q1, pts_e, EPS, STEPS, flags, res, stream)
        res_h.copy_(res, non_blocking=True)
        torch.cuda.synchronize()
        if k >= args.warmup:
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_total = max_over_ranks(float(np.sum(e2e_ms)), dev)
    e2e_value = job_throughput(pairs_step, args.steps, e2e_total, world)

    # roofline of the dominant kernel
    import json as _json
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = _json.load(open(pk_path))
    n_verified = int(r["n_verified"].sum())
    mlp_ms, ver_ms = phases[1], phases[2]
    sm_max = 2070.0
    alu_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12      # FP32 TFLOP/s at the maximum SM clock
    if mlp_ms >= ver_ms:
        flop = pairs_step * FLOP_PER_PAIR
        achieved = flop / (mlp_ms * 1e-3) / 1e12
        if args.prec == "fp32":
            roof = {"kernel": "mlp_fp32", "bound": "alu", "achieved": achieved, "peak": alu_peak,
                    "unit": "TFLOP/s", "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2070 MHz"}
        else:
            scale = 2.0 if args.prec == "fp8" else 1.0
            pk = peaks.get("bf16_tflops_sustained")
            src = "measured sustained bf16 (MEASURED_PEAKS.json)" + (" x2 for fp8" if scale > 1 else "")
            if pk is None:
                pk, src = 1700.0, "fallback sustained bf16"
            roof = {"kernel": f"mlp_tc_{args.prec}", "bound": "tensor", "achieved": achieved, "peak": pk * scale,
                    "unit": "TFLOP/s", "peak_source": src}
    else:
        flop = n_verified * (STEPS + 1) * 7 * FLOP_PER_CAPSULE_TEST
        achieved = flop / (ver_ms * 1e-3) / 1e12
        roof = {"kernel": "verify", "bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2070 MHz"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = TC_TRAFFIC_BYTES.get(args.prec) if roof["kernel"].startswith("mlp_tc") else None

    # the plain FP32 path on the same workload and weights (SIMT network, same verifier)
    fp32 = None
    if args.prec != "fp32" and not args.no_fp32_path:
        m32, tau32 = make_model(svm.SVM_FP32)
        for _ in range(2):
            svm.svm_check_motions(m32, q0, q1, pts_d, EPS, STEPS, flags, res, stream)
        flush.fill_(0.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k32 = 3
        e0.record(stream)
        for _ in range(k32):
            svm.svm_check_motions(m32, q0, q1, pts_d, EPS, STEPS, flags, res, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms32 = e0.elapsed_time(e1) / k32
        r32 = svm.results_to_numpy(res)[:N_MOTIONS]
        fp32 = {"value": pairs_step / (ms32 / 1e3), "ms_per_step": ms32, "tau_m": tau32,
                "collisions": int(r32["collision"].sum()),
                "verdicts_equal": bool(np.array_equal(r32["collision"], r["collision"]))}
        svm.svm_destroy_model(m32)

    # prologue, network, probe (early exit on), plan + verify, ties, finalize; strict adds plan + verify
    launches_per_step = 6 + (0 if flags & svm.SVM_NO_EARLY_EXIT else 1) + (2 if flags & svm.SVM_STRICT else 0)
    line = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAMES[args.prec], "data": "synthetic",
            "config": workload_config(args.prec, args.weights), "clocks": clocks,
            "e2e": {"value": e2e_value, "unit": "queries/s",
                    "h2d_bytes_per_step": int(pts.nbytes + 2 * q0.nbytes),
                    "d2h_bytes_per_step": int(res.numel())},
            "gpu_launches": launches_per_step * args.steps,
            "roofline": roof,
            "phases_ms": {"prologue": float(phases[0]), "network": float(phases[1]),
                          "verify": float(phases[2]), "finalize": float(phases[3])},
            "tau_m": tau, "collisions": int(r["collision"].sum()),
            "fp32_path": fp32, "speedup_vs_fp32_path": (value / fp32["value"]) if fp32 else None,
            "training": train_info,
            "flagged_fraction": float(r["n_flagged"].sum()) / pairs_step,
            "verified_fraction": n_verified / pairs_step,
            "margin_ties_fp64": int(r["n_ambiguous"].sum())}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, dt, cores = oracle_sample(robot, pts, q0, q1, layers, args.prec, EPS + tau, 2)
        line["cpu_baseline"] = {"value": v, "unit": "queries/s", "cores": cores, "kind": "oracle",
                                "sample": f"2 motions x {N_POINTS} points, same gate ({dt:.1f} s)"}
    svm.svm_destroy_model(model)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def profile_call(args):
    """One check call for an external profiler.  With --weights random: Glorot weights and the
    blob's gate, no other network launch (ncu -k regex:mlp_tc -c 1).  With --weights trained:
    the bench's training and gate calibration first, which launch the network kernel once
    (ncu -k regex:mlp_tc -s 1 -c 1)."""
    import torch
    import paper_2402_15281_gb300 as svm
    from paper_2402_15281_gb300 import training
    svm.build()
    robot, pts, q0, q1 = workload()
    m = min(args.profile_call, N_MOTIONS)
    pts_d = torch.from_numpy(pts).cuda()
    h = svm.svm_create_model(robot, WIDTH, HIDDEN, svm.SVM_RELU, PREC_NAMES[args.prec], 0)
    if args.weights == "trained":
        tq0, tq1 = training.bin_training_motions(robot, 1024, seed=41)
        blob, _ = training.train_model(svm, robot, tq0, tq1, samples_per_motion=4096, steps=STEPS,
                                       batch=65536, epochs=30, patience=10)
        svm.svm_load_weights(h, blob)
        cq0, cq1 = S.bin_motions(robot, 16, seed=1000)
        if args.prec == "fp8":
            svm.svm_calibrate_act_scales(h, cq0, cq1, pts_d, 2.0)
        svm.svm_set_gate(h, training.calibrate_tau(svm, h, robot, pts_d, EPS, STEPS, cq0, cq1))
    else:
        svm.svm_load_weights(h, svm.make_blob(weights()))
        if args.prec == "fp8":
            svm.svm_set_act_scales(h, np.full(HIDDEN, 1 / 64, np.float32))
    res = svm.new_results(m)
    svm.svm_check_motions(h, q0[:m], q1[:m], pts_d, EPS, STEPS, 0, res)
    torch.cuda.synchronize()
    r = svm.results_to_numpy(res)[:m]
    print("profile call:", m, "motions,", int(r["collision"].sum()), "collisions, status", int(r["status"].max()))
    svm.svm_destroy_model(h)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", choices=list(PREC_NAMES), default="bf16")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32-path", action="store_true")
    ap.add_argument("--weights", choices=["trained", "random"], default="trained")
    ap.add_argument("--profile-call", type=int, default=0, metavar="M",
                    help="for profilers: one svm_check_motions call on the first M bench motions (weights "
                         "as --weights), then exit (no timing, no JSON line)")
    args = ap.parse_args()
    if args.profile_call > 0:
        profile_call(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
