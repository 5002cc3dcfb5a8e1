"""Benchmark: registrations of the stereo-like street pair on GB300.

One step = one full registration (cvo_register_pair) of the 20,000-point
street pair: grid and query setup, then up to 100 annealed iterations of the
fused sweep + on-device step (lengthscale 0.3 -> 0.05 m, cutoff 3
lengthscales, RGB + 19-class labels).  Inputs are resident in HBM when the
timed region starts; L2 is flushed (256 MB write) between steps.

value  = in-cutoff kernel-pair evaluations per second, summed over ranks
e2e    = the same metric through the C ABI with pinned host buffers (host to
         device copies inside the timed region)
roofline = the sweep kernel's algorithmic FP32 FLOPs per launch over its
         event-timed duration, against the FP32 peak from the unit counts;
         with the DRAM traffic and the warp-instruction issue rate of the
         committed ncu capture when it was taken on the current source
sections = batch (64 cube pairs batched vs one by one), backward (room pair),
         large (200,000-point pair), tuning (the autotuner's choice, timed
         registrations; untimed here)
cpu_baseline = the FP64 oracle's own registration loop on the same pair,
         first 20 iterations, on the host cores

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cvo|reference]
"""
import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "kernel-pair evals/s & registered pairs/s, batched vs plain GPU, at oracle tol"
UNIT = "pair-evals/s"
SM_COUNT = 152
FP32_LANES_PER_SM = 128
EX2_PER_CLK_SM = 29   # measured ex2.approx.f32 throughput per SM per clock on a GB300


def flops_per_pair(blocks):
    """Algorithmic FP32 FLOPs of one in-cutoff pair (FMA = 2): offset 3,
    squared distance 5, exponent scale 1, moments W/E/Q 19; a squared-
    exponential block of d entries 3d + 1; an inner-product block of d
    entries 2d - 1 plus the product with the kernel value 1.  The ex2 runs on
    the XU pipe and is not counted."""
    f = 3 + 5 + 1 + 19
    for kind, dim, _, _ in blocks:
        f += 3 * dim + 1 if kind == "se" else 2 * dim
    return f


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def profile_value(kernel_src, key):
    """A per-launch figure of the sweep (key: traffic_bytes_per_launch,
    warp_instructions_per_launch) from the committed ncu summary, if it was
    taken on the current kernel source (the files in kernel_src, hashed in
    order); else None."""
    path = os.path.join(ROOT, "profiles", "sweep_street-20k.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    t = re.search(key + r":\s*([0-9.eE+]+)", text)
    if not m or not t:
        return None
    data = b"".join(open(f, "rb").read() for f in kernel_src)
    sha = hashlib.sha256(data).hexdigest()
    return float(t.group(1)) if sha == m.group(1) else None


class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index, command=None):
        self.proc = None
        self.first = ""
        self.index = index
        self.command = command or ["nvidia-smi", "-i", str(index), "--query-gpu=" + ",".join(self.FIELDS),
                                   "--format=csv,noheader,nounits", "-lms", "100"]

    def start(self):
        """Starts sampling and waits (at most 3 s) for the first sample, so
        that the samples cover the timed region from its start."""
        import select
        try:
            self.proc = subprocess.Popen(self.command, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        try:
            ready, _, _ = select.select([self.proc.stdout], [], [], 3.0)
            if ready:
                self.first = self.proc.stdout.readline()
        except Exception:
            self.first = ""

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        out = (self.first or "") + (out or "")
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_setup(backend):
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist, world, rank, local


def max_over_ranks(dist, world, value, device=None):
    if world == 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, world, value, device=None):
    if world == 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def workload():
    import scenes
    p = scenes.street_pair()
    pr = p.params
    kw = dict(blocks=p.blocks, ell=pr["ell"], ell_min=pr["ell_min"], cutoff_mult=pr["cutoff_mult"],
              max_iters=pr["max_iters"], anneal=pr["anneal"])
    config = {"workload": "street-20k", "points_per_cloud": p.n,
              "features": "rgb (squared-exponential, scale 0.2) x 19-class labels (inner product), float32",
              "lengthscale": "0.3 -> 0.05 m annealed (2 % decays)", "cutoff": "3 lengthscales",
              "max_iters": pr["max_iters"], "l2": "flushed between steps (256 MB write)"}
    return p, kw, config


def batch_section(cvo, torch, dev, flush, reps=2):
    """64 cube pairs of 5k-60k points (RGB + labels in bf16): one batched
    registration (one graph launch for the whole batch) against the same pairs
    registered one after another through cvo_register_pair."""
    import scenes
    pairs = scenes.batch_pairs()
    pr = pairs[0].params
    kw = dict(blocks=pairs[0].blocks, ell=pr["ell"], cutoff_mult=pr["cutoff_mult"], max_iters=pr["max_iters"])
    args = []
    for p in pairs:
        args.append((torch.tensor(p.X, device=dev), torch.tensor(p.Z, device=dev), np.eye(4),
                     torch.tensor(p.FX, device=dev).to(torch.bfloat16),
                     torch.tensor(p.FZ, device=dev).to(torch.bfloat16)))
    out = {"workload": "batch-64: cube pairs, 5k-60k points per cloud, rgb + 19 labels in bf16, "
                       f"l = {pr['ell']}, cutoff 3 l, {pr['max_iters']} iterations",
           "pairs": len(pairs), "points": int(sum(p.n + p.m for p in pairs))}
    with cvo.CVO(**kw) as h:
        # cell size and query-group extent tuned on the largest pair (untimed)
        big = max(range(len(pairs)), key=lambda k: pairs[k].n + pairs[k].m)
        out["tuning"] = h.autotune(*args[big])
        h.register_batch(args)
        torch.cuda.synchronize()
        t_b, evals_b = 0.0, 0
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, infos, _ = h.register_batch(args)
            torch.cuda.synchronize()
            t_b += time.perf_counter() - t0
            evals_b += sum(i["pairs"] for i in infos)
        for a in args[:2]:
            h.register(*a)
        t_p, evals_p = 0.0, 0
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for a in args:
                _, info = h.register(*a)
                evals_p += info["pairs"]
            torch.cuda.synchronize()
            t_p += time.perf_counter() - t0
    out["batched"] = {"registered_pairs_per_s": reps * len(pairs) / t_b, "pair_evals_per_s": evals_b / t_b,
                      "ms_per_batch": 1e3 * t_b / reps}
    out["plain"] = {"registered_pairs_per_s": reps * len(pairs) / t_p, "pair_evals_per_s": evals_p / t_p,
                    "ms_per_batch": 1e3 * t_p / reps}
    out["speedup"] = t_p / t_b
    return out


def backward_section(cvo, torch, dev, flush, reps=5):
    """Room pair (19,200 points per cloud, rgb, l = 0.1, cutoff 3 l): one
    forward evaluation and one backward pass (gradients for both clouds'
    points and features and for l, device outputs), CUDA-event timed."""
    import scenes
    p = scenes.room_pair()
    pr = p.params
    X, Z = torch.tensor(p.X, device=dev), torch.tensor(p.Z, device=dev)
    FX, FZ = torch.tensor(p.FX, device=dev), torch.tensor(p.FZ, device=dev)
    T = p.T_true
    out = {"workload": f"room-19k: {p.n} + {p.m} points, rgb, l = {pr['ell']}, cutoff 3 l"}
    with cvo.CVO(blocks=p.blocks, ell=pr["ell"], cutoff_mult=pr["cutoff_mult"]) as h:
        ev = h.evaluate(X, Z, T, FX, FZ)
        h.backward(X, Z, T, FX, FZ)
        stream = torch.cuda.current_stream()
        t = {"forward": 0.0, "backward": 0.0}
        for _ in range(reps):
            for name in ("forward", "backward"):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                if name == "forward":
                    h.evaluate(X, Z, T, FX, FZ)
                else:
                    h.backward(X, Z, T, FX, FZ)
                e1.record(stream)
                e1.synchronize()
                t[name] += e0.elapsed_time(e1)
    out["pairs"] = int(ev["pairs"])
    out["ms_forward"] = t["forward"] / reps
    out["ms_backward"] = t["backward"] / reps
    # the backward sweeps every in-cutoff pair twice (once per cloud)
    out["backward_pair_evals_per_s"] = 2 * ev["pairs"] / (1e-3 * out["ms_backward"])
    out["timing"] = "whole calls (setup, sweeps, copies) between CUDA events, L2 flushed before each"
    return out


def large_section(cvo, torch, dev, flush, reps=2):
    """The large semantic pair (200,000 points per cloud, 20 x 10 x 80 m box,
    rgb + 19 labels, l 0.5 -> 0.05 m, cutoff 3 l, <= 200 iterations): full
    registration latency (inputs resident, CUDA events) and the indicator."""
    import scenes
    p = scenes.large_pair()
    pr = p.params
    kw = dict(blocks=p.blocks, ell=pr["ell"], ell_min=pr["ell_min"], cutoff_mult=pr["cutoff_mult"],
              max_iters=pr["max_iters"], anneal=pr["anneal"])
    X, Z = torch.tensor(p.X, device=dev), torch.tensor(p.Z, device=dev)
    FX, FZ = torch.tensor(p.FX, device=dev), torch.tensor(p.FZ, device=dev)
    out = {"workload": f"box80-200k: {p.n} + {p.m} points, rgb + 19 labels, l 0.5 -> 0.05 m, cutoff 3 l, "
                       f"<= {pr['max_iters']} iterations"}
    with cvo.CVO(**kw) as h:
        out["tuning"] = h.autotune(X, Z, np.eye(4), FX, FZ)
        h.register(X, Z, np.eye(4), FX, FZ)
        stream = torch.cuda.current_stream()
        ms = []
        for _ in range(reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            T, info = h.register(X, Z, np.eye(4), FX, FZ)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
    D = np.linalg.inv(T) @ p.T_true
    out.update({"ms_per_registration": float(np.mean(ms)), "iterations": info["iters"],
                "ell_final": info["ell_final"], "i_theta": info["i_theta"], "pairs": info["pairs"],
                "pair_evals_per_s": info["pairs"] / (1e-3 * float(np.mean(ms))),
                "pose_err_vs_truth": {"rot_rad": float(math.acos(max(-1.0, min(1.0, (np.trace(D[:3, :3]) - 1) / 2)))),
                                      "trans_m": float(np.linalg.norm(D[:3, 3]))}})
    return out


def cpu_baseline(p, kw, iters=20):
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    _, info, _ = oracle.register(p.X, p.Z, np.eye(4), FX=p.FX, FZ=p.FZ, **dict(kw, max_iters=iters))
    dt = time.perf_counter() - t0
    return {"value": info["pairs_total"] / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"first {info['iters']} of <= {kw['max_iters']} iterations of the FP64 oracle's registration "
                      f"of the full street-20k pair ({info['pairs_total']} in-cutoff pairs, {dt:.1f} s)",
            "seconds": dt}


def run_reference(args):
    """The oracle as the reference arm: each step is a bounded sample of the
    same workload (the first iterations of the oracle's registration)."""
    dist, world, rank, _ = dist_setup("gloo")
    if rank != 0:
        return
    p, kw, config = workload()
    iters = 4
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        oracle.register(p.X, p.Z, np.eye(4), FX=p.FX, FZ=p.FZ, **dict(kw, max_iters=iters))
    pairs, total = 0, 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, info, _ = oracle.register(p.X, p.Z, np.eye(4), FX=p.FX, FZ=p.FZ, **dict(kw, max_iters=iters))
        total += time.perf_counter() - t0
        pairs += info["pairs_total"]
    value = pairs / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config,
            "cpu_baseline": {"kind": "oracle", "cores": oracle.num_threads(), "value": value, "unit": UNIT,
                             "sample": f"each step: first {iters} iterations of the FP64 oracle's registration of "
                                       f"the full street-20k pair"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cvo", choices=["cvo", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-vs-plain section")
    ap.add_argument("--no-backward", action="store_true", help="skip the forward/backward section")
    ap.add_argument("--no-large", action="store_true", help="skip the 200,000-point section")
    ap.add_argument("--tuning", default=None,
                    help="cell_factor,super_delta,chunk_len for the street pair instead of autotuning "
                         "(fixed launch sequence for profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import paper_2012_03683_gb300 as cvo

    dist, world, rank, local = dist_setup("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    p, kw, config = workload()
    config["parallelism"] = f"replicas x{world}" if world > 1 else "single pair"
    X = torch.tensor(p.X, device=dev)
    Z = torch.tensor(p.Z, device=dev)
    FX = torch.tensor(p.FX, device=dev)
    FZ = torch.tensor(p.FZ, device=dev)
    h = cvo.CVO(**kw)
    # sweep tuning for this pair at its start (untimed, before the warm-up)
    if args.tuning:
        cf, sd, ip = args.tuning.split(",")
        h.apply_tuning(float(cf), int(sd), int(ip))
        tuning = dict(h.tuning(), source="--tuning")
    else:
        tuning = h.autotune(X, Z, np.eye(4), FX, FZ)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    T0 = np.eye(4)

    for _ in range(max(args.warmup, 3)):
        h.register(X, Z, T0, FX, FZ)
    torch.cuda.synchronize()

    # ---- timed region: device-resident inputs -------------------------------
    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = cvo.cvo_kernel_launches()
    step_ms, pairs, cands, iters = [], 0, 0, []
    T_last = None
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        T_last, info = h.register(X, Z, T0, FX, FZ)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        pairs += info["pairs"]
        cands += info["candidates"]
        iters.append(info["iters"])
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = cvo.cvo_kernel_launches() - launches0

    # ---- sweep kernel duration: the same registrations with CUDA events
    # around every sweep launch (host-queued iterations instead of the graph)
    cvo.cvo_set_timing(h.h, True)
    sweep_ms, sweep_n, sweep_pairs, timed_ms = 0.0, 0, 0, 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, info = h.register(X, Z, T0, FX, FZ)
        timed_ms += 1e3 * (time.perf_counter() - t0)
        ms, n = cvo.cvo_sweep_time(h.h)
        sweep_ms += ms * n
        sweep_n += n
        sweep_pairs += info["pairs"]
    cvo.cvo_set_timing(h.h, False)
    clocks = sampler.stop()
    total_ms = float(sum(step_ms))
    total_ms_max = max_over_ranks(dist, world, total_ms, dev)
    pairs_all = sum_over_ranks(dist, world, float(pairs), dev)
    value = pairs_all / (total_ms_max * 1e-3)
    regs_per_s = world * args.steps / (total_ms_max * 1e-3)

    # ---- end to end: pinned host buffers through the C ABI -----------------
    Xh, Zh = torch.tensor(p.X).pin_memory(), torch.tensor(p.Z).pin_memory()
    FXh, FZh = torch.tensor(p.FX).pin_memory(), torch.tensor(p.FZ).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in (Xh, Zh, FXh, FZh))
    import ctypes
    d2h = 16 * 8 + ctypes.sizeof(cvo.Info)
    h.register(Xh, Zh, T0, FXh, FZh)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e2e_ms, e2e_pairs = 0.0, 0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, info = h.register(Xh, Zh, T0, FXh, FZh)
        torch.cuda.synchronize()
        e2e_ms += 1e3 * (time.perf_counter() - t0)
        e2e_pairs += info["pairs"]
    e2e_ms = max_over_ranks(dist, world, e2e_ms, dev)
    e2e_pairs = sum_over_ranks(dist, world, float(e2e_pairs), dev)
    h.close()
    batch = batch_section(cvo, torch, dev, flush) if (rank == 0 and not args.no_batch) else None
    backward = backward_section(cvo, torch, dev, flush) if (rank == 0 and not args.no_backward) else None
    large = large_section(cvo, torch, dev, flush) if (rank == 0 and not args.no_large) else None

    if rank != 0:
        return
    peaks, peak_src = load_peaks()
    fpp = flops_per_pair(kw["blocks"])
    achieved = sweep_pairs * fpp / (sweep_ms * 1e-3) / 1e12 if sweep_ms > 0 else None
    peak = SM_COUNT * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    csrc = os.path.join(ROOT, "paper_2012_03683_gb300", "csrc")
    sweep_src = [os.path.join(csrc, "cvo_sweep.cu"), os.path.join(csrc, "cvo_sweep_dev.cuh")]
    traffic = profile_value(sweep_src, "traffic_bytes_per_launch")
    winst = profile_value(sweep_src, "warp_instructions_per_launch")
    sweep_ms_avg = sweep_ms / max(sweep_n, 1)
    # the same launches against the SM's instruction issue rate (one warp
    # instruction per scheduler per clock, 4 schedulers per SM): the bound of
    # a kernel whose FP32 pipes are not the limit
    issue_peak = SM_COUNT * 4 * peaks.get("sm_max_mhz", 2070.0) * 1e6
    issue = {"achieved_warp_inst_per_s": winst / (sweep_ms_avg * 1e-3) if (winst and sweep_ms_avg > 0) else None,
             "peak_warp_inst_per_s": issue_peak,
             "frac": (winst / (sweep_ms_avg * 1e-3) / issue_peak) if (winst and sweep_ms_avg > 0) else None,
             "warp_instructions_per_launch": winst,
             "source": "smsp__inst_executed.sum, mean of the 3 launches of the committed ncu capture "
                       "(profiles/sweep_street-20k.md, "
                       "same source hash) over the CUDA-event time per launch; peak: 152 SMs x 4 schedulers "
                       "x sm_max_mhz"}
    dT = np.linalg.inv(T_last) @ p.T_true
    pose_err = {"rot_rad": float(math.acos(max(-1.0, min(1.0, (np.trace(dT[:3, :3]) - 1.0) / 2.0)))),
                "trans_m": float(np.linalg.norm(dT[:3, 3]))}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config,
        "registered_pairs_per_s": regs_per_s,
        "pairs_per_registration": pairs / args.steps, "candidates_per_registration": cands / args.steps,
        "iterations": iters,
        "e2e": {"value": e2e_pairs / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "tuning": tuning,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": traffic, "kernel": "k_sweep (fused neighbour sweep)",
                     "flops_per_pair": fpp, "sweep_ms_avg": sweep_ms_avg, "sweep_launches": sweep_n,
                     "timing": "CUDA events around each sweep launch, over the same registrations queued "
                               "from the host (the timed steps run the loop as one CUDA graph)",
                     "ms_per_registration_event_timed": timed_ms / args.steps,
                     "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {peaks.get('sm_max_mhz', 2070.0)} MHz "
                                    f"(sm_max_mhz {peak_src})",
                     # the one ex2 per in-cutoff pair against the XU pipe's rate
                     "sfu": {"achieved_ex2_per_s": (sweep_pairs / (sweep_ms * 1e-3)) if sweep_ms > 0 else None,
                             "peak_ex2_per_s": SM_COUNT * EX2_PER_CLK_SM * peaks.get("sm_max_mhz", 2070.0) * 1e6,
                             "frac": (sweep_pairs / (sweep_ms * 1e-3)) /
                                     (SM_COUNT * EX2_PER_CLK_SM * peaks.get("sm_max_mhz", 2070.0) * 1e6)
                                     if sweep_ms > 0 else None,
                             "peak_source": f"152 SMs x {EX2_PER_CLK_SM} ex2/clk/SM (measured on a GB300 with an "
                                            "independent-chain ex2.approx throughput loop) x sm_max_mhz"},
                     "issue": issue},
        "clocks": clocks,
        "final_pose_err_vs_truth": pose_err,
        "batch": batch,
        "backward": backward,
        "large": large,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p, kw)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
