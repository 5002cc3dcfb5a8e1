"""Benchmark: batched registration of 64 frame pairs against the plain
single-pair form, on GB300.

Headline workload (batch-64): 64 cube pairs, 5,000-60,000 points per cloud,
RGB (squared exponential, scale 0.2) x 19-class labels (inner product), both
stored in bfloat16 with float32 arithmetic, lengthscale 0.1 m, cutoff 3
lengthscales, <= 50 iterations, per-pair convergence masks.  One step = one
batched registration of all 64 pairs (cvo_register_batch: every pair's
setup, then one CUDA graph whose loop runs the batched sweep and the
per-pair steps until every pair has stopped).  Inputs are resident in HBM
when the timed region starts; L2 is flushed (256 MB write) before every
step; steps are timed with CUDA events on the launching stream.

value     = in-cutoff kernel-pair evaluations per second of the batched form,
            summed over ranks (replicas: each rank registers its own batch)
registered_pairs_per_s = completed registrations per second, batched
plain     = the same 64 pairs through cvo_register_pair one after another
            (CUDA events around each pass over the 64), and the speedup
e2e       = the batched form through the C ABI with pinned host buffers
            (host to device copies of every pair inside the timed region)
roofline  = the batched sweep kernel (k_sweep, bfloat16 label tile on the
            tensor cores): algorithmic FP32 FLOPs of its in-cutoff pairs over
            its CUDA-event time per launch (the loop queued from the host),
            against the FP32 peak from the unit counts; DRAM traffic and warp
            instructions from the committed ncu summary when it was taken on
            the current kernel source
sections  = street (street-20k single pair), cube (the dense 2,000-point
            pair), backward (room-19k gradients), large (box80-200k), shard
            (box80-200k with X's rows split over the ranks, one NCCL all-reduce
            of the sweep statistics per iteration; N > 1)
cpu_baseline = the FP64 oracle on 8 seeded pairs of the batch (the first
            iteration of each registration), on the host cores

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
FP32_LANES_PER_SM = 128
EX2_PER_CLK_SM = 29   # measured ex2.approx.f32 throughput per SM per clock on a GB300
ISSUE_PER_CLK_SM = 4  # warp instructions per SM per clock (4 schedulers)
CPU_SAMPLE_PAIRS = 8
CSRC = os.path.join(ROOT, "paper_2012_03683_gb300", "csrc")
SWEEP_SRC = [os.path.join(CSRC, "cvo_sweep.cu"), os.path.join(CSRC, "cvo_sweep_dev.cuh")]


def flops_per_pair(blocks):
    """Algorithmic FP32 FLOPs of one in-cutoff pair in the sweep (FMA = 2):
    offset 3, squared distance 5, exponent scale 1, moments W/E/Q 19; a
    squared-exponential block of d entries 3d + 1; an inner-product block of d
    entries 2d - 1 plus the product with the kernel value 1.  The ex2 runs on
    the XU pipe and is not counted."""
    f = 3 + 5 + 1 + 19
    for kind, dim, _, _ in blocks:
        f += 3 * dim + 1 if kind == "se" else 2 * dim
    return f


def grad_flops_per_pair(blocks):
    """Algorithmic FP32 FLOPs of one in-cutoff pair in the gradient sweep:
    offset 3, squared distance 5, exponent scale 1, weight product 1, the
    accumulators sum w e (3 FMA) and sum w d^2 (1 FMA) 8; a squared-
    exponential block of d entries 3d + 1 for its exponent and 3d for its
    accumulator (difference, FMA); an inner-product block 2d for its product
    and 2d for its accumulator."""
    f = 3 + 5 + 1 + 1 + 8
    for kind, dim, _, _ in blocks:
        f += (3 * dim + 1 + 3 * dim) if kind == "se" else 4 * dim
    return f


def with_measured_throughput(cvo, peaks):
    """The peaks with the FP32 FMA and ex2 rates measured on this GPU now
    (cvo_measure_throughput, about 20 ms, outside every timed region); if
    the measurement fails, the unit counts stand in (the roofline's
    peak_source then says so)."""
    out = dict(peaks)
    try:
        t = cvo.cvo_measure_throughput()
    except Exception as e:  # noqa: BLE001 - the bench line must still be printed
        print(f"cvo_measure_throughput failed ({e}); unit-count peaks", file=sys.stderr)
        return out
    out["ffma_flops"] = t["ffma_flops"]
    out["ex2_per_s"] = t["ex2_per_s"]
    return out


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def profile_value(kernel_src, key, profile="sweep_batch-64.md"):
    """A per-launch figure (key: traffic_bytes_per_launch,
    warp_instructions_per_launch, ...) from a committed ncu summary under
    profiles/, if it was taken on the current kernel source (the files in
    kernel_src, hashed in order); else None."""
    path = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    t = re.search(re.escape(key) + r":\s*([0-9.eE+]+)", text)
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


def spread(ms):
    """min / median / max of per-rep times (ms)."""
    a = np.asarray(ms, dtype=np.float64)
    return {"min": float(a.min()), "median": float(np.median(a)), "max": float(a.max()), "reps": int(a.size)}


def batch_workload():
    import scenes
    pairs = scenes.batch_pairs()
    pr = pairs[0].params
    kw = dict(blocks=pairs[0].blocks, ell=pr["ell"], cutoff_mult=pr["cutoff_mult"], max_iters=pr["max_iters"])
    config = {"workload": "batch-64", "pairs": len(pairs),
              "points_per_cloud": "5,000-60,000 (uniform)", "points": int(sum(p.n + p.m for p in pairs)),
              "scene": "4 m cube faces + N(0, 5 mm), motion <= 8 deg / 0.4 m per pair",
              "features": "rgb (squared-exponential, scale 0.2) x 19-class labels (inner product), "
                          "bfloat16 storage, float32 arithmetic",
              "lengthscale": pr["ell"], "cutoff": "3 lengthscales", "max_iters": pr["max_iters"],
              "loop": "one CUDA graph for all pairs (batched sweep + per-pair steps, convergence masks)",
              "l2": "flushed between steps (256 MB write)"}
    return pairs, kw, config


def sample_pairs(n_pairs, k=CPU_SAMPLE_PAIRS, seed=20121203):
    """The indices of the k seeded pairs of the batch the CPU baseline times."""
    r = np.random.Generator(np.random.PCG64(seed))
    return sorted(int(i) for i in r.permutation(n_pairs)[:k])


# ---- sections --------------------------------------------------------------

def sweep_roofline(name, pairs_evaluated, sweep_ms_total, launches, fpp, peaks, peak_src, sms, profile=None):
    """Roofline figures of a sweep kernel from its CUDA-event times."""
    clk = peaks.get("sm_max_mhz", 2070.0) * 1e6
    unit_peak = sms * FP32_LANES_PER_SM * 2 * clk / 1e12
    measured = peaks.get("ffma_flops")
    peak = measured / 1e12 if measured else unit_peak
    sec = sweep_ms_total * 1e-3
    achieved = pairs_evaluated * fpp / sec / 1e12 if sec > 0 else None
    avg_ms = sweep_ms_total / max(launches, 1)
    traffic = winst = xu = issue_active = None
    if profile:
        traffic = profile_value(SWEEP_SRC, "traffic_bytes_per_launch", profile)
        winst = profile_value(SWEEP_SRC, "warp_instructions_per_launch", profile)
        xu = profile_value(SWEEP_SRC, "xu_pipe_frac", profile)
        issue_active = profile_value(SWEEP_SRC, "issue_active_frac", profile)
    issue_peak = sms * ISSUE_PER_CLK_SM * clk
    ex2_measured = peaks.get("ex2_per_s")
    ex2_peak = ex2_measured if ex2_measured else sms * EX2_PER_CLK_SM * clk
    unit_text = f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {clk / 1e6:.0f} MHz (sm_max_mhz {peak_src})"
    return {
        "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
        "frac": achieved / peak if achieved else None, "traffic": traffic, "kernel": name,
        "traffic_source": (f"dram__bytes_read.sum + dram__bytes_write.sum per launch of the committed ncu capture "
                           f"(profiles/{profile}), a launch with every pair running; null when the kernel source "
                           f"changed since") if profile else None,
        "flops_per_pair": fpp, "sweep_ms_avg": avg_ms, "sweep_launches": launches,
        "pairs_per_launch": pairs_evaluated / max(launches, 1),
        "peak_source": (f"of measured: FP32 FMA rate measured in this run on this GPU (cvo_measure_throughput: "
                        f"independent fma.rn.f32 chains, 8 blocks of 256 threads per SM, best of 5 launches); "
                        f"unit count {unit_text} = {unit_peak:.1f} TFLOP/s") if measured
                       else f"unit counts, not a measured FFMA peak: {unit_text}",
        "peak_unit_count": unit_peak,
        "sfu": {"achieved_ex2_per_s": pairs_evaluated / sec if sec > 0 else None, "peak_ex2_per_s": ex2_peak,
                "frac": pairs_evaluated / sec / ex2_peak if sec > 0 else None,
                "ncu_xu_pipe_frac": xu,
                "peak_source": ("of measured: ex2.approx.ftz.f32 rate measured in this run on this GPU "
                                "(cvo_measure_throughput: independent chains, best of 5 launches)") if ex2_measured
                               else (f"{sms} SMs x {EX2_PER_CLK_SM} ex2/clk/SM (measured on a GB300 with an "
                                     "independent-chain ex2.approx throughput loop) x sm_max_mhz")},
        "issue": {"frac": issue_active, "peak_warp_inst_per_s": issue_peak,
                  "warp_instructions_per_launch": winst,
                  "source": (f"smsp__issue_active (share of scheduler cycles issuing) and smsp__inst_executed.sum of "
                             f"the launches of the committed ncu capture (profiles/{profile}, same source hash); "
                             if profile else "no committed capture read for this kernel; ")
                            + f"peak {sms} SMs x {ISSUE_PER_CLK_SM} schedulers x sm_max_mhz"},
    }


def parse_tuning(text):
    """--tuning "cell_factor,super_delta,chunk_len[,query_lanes]" as apply_tuning's arguments."""
    parts = text.split(",")
    return (float(parts[0]), int(parts[1]), int(parts[2]), int(parts[3]) if len(parts) > 3 else 1)


def tuning_args(t):
    return (t["cell_factor"], t["super_delta"], t["chunk_len"], t.get("query_lanes", 1))


def plain_section(h, args, torch, flush, reps):
    """The 64 pairs through cvo_register_pair one after another; CUDA events
    around each pass over the batch."""
    stream = torch.cuda.current_stream()
    for a in args[:2]:
        h.register(*a)
    ms, evals = [], 0
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        n = 0
        for a in args:
            _, info = h.register(*a)
            n += info["pairs"]
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        evals += n
    t = sum(ms) * 1e-3
    return {"registered_pairs_per_s": reps * len(args) / t, "pair_evals_per_s": evals / t,
            "ms_per_batch": spread(ms), "timing": "CUDA events around each pass of 64 cvo_register_pair calls"}


def street_section(cvo, torch, dev, flush, peaks, peak_src, sms, reps=10, tuning=None):
    """street-20k: one registration of the 20,000-point street pair (RGB +
    labels in float32, l 0.3 -> 0.05 m annealed, cutoff 3 l, <= 100
    iterations), autotuned, graph loop; then the same registrations with the
    sweep timed per launch."""
    import scenes
    p = scenes.street_pair()
    pr = p.params
    kw = dict(blocks=p.blocks, ell=pr["ell"], ell_min=pr["ell_min"], cutoff_mult=pr["cutoff_mult"],
              max_iters=pr["max_iters"], anneal=pr["anneal"])
    X, Z = torch.tensor(p.X, device=dev), torch.tensor(p.Z, device=dev)
    FX, FZ = torch.tensor(p.FX, device=dev), torch.tensor(p.FZ, device=dev)
    out = {"workload": f"street-20k: {p.n} + {p.m} points, rgb + 19 labels (float32), l 0.3 -> 0.05 m, cutoff 3 l, "
                       f"<= {pr['max_iters']} iterations"}
    stream = torch.cuda.current_stream()
    with cvo.CVO(**kw) as h:
        if tuning:
            h.apply_tuning(*tuning)
            out["tuning"] = dict(h.tuning(), source="--tuning")
        else:
            out["tuning"] = h.autotune(X, Z, np.eye(4), FX, FZ)
        for _ in range(3):
            h.register(X, Z, np.eye(4), FX, FZ)
        ms, pairs, iters = [], 0, []
        for _ in range(reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            T, info = h.register(X, Z, np.eye(4), FX, FZ)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            pairs += info["pairs"]
            iters.append(info["iters"])
        cvo.cvo_set_timing(h.h, True)
        sw_ms, sw_n, sw_pairs = 0.0, 0, 0
        for _ in range(reps):
            flush.zero_()
            _, inf2 = h.register(X, Z, np.eye(4), FX, FZ)
            a, n = cvo.cvo_sweep_time(h.h)
            sw_ms += a * n
            sw_n += n
            sw_pairs += inf2["pairs"]
        cvo.cvo_set_timing(h.h, False)
    t = sum(ms) * 1e-3
    D = np.linalg.inv(T) @ p.T_true
    out.update({"pair_evals_per_s": pairs / t, "registered_pairs_per_s": reps / t, "ms_per_registration": spread(ms),
                "iterations": iters, "ell_final": info["ell_final"], "status": info["status"],
                "pose_err_vs_truth": {"rot_rad": float(math.acos(max(-1.0, min(1.0, (np.trace(D[:3, :3]) - 1) / 2)))),
                                      "trans_m": float(np.linalg.norm(D[:3, 3]))},
                "roofline": sweep_roofline("k_sweep<FeatFixed<3,19,float32>>", sw_pairs, sw_ms, sw_n,
                                           flops_per_pair(p.blocks), peaks, peak_src, sms,
                                           profile="sweep_street-20k.md")})
    return out


def cube_section(cvo, torch, dev, flush, reps=10):
    """The dense cube pair (2,000 points per cloud, RGB, l = 0.1, every pair,
    50 iterations): registration latency between CUDA events."""
    import scenes
    p = scenes.cube_pair()
    pr = p.params
    kw = dict(blocks=p.blocks, ell=pr["ell"], cutoff_mult=pr["cutoff_mult"], max_iters=pr["max_iters"])
    X, Z = torch.tensor(p.X, device=dev), torch.tensor(p.Z, device=dev)
    FX, FZ = torch.tensor(p.FX, device=dev), torch.tensor(p.FZ, device=dev)
    stream = torch.cuda.current_stream()
    with cvo.CVO(**kw) as h:
        for _ in range(3):
            h.register(X, Z, np.eye(4), FX, FZ)
        ms, pairs = [], 0
        for _ in range(reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            T, info = h.register(X, Z, np.eye(4), FX, FZ)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            pairs += info["pairs"]
    t = sum(ms) * 1e-3
    D = np.linalg.inv(T) @ p.T_true
    return {"workload": f"cube-2000: {p.n} + {p.m} points, rgb, l = 0.1, dense, {pr['max_iters']} iterations",
            "ms_per_registration": spread(ms), "pair_evals_per_s": pairs / t, "iterations": info["iters"],
            "pose_err_vs_truth": {"rot_rad": float(math.acos(max(-1.0, min(1.0, (np.trace(D[:3, :3]) - 1) / 2)))),
                                  "trans_m": float(np.linalg.norm(D[:3, 3]))}}


def backward_section(cvo, torch, dev, flush, peaks, peak_src, sms, reps=5):
    """Room pair (19,200 points per cloud, rgb, l = 0.1, cutoff 3 l): one
    forward evaluation and one backward pass (gradients for both clouds'
    points and features and for l, device outputs), CUDA-event timed; the
    gradient sweeps also per launch."""
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
        t = {"forward": [], "backward": []}
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
                t[name].append(e0.elapsed_time(e1))
        cvo.cvo_set_timing(h.h, True)
        g_ms, g_n = 0.0, 0
        for _ in range(reps):
            flush.zero_()
            h.backward(X, Z, T, FX, FZ)
            a, n = cvo.cvo_sweep_time(h.h)
            g_ms += a * n
            g_n += n
        cvo.cvo_set_timing(h.h, False)
    out["pairs"] = int(ev["pairs"])
    out["ms_forward"] = spread(t["forward"])
    out["ms_backward"] = spread(t["backward"])
    # the backward sweeps every in-cutoff pair twice (once per cloud)
    out["backward_pair_evals_per_s"] = 2 * ev["pairs"] / (1e-3 * float(np.median(t["backward"])))
    out["timing"] = "whole calls (setup, sweeps, copies) between CUDA events, L2 flushed before each"
    out["roofline"] = sweep_roofline("k_grad + k_grad_reduce (gradient sweep, one per cloud)", ev["pairs"] * g_n,
                                     g_ms, g_n, grad_flops_per_pair(p.blocks), peaks, peak_src, sms,
                                     profile="grad_room-19k.md")
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
    out.update({"ms_per_registration": spread(ms), "iterations": info["iters"], "status": info["status"],
                "ell_final": info["ell_final"], "i_theta": info["i_theta"], "pairs": info["pairs"],
                "pair_evals_per_s": info["pairs"] / (1e-3 * float(np.mean(ms))),
                "pose_err_vs_truth": {"rot_rad": float(math.acos(max(-1.0, min(1.0, (np.trace(D[:3, :3]) - 1) / 2)))),
                                      "trans_m": float(np.linalg.norm(D[:3, 3]))}})
    return out


def shard_section(cvo, torch, dev, dist, world, rank, flush, reps=2):
    """box80-200k with X's rows split over the ranks (one GPU each) and Z on
    every rank: per iteration each rank sweeps its rows, one NCCL all-reduce
    sums the 45 statistics, and every rank takes the same step.  Latency of
    the whole registration between a barrier and CUDA events, max over
    ranks."""
    import scenes
    p = scenes.large_pair()
    pr = p.params
    kw = dict(blocks=p.blocks, ell=pr["ell"], ell_min=pr["ell_min"], cutoff_mult=pr["cutoff_mult"],
              max_iters=pr["max_iters"], anneal=pr["anneal"])
    lo, hi = cvo.shard_rows(p.n, world, rank)
    Xr, FXr = torch.tensor(p.X[lo:hi], device=dev), torch.tensor(p.FX[lo:hi], device=dev)
    Z, FZ = torch.tensor(p.Z, device=dev), torch.tensor(p.FZ, device=dev)
    stream = torch.cuda.current_stream()
    ms = []
    with cvo.CVO(**kw) as h:
        h.register_sharded(Xr, Z, p.n, np.eye(4), FXr, FZ, allreduce=dist.all_reduce)
        for _ in range(reps):
            flush.zero_()
            dist.barrier()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            T, info = h.register_sharded(Xr, Z, p.n, np.eye(4), FXr, FZ, allreduce=dist.all_reduce)
            e1.record(stream)
            e1.synchronize()
            ms.append(max_over_ranks(dist, world, e0.elapsed_time(e1), dev))
    return {"workload": f"box80-200k split by rows of X over {world} GPUs (NCCL all-reduce of 45 statistics per "
                        "iteration)", "ms_per_registration": spread(ms), "iterations": info["iters"],
            "ell_final": info["ell_final"], "status": info["status"], "pairs": info["pairs"],
            "pair_evals_per_s": info["pairs"] / (1e-3 * float(np.median(ms)))}


def cpu_baseline(pairs, kw, iters=1):
    """The FP64 oracle's registration of 8 seeded pairs of the batch, first
    iteration(s) each, on all host cores."""
    import oracle
    oracle.build()
    idx = sample_pairs(len(pairs))
    total, evals = 0.0, 0
    for k in idx:
        p = pairs[k]
        t0 = time.perf_counter()
        _, info, _ = oracle.register(p.X, p.Z, np.eye(4), FX=p.FX, FZ=p.FZ, **dict(kw, max_iters=iters))
        total += time.perf_counter() - t0
        evals += info["pairs_total"]
    return {"value": evals / total, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"the first {iters} iteration(s) of the FP64 oracle's registration of {len(idx)} seeded pairs "
                      f"of batch-64 (pairs {idx}; {evals} in-cutoff pairs, {total:.1f} s), per pair-eval",
            "seconds": total}


def run_reference(args):
    """The oracle as the reference arm: each step is a bounded sample of the
    same workload (the first iteration of the oracle's registration of one of
    the 8 seeded pairs of the batch, in turn)."""
    dist, world, rank, _ = dist_setup("gloo")
    if rank != 0:
        return
    pairs, kw, config = batch_workload()
    import oracle
    oracle.build()
    idx = sample_pairs(len(pairs))

    def step(s):
        p = pairs[idx[s % len(idx)]]
        _, info, _ = oracle.register(p.X, p.Z, np.eye(4), FX=p.FX, FZ=p.FZ, **dict(kw, max_iters=1))
        return info["pairs_total"]

    for s in range(args.warmup):
        step(s)
    evals, total = 0, 0.0
    for s in range(args.steps):
        t0 = time.perf_counter()
        evals += step(s)
        total += time.perf_counter() - t0
    value = evals / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config,
            "cpu_baseline": {"kind": "oracle", "cores": oracle.num_threads(), "value": value, "unit": UNIT,
                             "sample": f"each step: the first iteration of the FP64 oracle's registration of one of "
                                       f"the pairs {idx} of batch-64, in turn"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cvo", choices=["cvo", "reference"])
    ap.add_argument("--reps", type=int, default=10, help="repetitions of the plain pass and of the timed sweeps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sections", action="store_true", help="only the batched headline")
    ap.add_argument("--no-street", action="store_true")
    ap.add_argument("--no-cube", action="store_true")
    ap.add_argument("--no-backward", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--only", default=None, choices=["street", "cube", "backward", "large"],
                    help="run only this section and print its JSON (a fixed launch sequence for profiling)")
    ap.add_argument("--tuning", default=None,
                    help="cell_factor,super_delta,chunk_len[,query_lanes] for the batch (or, with --only street, the "
                         "street pair) instead of autotuning (fixed launch sequence for profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import paper_2012_03683_gb300 as cvo

    dist, world, rank, local = dist_setup("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    if args.only:
        peaks, peak_src = load_peaks()
        peaks = with_measured_throughput(cvo, peaks)
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
        tun = None
        if args.tuning:
            tun = parse_tuning(args.tuning)
        run = {"street": lambda: street_section(cvo, torch, dev, flush, peaks, peak_src, sms, reps=args.reps,
                                                tuning=tun),
               "cube": lambda: cube_section(cvo, torch, dev, flush, reps=args.reps),
               "backward": lambda: backward_section(cvo, torch, dev, flush, peaks, peak_src, sms, reps=args.reps),
               "large": lambda: large_section(cvo, torch, dev, flush, reps=args.reps)}[args.only]
        print(json.dumps({args.only: run()}), flush=True)
        return
    pairs, kw, config = batch_workload()
    config["parallelism"] = f"replicas x{world}" if world > 1 else "one GPU"
    args_dev = [(torch.tensor(p.X, device=dev), torch.tensor(p.Z, device=dev), np.eye(4),
                 torch.tensor(p.FX, device=dev).to(torch.bfloat16), torch.tensor(p.FZ, device=dev).to(torch.bfloat16))
                for p in pairs]
    h = cvo.CVO(**kw)
    # cell size, query-group extent and item length (untimed, before the
    # warm-up): the plain form's tuned on the largest pair registered alone,
    # the batch's on the batch itself (its grid holds every pair's items, so
    # it prefers longer ones)
    if args.tuning:
        h.apply_tuning(*parse_tuning(args.tuning))
        tuning = tuning_plain = dict(h.tuning(), source="--tuning")
    else:
        big = max(range(len(pairs)), key=lambda k: pairs[k].n + pairs[k].m)
        tuning_plain = dict(h.autotune(*args_dev[big]), source=f"autotuned on pair {big}")
        tuning = dict(h.autotune_batch(args_dev), source="autotuned on the batch (cvo_autotune_batch)")
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    for _ in range(max(args.warmup, 3)):
        h.register_batch(args_dev)
    torch.cuda.synchronize()

    # ---- timed region: batched registrations, device-resident inputs --------
    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = cvo.cvo_kernel_launches()
    step_ms, evals, conv, iters, tests = [], 0, 0, [], 0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, infos, _ = h.register_batch(args_dev)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        evals += sum(i["pairs"] for i in infos)
        tests += sum(i["candidates"] for i in infos)
        conv += sum(1 for i in infos if i["status"] == 0)
        iters = [i["iters"] for i in infos]
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = cvo.cvo_kernel_launches() - launches0
    clocks = sampler.stop()
    total_ms = float(sum(step_ms))
    total_ms_max = max_over_ranks(dist, world, total_ms, dev)
    evals_all = sum_over_ranks(dist, world, float(evals), dev)
    value = evals_all / (total_ms_max * 1e-3)
    regs_per_s = world * args.steps * len(pairs) / (total_ms_max * 1e-3)

    # ---- the batched sweep per launch: the same registrations with the loop
    # queued from the host and CUDA events around every sweep launch
    cvo.cvo_set_timing(h.h, True)
    sw_ms, sw_n, sw_evals = 0.0, 0, 0
    for _ in range(args.reps):
        flush.zero_()
        _, infos, _ = h.register_batch(args_dev)
        a, n = cvo.cvo_sweep_time(h.h)
        sw_ms += a * n
        sw_n += n
        sw_evals += sum(i["pairs"] for i in infos)
    cvo.cvo_set_timing(h.h, False)

    # ---- the plain form: the same pairs one by one -----------------------------
    if rank == 0:
        h.apply_tuning(*tuning_args(tuning_plain))
        plain = plain_section(h, args_dev, torch, flush, args.reps)
        plain["tuning"] = tuning_plain
        h.apply_tuning(*tuning_args(tuning))
    else:
        plain = None

    # ---- end to end: pinned host buffers through the C ABI ------------------
    args_host = [(torch.tensor(p.X).pin_memory(), torch.tensor(p.Z).pin_memory(), np.eye(4),
                  torch.tensor(p.FX).to(torch.bfloat16).pin_memory(),
                  torch.tensor(p.FZ).to(torch.bfloat16).pin_memory()) for p in pairs]
    h2d = sum(t.numel() * t.element_size() for a in args_host for t in (a[0], a[1], a[3], a[4]))
    import ctypes
    d2h = len(pairs) * (16 * 8 + ctypes.sizeof(cvo.Info))
    h.register_batch(args_host)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e2e_ms, e2e_evals = 0.0, 0
    for _ in range(max(1, args.steps // 3)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, infos, _ = h.register_batch(args_host)
        torch.cuda.synchronize()
        e2e_ms += 1e3 * (time.perf_counter() - t0)
        e2e_evals += sum(i["pairs"] for i in infos)
    e2e_ms = max_over_ranks(dist, world, e2e_ms, dev)
    e2e_evals = sum_over_ranks(dist, world, float(e2e_evals), dev)
    h.close()

    peaks, peak_src = load_peaks()
    peaks = with_measured_throughput(cvo, peaks)
    sections = {}
    if world > 1 and not args.no_sections and not args.no_large:
        sections["shard"] = shard_section(cvo, torch, dev, dist, world, rank, flush)
    if rank == 0 and not args.no_sections:
        if not args.no_street:
            sections["street"] = street_section(cvo, torch, dev, flush, peaks, peak_src, sms)
        if not args.no_cube:
            sections["cube"] = cube_section(cvo, torch, dev, flush)
        if not args.no_backward:
            sections["backward"] = backward_section(cvo, torch, dev, flush, peaks, peak_src, sms)
        if not args.no_large:
            sections["large"] = large_section(cvo, torch, dev, flush)
    if rank != 0:
        return

    roof = sweep_roofline("k_sweep<FeatMMA<3>> (batched sweep, bfloat16 label tile on the tensor cores)", sw_evals,
                          sw_ms, sw_n, flops_per_pair(kw["blocks"]), peaks, peak_src, sms,
                          profile="sweep_batch-64.md")
    roof["timing"] = ("CUDA events around each batched sweep launch, over the same batched registrations queued "
                      "from the host (the timed steps run the loop as one CUDA graph)")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "storage": "bf16 features", "data": "synthetic",
        "config": config,
        "registered_pairs_per_s": regs_per_s,
        "ms_per_batch": spread(step_ms),
        "pair_evals_per_batch": evals / args.steps,
        # the sweep's (query, candidate) distance tests per in-cutoff pair: the
        # candidates its streams examine beyond the pairs the method counts
        "sweep_tests_per_pair": tests / max(evals, 1),
        "converged_per_batch": conv / args.steps,
        "iterations": iters,
        "plain": plain,
        "batched_vs_plain": (regs_per_s / world) / plain["registered_pairs_per_s"] if plain else None,
        "e2e": {"value": e2e_evals / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "tuning": tuning,
        "roofline": roof,
        "clocks": clocks,
        "sm_count": sms,
    }
    line.update(sections)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(pairs, kw)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
