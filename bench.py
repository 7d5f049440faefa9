#!/usr/bin/env python3
"""Benchmark of the BOAC hot path: batched Bayesian-optimisation candidate
evaluation (rasterise mu -> 50 MLEM iterations -> Poisson score) at 128x128
pixels, 120 views, 128 bins, 256 candidates per GPU.

One step = the whole hot path for one batch: boac_rasterize_mu (Eq. 3-4) and
boac_mlem (sensitivity, 50 fused MLEM iterations, Eq. 5 score) for all 256
candidates.  Metric: candidate-iterations per second (256 * 50 per step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
(the only reference this paper has: it publishes no code) on the host cores.
Multi-GPU (torchrun): every rank evaluates its own 256 candidates (weak
scaling, no collective on the data path); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2109_11920_gb300 import synth  # noqa: E402

WL = synth.BATCHED
METRIC = "MLEM candidate-iterations/sec at 128x128x120 views and % HBM roofline vs plain GPU path"
UNIT = "candidate-iterations/s"
CONFIG = {
    "workload": f"{WL.name}: {WL.B} BO candidates x {WL.K} MLEM iterations, "
                f"{WL.n}x{WL.n} px of {WL.dx} cm, {WL.V} views over 360 deg, {WL.n} bins, "
                f"{WL.counts:.0e} counts, shared sinogram",
    "candidates_per_gpu": WL.B,
    "iterations": WL.K,
    "image": WL.n,
    "views": WL.V,
    "bins": WL.n,
    "l2": "flushed (256 MiB write) before every timed step; per-step CUDA events summed",
}
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
PROFILE_FILE = os.path.join(ROOT, "profiles", "mlem_fused_bo_batch128_v120.md")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ----------------------------------------------------------------- inputs
def make_inputs_gpu(dev, boac, Geom, Tissue, seed=0):
    """Synthetic workload built on the device: true head (Legendre c_true) ->
    rasterised mu -> phantom (brain 1.0, four ellipses 4.0) -> projected,
    scaled to the count level, Poisson noise -> 256 perturbed candidates."""
    import torch
    g = Geom.make(WL.n, WL.dx, WL.V)
    t = Tissue(*synth.TISSUE)
    ph, noise, cand = synth.streams(seed)
    c_true = torch.tensor([synth.C_TRUE], dtype=torch.float32, device=dev)
    mu_true = boac.boac_rasterize_mu(g, t, c_true)
    brain = (mu_true[0] == np.float32(synth.TISSUE[0])).cpu().numpy()
    F_true = synth.paint_activity(WL.n, float(np.float32(WL.dx)), brain, synth.ellipses(ph, synth.C_TRUE[0]))
    q = boac.boac_project(g, mu_true, torch.tensor(F_true[None], dtype=torch.float32, device=dev))
    S = synth.poisson_sinogram(noise, q[0].double().cpu().numpy(), WL.counts)
    coefs = synth.candidates(cand, WL.B).astype(np.float32)
    return g, t, coefs, S.astype(np.float32)


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- helpers
def measured_peak_gbs():
    try:
        with open(PEAKS_FILE) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def fused_source_hash():
    h = hashlib.sha256()
    for f in ("boac_fused.cu", "boac_device.cuh", "boac_sched.cuh"):
        with open(os.path.join(ROOT, "paper_2109_11920_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_bytes(key="dram_bytes_per_launch_full_size"):
    """A per-launch byte count of the fused kernel (DRAM or L2) read from the
    committed ncu summary -- the bench does not run ncu itself -- if that
    summary was taken on the current kernel source (else None)."""
    try:
        text = open(PROFILE_FILE).read()
    except OSError:
        return None
    m_src = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]{16})", text)
    m_b = re.search(key + r":\s*([0-9.eE+]+)", text)
    if not m_src or not m_b or m_src.group(1) != fused_source_hash():
        return None
    return float(m_b.group(1))


def profiled_traffic():
    return profiled_bytes("dram_bytes_per_launch_full_size")


# FP32 work per ray sample per view per iteration: two bilinear gathers (F and
# mu), the attenuation scan and exponential, the accumulation, and the
# transposed bilinear scatter of the back-projection.
FLOPS_PER_SAMPLE = 50


def sm_max_mhz():
    """Maximum SM clock: the measured-peaks file's figure, else nvidia-smi's."""
    try:
        with open(PEAKS_FILE) as fh:
            return float(json.load(fh)["sm_max_mhz"]), "MEASURED_PEAKS.json sm_max_mhz"
    except (OSError, KeyError, ValueError):
        pass
    try:
        out = subprocess.run(["nvidia-smi", "--id=0", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=20).stdout.strip().splitlines()
        return float(out[0]), "nvidia-smi clocks.max.sm"
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        return 2070.0, "nominal 2070 MHz"


_FP32 = {}


def fp32_peak(dev=None):
    """FP32 FMA rate of the device: SMs (read from the device) x 128 FP32
    lanes x 2 flop x the maximum SM clock.  Returns (TFLOP/s, description)."""
    if "v" not in _FP32:
        import torch
        d = dev if dev is not None else torch.device("cuda", torch.cuda.current_device())
        sms = torch.cuda.get_device_properties(d).multi_processor_count
        mhz, src = sm_max_mhz()
        _FP32["v"] = (sms * 128 * 2 * mhz * 1e6 / 1e12,
                      f"derived: {sms} SMs (device) x 128 FP32 lanes x 2 flop x {mhz:.0f} MHz ({src})")
    return _FP32["v"]


def fp32_peak_tflops(dev=None):
    return fp32_peak(dev)[0]


def l2_probe_gbs(dev, mib=24, reps=20):
    """L2 bandwidth probe: a copy of a buffer pair that stays resident in L2
    (2 x 24 MiB, well under the 129 MB L2), timed with CUDA events after
    warm-up; read + write bytes over time, best of 3."""
    import torch
    n = (mib << 20) // 4
    a = torch.ones(n, dtype=torch.float32, device=dev)
    b = torch.empty_like(a)
    for _ in range(5):
        b.copy_(a)
    torch.cuda.synchronize(dev)
    best = float("inf")
    st = torch.cuda.current_stream(dev)
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            b.copy_(a)
        e1.record(st)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / reps)
    return 2.0 * n * 4 / (best / 1e3) / 1e9


def algorithmic_bytes_per_cand_iter(n, V):
    """Per candidate-iteration: the attenuation table read in the forward and
    in the backward pass (2 x 4 V n^2 bytes), plus F read+write, sens read
    (3 x 4 n^2) and the sinogram (4 V n)."""
    return 8.0 * V * n * n + 4.0 * (3 * n * n + V * n)


# ----------------------------------------------------------------- ranks
def max_over_ranks(x: float, world: int) -> float:
    """Largest value of x over all ranks (the job's wall time); identity at N=1."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(world: int, per_rank_units: int, steps: int, max_ms: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * per_rank_units * steps / (max_ms / 1e3)


# ----------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    import oracle
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    K_ref = 20
    import sys as _s
    _s.path.insert(0, os.path.join(ROOT, "tests"))
    from problems import make_problem
    p = make_problem(WL.n, WL.dx, WL.V, WL.counts, B=cores, seed=WL.seed)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        _, _, used = oracle.mlem_batch(p.geom, p.mu, p.S, K_ref, with_score=True, nthreads=cores)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = cores * K_ref * len(times) / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": CONFIG,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                         "sample": f"per step {cores} candidates x {K_ref} MLEM iterations + score "
                                   f"of the {WL.n}x{WL.n}/{WL.V}-view batch, one candidate per thread",
                         "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_model() -> str:
    """The host CPU's model name (/proc/cpuinfo; on Arm the implementer and
    part codes when no name is given), else the machine type."""
    import platform
    fields = {}
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ":" in ln:
                    k, v = ln.split(":", 1)
                    fields.setdefault(k.strip().lower(), v.strip())
    except OSError:
        pass
    if fields.get("model name"):
        return fields["model name"]
    if fields.get("cpu part"):
        return f"{platform.machine()} (implementer {fields.get('cpu implementer', '?')}, part {fields['cpu part']})"
    return platform.machine() or "unknown"


def cpu_baseline_sample(dev=None):
    """The oracle as it stands, timed on this host's cores (bounded sample);
    the same candidates through the CUDA path give its error against the
    oracle (images after the full iteration count, scores)."""
    import oracle
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from problems import make_problem
    cores = os.cpu_count() or 1
    K = WL.K
    B = 4 * cores
    p = make_problem(WL.n, WL.dx, WL.V, WL.counts, B=B, seed=WL.seed)
    t0 = time.perf_counter()
    Fo, Lo, used = oracle.mlem_batch(p.geom, p.mu, p.S, K, with_score=True, nthreads=cores)
    dt = time.perf_counter() - t0
    # the same code on one thread: one candidate of the sample
    t1 = time.perf_counter()
    oracle.mlem_batch(p.geom, p.mu[:1], p.S, K, with_score=True, nthreads=1)
    dt1 = time.perf_counter() - t1
    out = {"value": B * K / dt, "unit": UNIT, "cores": used, "kind": "oracle",
           "sample": f"{B} candidates x {K} MLEM iterations + score of the "
                     f"{WL.n}x{WL.n}/{WL.V}-view batch (FP64 C, candidates spread over "
                     f"{used} threads), {dt:.1f} s wall",
           "cpu_model": cpu_model(), "host_threads": cores,
           "value_1thread": K / dt1, "sample_1thread": f"1 candidate x {K} iterations + score, {dt1:.1f} s"}
    if dev is not None:
        import torch
        from paper_2109_11920_gb300 import Geom
        from paper_2109_11920_gb300 import api as boac
        g = Geom.make(p.n, p.dx, p.V)
        F = torch.ones(B, p.n, p.n, device=dev)
        F, L = boac.boac_mlem(g, torch.tensor(p.mu, dtype=torch.float32, device=dev),
                              torch.tensor(p.S, dtype=torch.float32, device=dev), F, K)
        F, L = F.double().cpu().numpy(), L.cpu().numpy()
        img = [float(np.linalg.norm(F[b] - Fo[b]) / np.linalg.norm(Fo[b])) for b in range(B)]
        out["error_vs_oracle"] = {"image_rel_l2_max": max(img),
                                  "score_rel_max": float(np.max(np.abs(L - Lo) / np.abs(Lo))),
                                  "candidates": B, "iterations": K}
    return out


# ----------------------------------------------------------------- GPU arm
def run_gpu(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_2109_11920_gb300 import Geom, Tissue
    from paper_2109_11920_gb300 import api as boac
    from paper_2109_11920_gb300 import build as pkg_build

    pkg_build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    g, t, coefs, S_np = make_inputs_gpu(dev, boac, Geom, Tissue, seed=WL.seed + rank)
    B, K = args.candidates, args.iters
    coefs = coefs[:B] if B <= len(coefs) else np.resize(coefs, (B, 6))
    c_d = torch.tensor(coefs, device=dev)
    S_d = torch.tensor(S_np, device=dev)
    mu = torch.empty(B, WL.n, WL.n, device=dev)
    F = torch.empty(B, WL.n, WL.n, device=dev)
    L = torch.empty(B, dtype=torch.float64, device=dev)
    ws = boac.workspace(g, B, boac._lib.OP_MLEM, dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(ev_k=None, check=False):
        boac.boac_rasterize_mu(g, t, c_d, out=mu)
        F.fill_(1.0)
        if ev_k is not None:
            ev_k[0].record(stream)
        # check: the public call's default (wait, then raise on a failed
        # device status); the device-timed loop keeps the launches queued
        # back to back and checks the status word once after it
        boac.boac_mlem(g, mu, S_d, F, K, score=True, ws=ws, L=L, check_status=check)
        if ev_k is not None:
            ev_k[1].record(stream)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    ev = [(E(), E()) for _ in range(args.steps)]
    evk = [(E(), E()) for _ in range(args.steps)]
    barrier()
    with ClockSampler(local_rank) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            step(evk[i])
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
    barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    kern_ms = [a.elapsed_time(b) for a, b in evk]
    tot_ms = max_over_ranks(sum(step_ms), world)
    value = weak_scaling_value(world, B * K, args.steps, tot_ms)
    assert torch.isfinite(L).all(), "non-finite score"
    boac._raise_on_device_status("boac_mlem", ws)

    # ---- end to end through the public API with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        e2e = e2e_timing(args, world, dev, stream, step, c_d, S_d, L, F, coefs, S_np, flush, B, K)
    if rank != 0:
        return
    plain = None if args.no_plain else plain_timing(g, boac, mu, S_d, dev, stream, K)
    grad = None if args.no_plain else grad_timing(g, t, boac, c_d, S_d, dev, stream)
    l2_gbs = l2_probe_gbs(dev)

    # ---- roofline of the dominant kernel (the fused MLEM kernel)
    kavg_s = sum(kern_ms) / len(kern_ms) / 1e3
    cand_its = B * K
    traffic = profiled_traffic() if (B, K) == (WL.B, WL.K) else None
    # On-chip bound (ALU/issue): the algorithm's FP32 work per candidate-
    # iteration against the FP32 FMA rate of the part.
    flops = FLOPS_PER_SAMPLE * WL.V * WL.n * WL.n * cand_its
    fp32_pk, fp32_kind = fp32_peak(dev)
    achieved = flops / kavg_s / 1e12
    roof = {"bound": "alu", "kernel": "mlem_fused_kernel<128,1024,4 views per grid>",
            "achieved": achieved, "peak": fp32_pk, "unit": "TFLOP/s", "frac": achieved / fp32_pk,
            "traffic": traffic,
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one full-size launch, "
                              "read from the committed profile summary while the kernel source is unchanged "
                              "(null otherwise)",
            "peak_kind": fp32_kind,
            "work_model": f"{FLOPS_PER_SAMPLE} FP32 ops per ray sample per view per iteration",
            "algorithmic_flops_per_launch": flops, "kernel_ms": 1e3 * kavg_s,
            "timed": "CUDA events around boac_mlem on its stream: the scatter-schedule check (a build "
                     "only on the geometry's first call) and tag kernels, the two small kernels that sum "
                     "the shared sinogram's ln S! term and the fused kernel"}
    peak, peak_kind = measured_peak_gbs()
    alg = algorithmic_bytes_per_cand_iter(WL.n, WL.V) * cand_its
    # What-if: the same launch against HBM, counting the bytes the
    # materialised-table algorithm would move (table read in the forward and
    # the backward pass).  The kernel does not move these bytes.
    hbm = {"what_if": "materialised-table algorithm's bytes over this kernel's time (not an achieved rate)",
           "achieved": alg / kavg_s / 1e9, "peak": peak, "unit": "GB/s",
           "frac": alg / kavg_s / 1e9 / peak, "peak_kind": f"{peak_kind} hbm_gbs (copy)",
           "algorithmic_bytes_per_launch": alg,
           "dram_bytes_per_launch": traffic}
    # Measured memory traffic of the launch against the measured peaks.
    l2_bytes = profiled_bytes("l2_bytes_per_launch_full_size") if (B, K) == (WL.B, WL.K) else None
    mem = {"dram": None if traffic is None else
           {"bytes_per_launch": traffic, "achieved_gbs": traffic / kavg_s / 1e9, "peak_gbs": peak,
            "frac": traffic / kavg_s / 1e9 / peak, "peak_kind": f"{peak_kind} hbm_gbs (copy)"},
           "l2": {"probe_gbs": l2_gbs,
                  "probe": "L2-resident copy (2 x 24 MiB, read + write bytes), CUDA events, this run",
                  "bytes_per_launch": l2_bytes,
                  "achieved_gbs": None if l2_bytes is None else l2_bytes / kavg_s / 1e9,
                  "frac": None if l2_bytes is None else l2_bytes / kavg_s / 1e9 / l2_gbs,
                  "bytes_source": "ncu lts__t_bytes.sum of one full-size launch from the committed "
                                  "profile summary (null when the kernel source changed)"}}
    config = dict(CONFIG, global_batch=world * B, parallelism=f"replicas{world}")
    if (B, K) != (WL.B, WL.K):
        config["reduced_case"] = f"{B} candidates x {K} iterations (not the benchmark workload)"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config,
        "roofline": roof,
        "roofline_hbm": hbm,
        "memory_traffic": mem,
        "e2e": e2e,
        # per step: rasterize_kernel, lgamma_partial_kernel, lgamma_final_kernel,
        # scatter_schedule_kernel (returns at once once the schedule is cached),
        # sched_tag_kernel and mlem_fused_kernel
        "gpu_launches": 6 * args.steps,
        "clocks": clk.summary(),
    }
    if plain is not None:
        line["plain_path"] = dict(plain, speedup_of_batched=value / world / plain["value"])
    if grad is not None:
        line["differentiable_score"] = grad
    if world == 1 and not args.no_workloads:
        # the other workloads of the hot path, each on its own inputs
        # (default launch shapes: what boac_mlem / boac_mlem_ragged pick)
        line["workloads"] = {name: workload_summary(workload_line(name, args, dev, tune=False))
                             for name in ("grad", "ragged", "large")}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample(dev)
    print(json.dumps(line), flush=True)


def e2e_timing(args, world, dev, stream, step, c_d, S_d, L, F, coefs, S_np, flush, B, K):
    """Same metric through the public API with pinned host buffers: H2D of the
    coefficients and sinogram, the step, D2H of the scores and images."""
    import torch
    import torch.distributed as dist
    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    c_h = torch.tensor(coefs).pin_memory()
    S_h = torch.tensor(S_np).pin_memory()
    L_h = torch.empty(B, dtype=torch.float64).pin_memory()
    F_h = torch.empty(B, WL.n, WL.n).pin_memory()

    def e2e_step():
        c_d.copy_(c_h, non_blocking=True)
        S_d.copy_(S_h, non_blocking=True)
        step(check=True)
        L_h.copy_(L, non_blocking=True)
        F_h.copy_(F, non_blocking=True)

    for _ in range(max(1, args.warmup // 2)):
        e2e_step()
    torch.cuda.synchronize(dev)
    e_ms = []
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        a, b = E(), E()
        a.record(stream)
        e2e_step()
        b.record(stream)
        b.synchronize()
        e_ms.append(a.elapsed_time(b))
    e_tot = max_over_ranks(sum(e_ms), world)
    return {"value": weak_scaling_value(world, B * K, args.steps, e_tot), "unit": UNIT,
            "h2d_bytes_per_step": c_h.numel() * 4 + S_h.numel() * 4,
            "d2h_bytes_per_step": L_h.numel() * 8 + F_h.numel() * 4}


def grad_timing(g, t, boac, c_d, S_d, dev, stream):
    """Score and d lnP / dc through unrolled MLEM (64 candidates, 10
    iterations, checkpoint every 2): candidate-iterations per second."""
    import torch
    wl = synth.GRAD
    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    c = c_d[:wl.B].contiguous()
    boac.boac_score_grad(g, t, c, S_d, wl.K, wl.extra["ckpt_every"])
    torch.cuda.synchronize(dev)
    a, b = E(), E()
    a.record(stream)
    boac.boac_score_grad(g, t, c, S_d, wl.K, wl.extra["ckpt_every"])
    b.record(stream)
    b.synchronize()
    return {"value": wl.B * wl.K / (a.elapsed_time(b) / 1e3), "unit": UNIT,
            "sample": f"{wl.B} candidates x {wl.K} iterations, score + gradient, checkpoint every "
                      f"{wl.extra['ckpt_every']}"}


def plain_timing(g, boac, mu, S_d, dev, stream, K):
    """The launch-per-step path (one candidate at a time), on 4 candidates."""
    import torch
    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    nplain = 4
    Fp = torch.ones(nplain, WL.n, WL.n, device=dev)
    wsp = boac.workspace(g, nplain, boac._lib.OP_MLEM_PLAIN, dev)
    mup = mu[:nplain].contiguous()
    boac.boac_mlem(g, mup, S_d, Fp, 2, plain=True, ws=wsp)
    torch.cuda.synchronize(dev)
    a, b = E(), E()
    Fp.fill_(1.0)
    a.record(stream)
    boac.boac_mlem(g, mup, S_d, Fp, K, plain=True, ws=wsp)
    b.record(stream)
    b.synchronize()
    return {"value": nplain * K / (a.elapsed_time(b) / 1e3), "unit": UNIT,
            "sample": f"{nplain} candidates x {K} iterations, 4 launches per iteration"}


# ----------------------------------------------------------------- other workloads
def _timed(fn, dev, reps=2, warm=True):
    """Best of `reps` CUDA-event timings of fn() after one warm-up call (ms)."""
    import torch
    if warm:
        fn()
    torch.cuda.synchronize(dev)
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(torch.cuda.current_stream(dev))
        fn()
        b.record(torch.cuda.current_stream(dev))
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def _phantom_sinograms(boac, Geom, Tissue, dev, n, dx, V, counts, seeds, c_true=None):
    """Seeded phantoms and Poisson sinograms built on the device, one per seed."""
    import torch
    g = Geom.make(n, dx, V)
    t = Tissue(*synth.TISSUE)
    out = []
    for s in seeds:
        ph, noise, _ = synth.streams(int(s))
        ct = synth.C_TRUE if c_true is None else c_true[int(s) % len(c_true)]
        mu_t = boac.boac_rasterize_mu(g, t, torch.tensor([ct], dtype=torch.float32, device=dev))
        brain = (mu_t[0] == np.float32(synth.TISSUE[0])).cpu().numpy()
        Ft = synth.paint_activity(n, float(np.float32(dx)), brain, synth.ellipses(ph, ct[0]))
        q = boac.boac_project(g, mu_t, torch.tensor(Ft[None], dtype=torch.float32, device=dev))
        out.append(torch.tensor(synth.poisson_sinogram(noise, q[0].double().cpu().numpy(), counts),
                                dtype=torch.float32, device=dev))
    return g, t, out


def workload_line(name, args, dev, tune=None):
    """Throughput of one of the other workloads of the hot path on one GPU:
    the single-candidate case, the ragged batch, the large slices, the
    differentiable score, the explicit system matrix.  Returns its JSON line
    (None for the quality study, which prints its own)."""
    import torch
    from paper_2109_11920_gb300 import Geom, Tissue
    from paper_2109_11920_gb300 import api as boac
    from paper_2109_11920_gb300 import autotune
    peak, peak_kind = fp32_peak(dev)
    if name == "small":
        wl = synth.SMALL
        g, t, (S,) = _phantom_sinograms(boac, Geom, Tissue, dev, wl.n, wl.dx, wl.V, wl.counts, [wl.seed])
        c = torch.tensor(synth.candidates(synth.streams(wl.seed)[2], 1).astype(np.float32), device=dev)
        mu = boac.boac_rasterize_mu(g, t, c)
        F = torch.ones(1, wl.n, wl.n, device=dev)
        ms = _timed(lambda: boac.boac_mlem(g, mu, S, F.fill_(1.0), wl.K), dev)
        msp = _timed(lambda: boac.boac_mlem(g, mu, S, F.fill_(1.0), wl.K, plain=True), dev)
        work = [(wl.V, wl.n, wl.K)]
        extra = {"plain_path_ms": msp}
        desc = f"{wl.name}: 1 candidate x {wl.K} iterations, {wl.n}x{wl.n}, {wl.V} views"
    elif name in ("ragged", "large"):
        if name == "ragged":
            wl = synth.RAGGED
            _, _, rng = synth.streams(wl.seed)
            cls, K = synth.ragged_schedule(rng, wl.B, wl.extra["mix"], wl.extra["k_range"])
            classes = wl.extra["classes"]
            mus, Ss, geoms = [], [], []
            for ci, (n, dx, V) in enumerate(classes):
                members = [b for b in range(wl.B) if cls[b] == ci]
                g, t, S_list = _phantom_sinograms(boac, Geom, Tissue, dev, n, dx, V, 2e5, [1000 + b for b in members])
                geoms.append(g)
                cc = torch.tensor(np.stack([synth.candidates(synth.streams(1000 + b)[2], 1)[0]
                                            for b in members]).astype(np.float32), device=dev)
                mu_c = boac.boac_rasterize_mu(g, t, cc)
                for i, b in enumerate(members):
                    mus.append((b, mu_c[i]))
                    Ss.append((b, S_list[i]))
            mus = [m for _, m in sorted(mus, key=lambda x: x[0])]
            Ss = [x for _, x in sorted(Ss, key=lambda x: x[0])]
            batch = boac.RaggedBatch(geoms, [int(x) for x in cls], [int(k) for k in K], mus, Ss, device=dev)
            work = [(classes[int(cls[b])][2], classes[int(cls[b])][0], int(K[b])) for b in range(wl.B)]
            desc = (f"{wl.name}: {wl.B} candidates, 64^2/60v : 96^2/90v : 128^2/120v = 1:1:2, "
                    f"K ~ U{{20..80}}, own phantom per candidate")
        else:
            wl = synth.LARGE
            n_sl, per = args.slices or wl.extra["slices"], wl.B
            K_l = args.wl_iters or wl.K
            c_sl = synth.slice_coefficients(np.random.default_rng(wl.seed), n_sl)
            g, t, S_list = _phantom_sinograms(boac, Geom, Tissue, dev, wl.n, wl.dx, wl.V, wl.counts,
                                              list(range(n_sl)), c_true=c_sl)
            mus, Ss = [], []
            for s in range(n_sl):
                cc = torch.tensor(synth.candidates(synth.streams(s)[2], per, c_sl[s]).astype(np.float32), device=dev)
                mu_c = boac.boac_rasterize_mu(g, t, cc)
                mus += list(mu_c)
                Ss += [S_list[s]] * per
            batch = boac.RaggedBatch([g], [0] * (n_sl * per), [K_l] * (n_sl * per), mus, Ss, device=dev)
            work = [(wl.V, wl.n, K_l)] * (n_sl * per)
            desc = f"{wl.name}: {n_sl} slices x {per} candidates, 256x256, 180 views, K={K_l}"
        tune = (not args.no_tune) if tune is None else tune
        config = autotune.tune_ragged(batch, probe_iters=2, repeats=1) if tune else None
        batch.prepare(config)
        if name == "large":
            # warm-up on the first slice's candidates only (module load, kernel
            # attributes), then one timed run of the whole batch (about 7 s)
            warm = boac.RaggedBatch([g], [0] * per, [2] * per, mus[:per], Ss[:per], device=dev)
            warm.prepare(config)
            warm.run()
            ms = _timed(lambda: (batch.F_pool.fill_(1.0), batch.run()), dev, reps=1, warm=False)
        else:
            ms = _timed(lambda: (batch.F_pool.fill_(1.0), batch.run()), dev, reps=2)
        if batch.status() != boac._lib.BOAC_OK:
            raise RuntimeError(f"{name}: device status {batch.status()}")
        extra = {"launch_config": config}
    elif name == "quality":
        from paper_2109_11920_gb300 import quality
        wl = quality.QUALITY
        rows, t0 = [], time.perf_counter()
        for case in range(wl.extra["cases"]):
            r = quality.run_case(case, dev)
            rows.append({"case": case, "c_true": [round(float(x), 4) for x in r["c_true"]],
                         "c_bo": [round(float(x), 4) for x in r["c_bo"]],
                         "scores": {k: {m: round(v, 4) for m, v in sc.items()} for k, sc in r["scores"].items()}})
        wall = time.perf_counter() - t0
        print(json.dumps({"metric": "SSIM / CNR / PSNR of MLEM-BOAC vs MLEM-NAC (quality workload)",
                          "unit": "score", "n_gpus": 1, "wall_s": wall, "data": "synthetic",
                          "config": {"workload": f"{wl.name}: {wl.extra['cases']} seeded heads, {wl.n}x{wl.n}, "
                                                 f"{wl.V} views, {wl.counts:g} counts, K={wl.K}, BO {wl.extra['bo_init']} "
                                                 f"initial + {wl.extra['bo_cycles']} cycles x {wl.B} candidates"},
                          "cases": rows}), flush=True)
        return None
    elif name == "sysmat":
        # the batched workload through the explicit system matrix
        wl = synth.BATCHED
        Bs = args.candidates  # the batched workload's 256 unless given (smaller cases for profiling)
        g, t, (S,) = _phantom_sinograms(boac, Geom, Tissue, dev, wl.n, wl.dx, wl.V, wl.counts, [wl.seed])
        c = torch.tensor(synth.candidates(synth.streams(wl.seed)[2], Bs).astype(np.float32), device=dev)
        mu = boac.boac_rasterize_mu(g, t, c)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        m = boac.SysMat(g, dev)
        torch.cuda.synchronize(dev)
        build_ms = (time.perf_counter() - t0) * 1e3
        vals = torch.empty(boac.SysMat.vals_shape(Bs, m.nnz), dtype=torch.float32, device=dev)
        ws = m.workspace(Bs)
        F = torch.ones(Bs, wl.n, wl.n, device=dev)
        ms = _timed(lambda: (m.values(mu, out=vals), m.mlem(vals, S, F.fill_(1.0), wl.K, ws=ws)), dev)
        ms_vals = _timed(lambda: m.values(mu, out=vals), dev)
        ms_k0 = _timed(lambda: m.mlem(vals, S, F, 0, ws=ws), dev)  # sensitivity + score
        it_ms = (ms - ms_vals - ms_k0) / wl.K
        peak_gbs, peak_kind = measured_peak_gbs()
        # per iteration the two products stream both value copies of every
        # candidate once (the shared pattern is read once per group of 8)
        it_bytes = Bs * 2 * 4 * m.nnz
        work = [(wl.V, wl.n, wl.K)] * Bs
        extra = {"nnz": m.nnz, "pattern_build_ms": build_ms, "values_ms": ms_vals, "iteration_ms": it_ms,
                 "roofline_hbm": {"kernels": "forward_kernel + backward_update_kernel (one MLEM iteration)",
                                  "achieved": it_bytes / (it_ms / 1e3) / 1e9, "peak": peak_gbs, "unit": "GB/s",
                                  "frac": it_bytes / (it_ms / 1e3) / 1e9 / peak_gbs,
                                  "peak_kind": f"{peak_kind} hbm_gbs (copy)",
                                  "algorithmic_bytes_per_iteration": it_bytes}}
        desc = (f"{wl.name} through the explicit system matrix: {Bs} candidates x {wl.K} MLEM iterations, "
                f"{wl.n}x{wl.n}, {wl.V} views; value fill + MLEM + score per step")
        m.close()
    elif name in ("grad", "grad_params"):
        wl = synth.GRAD
        g, t, (S,) = _phantom_sinograms(boac, Geom, Tissue, dev, wl.n, wl.dx, wl.V, wl.counts, [wl.seed])
        c_np = synth.candidates(synth.streams(wl.seed)[2], wl.B)
        ck = wl.extra["ckpt_every"]
        if name == "grad":
            c = torch.tensor(c_np.astype(np.float32), device=dev)
            ms = _timed(lambda: boac.boac_score_grad(g, t, c, S, wl.K, ck), dev)
            what = "d lnP/dc"
        else:
            # per-candidate tissue values: the 9-parameter model
            tis = synth.tissue_candidates(np.random.default_rng(wl.seed), wl.B)
            prm = torch.tensor(np.concatenate([c_np, tis], 1).astype(np.float32), device=dev)
            ms = _timed(lambda: boac.boac_score_grad_params(g, prm, S, wl.K, ck), dev)
            what = "d lnP/d(c, mu_b, mu_c, dR), tissue values per candidate,"
        # forward MLEM, recomputation of each checkpoint segment, and the
        # adjoint iteration (two projections, two back-projections, the
        # attenuation adjoint): about 4 MLEM iterations of work per iteration
        work = [(wl.V, wl.n, 4 * wl.K)] * wl.B
        extra = {"work_model_note": "4 MLEM-iteration equivalents per differentiated iteration"}
        desc = f"{wl.name}: {wl.B} candidates, {what} through {wl.K} iterations, checkpoint every {ck}"
    else:
        raise SystemExit(f"unknown workload {name}")
    cand_its = sum(k for _, _, k in work) if not name.startswith("grad") else wl.B * wl.K
    flops = sum(FLOPS_PER_SAMPLE * V * n * n * k for V, n, k in work)
    line = {"metric": f"MLEM candidate-iterations/sec ({name} workload)", "value": cand_its / (ms / 1e3),
            "unit": UNIT, "n_gpus": 1, "ms": ms, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic", "config": {"workload": desc},
            "roofline": {"bound": "alu", "achieved": flops / (ms / 1e3) / 1e12, "peak": peak,
                         "unit": "TFLOP/s", "frac": flops / (ms / 1e3) / 1e12 / peak, "peak_kind": peak_kind,
                         "work_model": f"{FLOPS_PER_SAMPLE} FP32 ops per ray sample per view per iteration"}}
    line.update(extra)
    return line


def run_workload(args):
    """One JSON line for the workload named by --workload."""
    import torch
    from paper_2109_11920_gb300 import build as pkg_build
    pkg_build.build()
    dev = torch.device("cuda", 0)
    line = workload_line(args.workload, args, dev)
    if line is not None:
        print(json.dumps(line), flush=True)


def workload_summary(line):
    """The compact form of a workload line carried by the benchmark line."""
    out = {"value": line["value"], "unit": line["unit"], "ms": line["ms"],
           "fp32_model_frac": line["roofline"]["frac"], "workload": line["config"]["workload"]}
    for k in ("launch_config", "work_model_note"):
        if k in line:
            out[k] = line[k]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    # smaller cases for profiling (the default is the full workload)
    ap.add_argument("--candidates", type=int, default=WL.B, help="candidates per GPU")
    ap.add_argument("--iters", type=int, default=WL.K, help="MLEM iterations")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-path comparison")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffer) timing")
    ap.add_argument("--slices", type=int, default=0, help="large workload: slices (default 64)")
    ap.add_argument("--wl-iters", type=int, default=0, help="large workload: MLEM iterations (default 100)")
    ap.add_argument("--workload", default="batched", choices=["batched", "small", "ragged", "large", "grad", "grad_params", "quality", "sysmat"],
                    help="batched: the benchmark; the others print their own throughput line")
    ap.add_argument("--no-tune", action="store_true", help="ragged/large: default launch shapes")
    ap.add_argument("--no-workloads", action="store_true",
                    help="batched: skip the gradient, ragged and large-slice lines")
    args = ap.parse_args()
    if args.workload != "batched":
        run_workload(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
