#!/usr/bin/env python3
"""Benchmark of the discrete DMK evaluation pass (3D Laplace) on GB300.

One step = one full evaluation pass (unit-box map, tree build, upward pass,
plane-wave downward pass, leaf evaluation, residual near field, unpermute) of
a synthetic point cloud already resident in HBM.  Default workload: N = 1e7
points, 50 Gaussian clusters plus 10% uniform background, net-zero normal
charges, eps = 1e-6, leaf capacity 200, mixed precision.  The FP64 path is
timed on the same input for the mixed-vs-FP64 comparison.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank evaluates its own independent cloud (different
seed): the method has no exchange step on one node, so scaling is weak and
there is no collective on the data path (only a barrier and a max-reduction
of the timings).  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "3D Laplace DMK points/s at rel-L2 1e-6, mixed-prec vs FP64 path, 1 GB300"
UNIT = "points/s"
FP32_LANES_PER_SM = 128
# threads of the anterpolation CTA: one (a, b pair) register tile each
ANTERP_FFMA_THREADS = 256
# nominal dense tensor rates of the part (TF32 / BF16), used only as a ratio to
# carry the measured BF16 rate over to TF32
TF32_PER_BF16 = 1.1 / 2.25
# FP32 FMA throughput measured on this machine's GB300 by a one-kernel probe
# (independent FMA chains, CUDA events, 152 SMs x 8 blocks x 256 threads) at
# the SM clock it ran at; scaled to the clock sampled during a run
FFMA_MEASURED_TFLOPS = 78.52
FFMA_MEASURED_MHZ = 2070.0
# FP64 FMA throughput from the same probe with double chains
DFMA_MEASURED_TFLOPS = 1.26


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="laplace3d_clustered_n1e7")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true", help="omit the host-buffer measurement (profiling runs)")
    ap.add_argument("--cpu-sample", type=int, default=100_000)
    ap.add_argument("--grad", action="store_true",
                    help="time the differentiable potential (forward with gradients, backward) instead")
    ap.add_argument("--batch", action="store_true",
                    help="time the batched workload (4096 independent systems, leaf capacity autotuned) instead")
    ap.add_argument("--yukawa", action="store_true",
                    help="time the Yukawa kernel exp(-10 r)/r on 4e6 uniform points instead")
    ap.add_argument("--log2d", action="store_true",
                    help="time the 2D kernel log r on 8e6 points (circle and disk) at eps 1e-8 instead")
    ap.add_argument("--leaf-cap", type=int, default=0,
                    help="--log2d: this leaf capacity instead of the autotuner's (profiling runs)")
    ap.add_argument("--log2d-mixed", action="store_true",
                    help="--log2d: the mixed path (FP32 residual pairs, FP64 far field) at eps 1e-6")
    ap.add_argument("--log2d-points", type=int, default=0,
                    help="--log2d: this many points of the same recipe instead of 8e6 (profiling runs)")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


NEAR_SCREEN_FLOPS = 8  # distance of a candidate pair: 3 differences, 3 squares, 2 adds


# DRAM bytes per unit of work, from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum) of every kernel launch of an evaluation of the
# 2e6-point clustered workload (profiles/dram_traffic_laplace3d_clustered_n2e6.md),
# each valid only for the kernel source it was taken on:
# kernel -> (source file, its sha256, bytes per unit, the unit)
TRAFFIC = {
    "k_near": ("paper_2308_00292_gb300/csrc/near.cu",
               "112cd3947ab28d2b05e8f021493f6e6ff7889daaac1e6856d8eecea9b7998034",
               (74050560 + 9337344) / 2296972300, "near_pairs_screened"),
    "k_local": ("paper_2308_00292_gb300/csrc/passes.cu",
                "0f4bf4204d6232a6b711d373f96deb4ffb1f235a578e7f7b72006c9f56c630c3",
                (980.77e6 + 120.51e6) / 45739717602, "local_flops"),
    "k_upward": ("paper_2308_00292_gb300/csrc/passes.cu",
                 "0f4bf4204d6232a6b711d373f96deb4ffb1f235a578e7f7b72006c9f56c630c3",
                 (127476992 + 192137984) / 2000000, "n_points"),
    "k_incoming": ("paper_2308_00292_gb300/csrc/incoming.cu",
                   "0ffb113e5a55fd71b119a1b20be0f6c40b1aba711c9d70abdd70a81941f26762",
                   (747262208 + 652316928) / 1218832664, "hbm_bytes"),
}


def traffic_per_unit(kernel: str):
    """DRAM bytes per unit of work of a kernel, or None if its source changed since the capture."""
    import hashlib
    if kernel not in TRAFFIC:
        return None
    src, sha_want, per_unit, _ = TRAFFIC[kernel]
    try:
        with open(os.path.join(ROOT, src), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
    except OSError:
        return None
    return per_unit if sha == sha_want else None


def near_flops_per_pair(qdeg: int) -> int:
    # a pair inside the support: the distance (8), x = 2 r^2/R^2 - 1 (2),
    # Horner q(x) (2 per degree), rsqrt (1), 1/r - q/R (2), charge times value and sum (2)
    return NEAR_SCREEN_FLOPS + 2 + 2 * qdeg + 1 + 2 + 2


def measured_peaks() -> dict:
    """The measured peaks (HBM copy, cuBLAS BF16), else the fallback figures."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return {"hbm_gbs": float(m["hbm_gbs"]), "bf16_tflops": float(m["bf16_tflops"]),
                "bf16_tflops_sustained": float(m.get("bf16_tflops_sustained", m["bf16_tflops"])),
                "basis": "of measured (MEASURED_PEAKS.json)"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "basis": "of fallback"}


def fp32_peak(sm_count: int, sm_mhz: float):
    """FP32 FMA peak in TFLOP/s at the sampled clock, and how it was obtained."""
    if FFMA_MEASURED_TFLOPS:
        return (FFMA_MEASURED_TFLOPS * sm_mhz / FFMA_MEASURED_MHZ,
                "FFMA probe %.1f TFLOP/s at %.0f MHz, scaled to %.0f MHz" % (FFMA_MEASURED_TFLOPS,
                                                                              FFMA_MEASURED_MHZ, sm_mhz))
    return (sm_count * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12,
            "%d SMs x %d FP32 lanes x 2 flops x %.0f MHz" % (sm_count, FP32_LANES_PER_SM, sm_mhz))


def kernel_work(stats: dict, prm: dict, n_src: int, n_tgt: int) -> dict:
    """Algorithmic work of each kernel of one evaluation, split by the unit
    that executes it: (amount, unit kind) pairs, unit kind one of
    'tensor' (flops of the 3xTF32 contractions, counted once per product),
    'fp32' (FP32 flops on the CUDA cores) and 'hbm' (bytes)."""
    p, nf = prm["p"], prm["nf"]
    nh, n1 = nf + 1, 2 * nf + 1
    mxp = (n1 + 1) & ~1
    nfout, nfin = stats["n_fout"], stats["n_fin"]
    w = {}
    # upward: anterpolation onto the parent grid (2 p^3 per source), child-to-parent shifts;
    # the single-precision anterpolation is register-tiled FFMA while one CTA's threads
    # cover p x ceil(p/2) (a, b) pairs, else 3xTF32 on the tensor cores
    anterp_unit = "fp32" if p * ((p + 1) // 2) <= ANTERP_FFMA_THREADS else "tensor"
    w["k_upward"] = [("anterpolation", 2.0 * p ** 3 * n_src, anterp_unit),
                     ("c2p shifts", 3.0 * p ** 3 * (p + 1) * max(nfout - 1, 0), "fp32")]
    # outgoing plane waves, parity-split mode products z, y, x per F_out box
    w["k_prox2pw"] = [("proxy to plane waves", float(nfout) * (2 * p ** 3 * nh + 4 * p * p * nh * nh
                                                               + 4 * n1 * p * nh * nh), "fp32")]
    if stats.get("incoming_reads", 0) > 0:
        contr = float(nfin) * (8 * p * nh ** 3 + 4 * p * p * nh * nh + 2 * p ** 3 * nh)
        w["k_incoming"] = [("plane waves to Chebyshev", contr, "tensor"),
                           ("translation", 8.0 * n1 * n1 * nh * stats["incoming_reads"], "fp32"),
                           ("plane waves read once, coefficients written",
                            8.0 * nfout * nh * n1 * mxp + 4.0 * nfin * p ** 3, "hbm")]
    ev = 2.0 * p ** 3 * n_tgt
    w["k_local"] = [("leaf evaluation", ev, "tensor"),
                    ("p2c shifts and sums", max(float(stats["local_flops"]) - ev, 0.0), "fp32")]
    # the near field: the distance screen of every pair the kernel tests (the
    # sources left after culling against each target group's bounding box),
    # and the residual kernel of every pair inside R_L
    screened, inside = stats["near_pairs_screened"], stats["near_pairs_inside"]
    w["k_near"] = [("screened pairs and residual kernel", float(screened * NEAR_SCREEN_FLOPS + inside * (
        near_flops_per_pair(prm["q_degree"]) - NEAR_SCREEN_FLOPS)), "fp32")]
    return w


def rooflines(work: dict, times_ms: dict, peaks: dict) -> dict:
    """Per kernel: each work component's achieved rate and fraction of its peak;
    the kernel's bound is the component with the largest fraction."""
    out = {}
    for k, comps in work.items():
        t = times_ms.get(k)
        if not t or t <= 0:
            continue
        parts = []
        for name, amount, kind in comps:
            if amount <= 0:
                continue
            if kind == "hbm":
                a, pk, unit, bound = amount / (t / 1e3) / 1e9, peaks["hbm"], "GB/s", "hbm"
            elif kind == "tensor":
                a, pk, unit, bound = amount / (t / 1e3) / 1e12, peaks["tensor"], "TFLOP/s", "tensor"
            elif kind == "fp64":
                a, pk, unit, bound = amount / (t / 1e3) / 1e12, peaks["fp64"], "TFLOP/s", "alu"
            else:
                a, pk, unit, bound = amount / (t / 1e3) / 1e12, peaks["fp32"], "TFLOP/s", "alu"
            parts.append({"work": name, "amount": amount, "bound": bound, "achieved": a, "peak": pk, "unit": unit,
                          "frac": a / pk})
        if not parts:
            continue
        top = max(parts, key=lambda d: d["frac"])
        out[k] = {"bound": top["bound"], "achieved": top["achieved"], "peak": top["peak"], "unit": top["unit"],
                  "frac": top["frac"], "ms_per_eval": t, "components": parts}
    return out


def rank_seed(cfg: dict, rank: int) -> int:
    """Seed of the independent cloud a rank evaluates (replicas, weak scaling)."""
    return cfg["seed"] + 17 * rank


def max_over_ranks(v: float, dist=None, device="cpu") -> float:
    """The slowest rank's time: an all-reduce(MAX) of one number (no data-path collective)."""
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(n_per_rank: int, world: int, ms: float) -> float:
    """Whole-job points/s: the points of all ranks over the slowest rank's time."""
    return n_per_rank * world / (ms / 1e3)


def cpu_baseline(cfg: dict, n_sample: int, seed_offset: int = 1000):
    """The oracle's plain FP64 DMK on a bounded sample of the same workload."""
    import oracle
    from paper_2308_00292_gb300 import inputs
    oracle.build()
    x, q = inputs.make(cfg["gen"], n_sample, cfg["seed"] + seed_offset)
    t0 = time.perf_counter()
    oracle.dmk(x, q, eps=cfg["eps"], leaf_cap=cfg["leaf_cap"])
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": n_sample / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d points of the %s workload (seed %d), eps %g, leaf cap %d, plain FP64 C oracle DMK, %.1f s"
                      % (n_sample, cfg["gen"], cfg["seed"] + seed_offset, cfg["eps"], cfg["leaf_cap"], dt)}


def run_reference(args, rank, world):
    from paper_2308_00292_gb300 import inputs
    if rank != 0:
        return
    cfg = inputs.CONFIGS[args.config]
    n_sample = args.cpu_sample
    # untimed: builds the oracle and touches its code once (it keeps no state)
    base = cpu_baseline(cfg, min(n_sample, 20000))
    times = []
    for k in range(args.steps):
        b = cpu_baseline(cfg, n_sample, seed_offset=1000 + k)
        times.append(n_sample / b["value"])
    tot = sum(times)
    value = n_sample * args.steps / tot
    cb = dict(base)
    cb["value"] = value
    cb["sample"] = "%d points of the %s workload per step, plain FP64 C oracle DMK" % (n_sample, cfg["gen"])
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(args, cfg),
            "cpu_baseline": cb, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_precision(cfg: dict) -> str:
    """The path a workload runs on: single precision with FP64 accumulation
    wherever it can reach its eps (eps >= 1e-7), else FP64."""
    return cfg.get("precision", "mixed" if cfg["eps"] >= 1e-7 else "fp64")


def config_dict(args, cfg):
    return {"workload": args.config, "n_points": cfg["n"], "distribution": cfg["gen"], "eps": cfg["eps"],
            "leaf_cap": cfg["leaf_cap"], "precision": config_precision(cfg), "seed": cfg["seed"],
            "l2": "inputs larger than L2 (%.0f MB of points and charges per rank)" % (cfg["n"] * 32 / 1e6),
            "parallelism": "independent replica per GPU" if args.gpus > 1 else "single GPU"}


def run_grad(args):
    """Forward (potentials and gradients) plus backward (dL/drho, dL/dx) of the
    differentiable potential, L = sum_i w_i u_i, one GPU, mixed precision."""
    import numpy as np
    import torch
    from paper_2308_00292_gb300 import dmk, inputs
    cfg = inputs.CONFIGS[args.config]
    x, q = inputs.make(cfg["gen"], cfg["n"], cfg["seed"])
    n = x.shape[0]
    w = torch.from_numpy(np.random.default_rng(cfg["seed"] + 1).standard_normal(n)).cuda()
    plan = dmk.Plan(cfg["eps"], precision=dmk.DMK_MIXED, leaf_cap=cfg["leaf_cap"])
    xd = torch.from_numpy(x).cuda()
    qd = torch.from_numpy(q).cuda()

    def step():
        xt = xd.clone().requires_grad_(True)
        qt = qd.clone().requires_grad_(True)
        (w * dmk.potential(plan, xt, qt)).sum().backward()
        return xt.grad, qt.grad

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    plan.close()
    line = {"metric": "3D Laplace DMK potentials + gradients (autograd forward and backward) points/s, 1 GB300",
            "value": n / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64acc", "data": "synthetic", "config": config_dict(args, cfg),
            "evaluations_per_step": 2}
    print(json.dumps(line), flush=True)


def run_batch(args):
    """4096 independent systems of 500 .. 50 000 points in one dmk_eval_batch
    call, mixed precision, with the leaf capacity chosen by the autotuner."""
    import numpy as np
    import torch
    from paper_2308_00292_gb300 import dmk, inputs
    name = "laplace3d_batched_4096"
    cfg = inputs.CONFIGS[name]
    x, q, off = inputs.batch(cfg["nsys"], seed=cfg["seed"])
    n, nsys = x.shape[0], len(off) - 1
    xd, qd = torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    plan = dmk.Plan(cfg["eps"], precision=dmk.DMK_MIXED)
    t0 = time.perf_counter()
    best, tune_ms = plan.tune_leaf_cap_batch(xd, qd, off, reps=1)
    tune_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        plan.eval_batch(xd, qd, off, out=out)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    phase = {"t_tree_ms": 0.0, "t_upward_ms": 0.0, "t_downward_ms": 0.0, "t_near_ms": 0.0, "t_local_ms": 0.0}
    launches = 0
    e0.record(stream)
    for _ in range(args.steps):
        plan.eval_batch(xd, qd, off, out=out)
        st = plan.stats()
        for k in phase:
            phase[k] += st[k]
        launches += st["n_launches"]
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    stats = plan.stats()
    u = out.cpu().numpy()
    # accuracy on 16 sampled systems: the oracle's compensated FP64 direct sum on
    # the host (up to 512 sampled targets per system, every point of the system
    # a source), outside the timed region
    import oracle
    oracle.build()
    rng = np.random.default_rng(cfg["seed"] + 7)
    num = den = 0.0
    for s in sorted(rng.choice(nsys, 16, replace=False)):
        a, b = int(off[s]), int(off[s + 1])
        tsel = np.sort(rng.choice(b - a, min(b - a, 512), replace=False))
        r = oracle.direct(x[a:b], q[a:b], x[a:b][tsel])
        num += float(np.sum((u[a:b][tsel] - r) ** 2))
        den += float(np.sum(r ** 2))
    # end to end through the public API: pinned host arrays copied in, potentials copied out
    e2e = None
    if not args.skip_e2e:
        xh, qh = torch.from_numpy(x).pin_memory(), torch.from_numpy(q).pin_memory()
        uh = torch.empty(n, dtype=torch.float64).pin_memory()
        xs, qs = torch.empty_like(xd), torch.empty_like(qd)
        torch.cuda.synchronize()
        ke = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        for _ in range(ke):
            xs.copy_(xh, non_blocking=True)
            qs.copy_(qh, non_blocking=True)
            plan.eval_batch(xs, qs, off, out=out)
            uh.copy_(out, non_blocking=True)
            torch.cuda.synchronize()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / ke
        e2e = {"value": n / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(x.nbytes + q.nbytes),
               "d2h_bytes_per_step": int(u.nbytes), "ms_per_step": e2e_ms}
    plan.close()
    fp64 = None
    if not args.skip_fp64:
        p64 = dmk.Plan(cfg["eps"], precision=dmk.DMK_FP64, leaf_cap=best)
        p64.eval_batch(xd, qd, off, out=out)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        p64.eval_batch(xd, qd, off, out=out)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1)
        fp64 = {"value": n / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64, "mixed_speedup": ms64 / ms}
        p64.close()
    per_step = {k: round(v / args.steps, 3) for k, v in phase.items()}
    line = {"metric": "3D Laplace DMK points/s over 4096 independent systems at 1e-6, mixed precision, 1 GB300",
            "value": n / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64acc", "data": "synthetic",
            "config": {"workload": name, "n_systems": nsys, "n_points": n, "distribution": cfg["gen"],
                       "eps": cfg["eps"], "leaf_cap": best, "precision": "mixed", "seed": cfg["seed"],
                       "l2": "inputs larger than L2 (%.0f MB of points and charges)" % (n * 32 / 1e6)},
            "autotune": {"leaf_cap": best, "ms_per_candidate": {str(k): round(v, 3) for k, v in tune_ms.items()},
                         "seconds": round(tune_s, 2)},
            "rel_l2_vs_oracle_direct_16_systems": (num / den) ** 0.5 if den > 0 else None,
            "e2e": e2e, "gpu_launches": launches, "clocks": clocks, "phases_ms": per_step, "fp64_path": fp64,
            "tree": {"levels": stats["n_levels"], "boxes": stats["n_boxes"], "leaves": stats["n_leaves"],
                     "near_pairs": stats["near_pairs"]}}
    print(json.dumps(line), flush=True)


def run_yukawa(args):
    """exp(-lambda r)/r, lambda = 10, 4e6 uniform points: the FP64 path at eps 1e-8
    (the accuracy the workload asks for, beyond single precision) and the mixed
    path at 1e-6, each with the leaf capacity chosen by the autotuner."""
    import numpy as np
    import torch
    import oracle
    from paper_2308_00292_gb300 import dmk, inputs
    name = "yukawa3d_uniform_n4e6"
    cfg = inputs.CONFIGS[name]
    x, q = inputs.make(cfg["gen"], cfg["n"], cfg["seed"])
    n, lam = x.shape[0], cfg["lam"]
    xd, qd = torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    # accuracy on 128 sampled targets against the oracle's direct Yukawa sum
    oracle.build()
    sample = np.sort(np.random.default_rng(cfg["seed"] + 11).choice(n, 128, replace=False))
    ref = oracle.direct(x, q, x[sample], lam=lam)
    stream = torch.cuda.current_stream()

    def measure(eps, precision, cands):
        plan = dmk.Plan(eps, precision=precision, kernel=dmk.DMK_YUKAWA, lam=lam)
        best, tune_ms = plan.tune_leaf_cap(xd, qd, candidates=cands, reps=1)
        for _ in range(args.warmup):
            plan.eval(xd, qd, out=out)
        torch.cuda.synchronize()
        sampler = ClockSampler(0)
        sampler.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        launches = 0
        e0.record(stream)
        for _ in range(args.steps):
            plan.eval(xd, qd, out=out)
            launches += plan.stats()["n_launches"]
        e1.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        ms = e0.elapsed_time(e1) / args.steps
        st = plan.stats()
        u = out.cpu().numpy()[sample]
        plan.close()
        return {"value": n / (ms / 1e3), "ms_per_step": ms, "eps": eps, "leaf_cap": best,
                "autotune_ms": {str(k): round(v, 3) for k, v in tune_ms.items()},
                "rel_l2_vs_direct_128_targets": float(np.linalg.norm(u - ref) / np.linalg.norm(ref)),
                "phases_ms": {k: round(st[k], 3) for k in ("t_tree_ms", "t_upward_ms", "t_downward_ms",
                                                            "t_near_ms", "t_local_ms")},
                "launches": launches, "clocks": clocks}

    f64 = measure(cfg["eps"], dmk.DMK_FP64, [200, 400, 800, 1200])
    mixed = None if args.skip_fp64 else measure(1e-6, dmk.DMK_MIXED, [100, 200, 280, 400])
    line = {"metric": "3D Yukawa exp(-10 r)/r DMK points/s at eps 1e-8 (FP64 path), 1 GB300",
            "value": f64["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": f64["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "n_points": n, "distribution": cfg["gen"], "eps": cfg["eps"],
                       "lambda": lam, "leaf_cap": f64["leaf_cap"], "precision": "fp64", "seed": cfg["seed"],
                       "l2": "inputs larger than L2 (%.0f MB of points and charges)" % (n * 32 / 1e6)},
            "gpu_launches": f64["launches"], "clocks": f64["clocks"], "fp64_eps1e-8": f64,
            "mixed_eps1e-6": mixed}
    print(json.dumps(line), flush=True)


def log2d_near_roofline(inside: int, prm: dict, near_ms: float, sm_mhz: float, mixed: bool) -> dict:
    """The 2D near field (k2_near) against its pipe's peak.  On the FP64 path
    it is bound by the FP64 pipe: per pair inside the support 24 flops
    (distance, log t by the table, the sums) and 2 per degree of the residual
    polynomial after the first (Horner, the form the plan takes at eps 1e-8).
    On the mixed path its pairs are FP32: 34 flops (distance from hi/lo
    offsets and r^2 9, t and 2x 3, Clenshaw's last step 4, logf counted as 8,
    the product 3, TwoSum 7) and 3 per degree of Clenshaw's recurrence, on the
    series cut for FP32 (q_degree_f32).  Peaks: the FFMA / DFMA probes scaled
    to the sampled SM clock."""
    if mixed:
        per_pair, unit = 34 + 3 * prm["q_degree_f32"], "fp32"
        peak = FFMA_MEASURED_TFLOPS * sm_mhz / FFMA_MEASURED_MHZ
        basis = "FFMA probe %.1f TFLOP/s at %.0f MHz, scaled to %.0f MHz" % (FFMA_MEASURED_TFLOPS,
                                                                             FFMA_MEASURED_MHZ, sm_mhz)
    else:
        per_pair, unit = 24 + 2 * (prm["q_degree"] - 1), "fp64"
        peak = DFMA_MEASURED_TFLOPS * sm_mhz / FFMA_MEASURED_MHZ
        basis = "DFMA probe %.2f TFLOP/s at %.0f MHz, scaled to %.0f MHz" % (DFMA_MEASURED_TFLOPS,
                                                                              FFMA_MEASURED_MHZ, sm_mhz)
    achieved = inside * per_pair / (near_ms * 1e-3) / 1e12
    return {"kernel": "k2_near", "bound": unit, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None, "ms_per_eval": near_ms, "peak_basis": basis,
            "work": "%d pairs inside the support x %d flops" % (inside, per_pair)}


def run_log2d(args):
    """log |x - y| in the plane, 8e6 points (half on the unit circle, half in the
    disk), eps 1e-8: the FP64 path (the 2D pass has no mixed path), leaf
    capacity chosen by the autotuner; e2e through dmk_eval_host from pinned
    host buffers."""
    import numpy as np
    import torch
    import oracle
    from paper_2308_00292_gb300 import dmk, inputs
    name = "log2d_circle_disk_n8e6"
    cfg = inputs.CONFIGS[name]
    x, q = inputs.make(cfg["gen"], args.log2d_points or cfg["n"], cfg["seed"])
    n = x.shape[0]
    if args.log2d_points:
        name += "_points%d" % n
    xd, qd = torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    oracle.build()
    sample = np.sort(np.random.default_rng(cfg["seed"] + 11).choice(n, 128, replace=False))
    ref = oracle.direct_log2d(x, q, x[sample])
    stream = torch.cuda.current_stream()
    eps = 1e-6 if args.log2d_mixed else cfg["eps"]
    prec = dmk.DMK_MIXED if args.log2d_mixed else dmk.DMK_FP64
    if args.log2d_mixed:
        name += "_mixed_eps1e-6"
    plan = dmk.Plan(eps, kernel=dmk.DMK_LOG2D, dim=2, leaf_cap=args.leaf_cap, precision=prec)
    if args.leaf_cap > 0:
        best, tune_ms = args.leaf_cap, {}
    else:
        best, tune_ms = plan.tune_leaf_cap(xd, qd, candidates=[80, 120, 160, 240, 320], reps=1)
    for _ in range(args.warmup):
        plan.eval(xd, qd, out=out)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    t_near = []
    e0.record(stream)
    for _ in range(args.steps):
        plan.eval(xd, qd, out=out)
        st = plan.stats()
        launches += st["n_launches"]
        t_near.append(st["t_near_ms"])
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    st = plan.stats()
    prm = plan.params()
    sm_mhz = clocks["sm_mhz"] if clocks and clocks.get("sm_mhz") else FFMA_MEASURED_MHZ
    near_ms = float(np.median(t_near))
    roofline = log2d_near_roofline(st["near_pairs_inside"], prm, near_ms, sm_mhz, args.log2d_mixed)
    roofline["timing"] = ("CUDA events the library records around the kernel on the evaluation's stream, "
                          "median over the timed steps")
    u = out.cpu().numpy()[sample]
    e2e = None
    if not args.skip_e2e:
        hx = torch.from_numpy(x).pin_memory().numpy()
        hq = torch.from_numpy(q).pin_memory().numpy()
        hu = torch.empty(n, dtype=torch.float64).pin_memory().numpy()
        plan.eval_host(hx, hq, out=hu)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            plan.eval_host(hx, hq, out=hu)
        e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
        e2e = {"value": n / (e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": n * 24, "d2h_bytes_per_step": n * 8,
               "ms_per_step": e_ms}
    plan.close()
    cpu = None
    if not args.skip_cpu_baseline:
        # the oracle's 2D pass on 50 000 points of the same recipe, the leaf
        # capacity the GPU used
        xs, qs = inputs.make(cfg["gen"], 50_000, cfg["seed"] + 1000)
        t0 = time.perf_counter()
        oracle.dmk_log2d(xs, qs, eps=eps, leaf_cap=best)
        dt = time.perf_counter() - t0
        cpu = {"value": 50_000 / dt, "unit": UNIT, "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
               "kind": "oracle",
               "sample": "50000 points of the %s workload (seed %d), eps %g, leaf cap %d, plain FP64 C oracle "
                         "2D DMK, %.1f s" % (cfg["gen"], cfg["seed"] + 1000, cfg["eps"], best, dt)}
    metric = ("2D log|x-y| DMK points/s at eps 1e-6 (mixed path), 1 GB300" if args.log2d_mixed
              else "2D log|x-y| DMK points/s at eps 1e-8 (FP64 path), 1 GB300")
    line = {"metric": metric,
            "value": n / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64acc" if args.log2d_mixed else "f64", "data": "synthetic",
            "config": {"workload": name, "n_points": n, "distribution": cfg["gen"], "eps": eps,
                       "leaf_cap": best, "precision": "mixed" if args.log2d_mixed else "fp64", "seed": cfg["seed"],
                       "l2": "inputs larger than L2 (%.0f MB of points and charges)" % (n * 24 / 1e6)},
            "autotune_ms": {str(k): round(v, 3) for k, v in tune_ms.items()},
            "rel_l2_vs_direct_128_targets": float(np.linalg.norm(u - ref) / np.linalg.norm(ref)),
            "tree": {"levels": st["n_levels"], "boxes": st["n_boxes"], "leaves": st["n_leaves"],
                     "near_pairs": st["near_pairs"], "near_pairs_inside": st["near_pairs_inside"]},
            "roofline": roofline,
            "e2e": e2e, "gpu_launches": launches, "clocks": clocks, "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2308_00292_gb300 import dmk, inputs

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    cfg = inputs.CONFIGS[args.config]
    x, q = inputs.make(cfg["gen"], cfg["n"], rank_seed(cfg, rank))
    n = x.shape[0]
    xd = torch.from_numpy(x).cuda()
    qd = torch.from_numpy(q).cuda()
    out = torch.empty(n, dtype=torch.float64, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    mixed = config_precision(cfg) == "mixed"
    prec = dmk.DMK_MIXED if mixed else dmk.DMK_FP64
    plan = dmk.Plan(cfg["eps"], precision=prec, leaf_cap=cfg["leaf_cap"])
    for _ in range(args.warmup):
        plan.eval(xd, qd, out=out)
    barrier()
    sampler = ClockSampler(local_rank) if rank == 0 else None
    if sampler:
        sampler.start()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    phase = {"t_tree_ms": 0.0, "t_upward_ms": 0.0, "t_downward_ms": 0.0, "t_near_ms": 0.0, "t_local_ms": 0.0}
    launches = 0
    e0.record(stream)
    for _ in range(args.steps):
        plan.eval(xd, qd, out=out)
        st = plan.stats()
        for k in phase:
            phase[k] += st[k]
        launches += st["n_launches"]
    e1.record(stream)
    barrier()
    clocks = sampler.stop() if sampler else None
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, "cuda")
    stats = plan.stats()
    prm = plan.params()
    value = job_throughput(n, world, ms)
    out_timed = out.cpu().numpy()

    # end to end through the host entry point: pinned inputs, H2D + eval + D2H per step
    e2e = None
    if not args.skip_e2e:
        xh = torch.from_numpy(x).pin_memory().numpy()
        qh = torch.from_numpy(q).pin_memory().numpy()
        uh = torch.empty(n, dtype=torch.float64).pin_memory().numpy()
        plan.eval_host(xh, qh, out=uh)
        barrier()
        ke = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        for _ in range(ke):
            plan.eval_host(xh, qh, out=uh)
        barrier()
        e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / ke, dist, "cuda")
        e2e = {"value": job_throughput(n, world, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": int(x.nbytes + q.nbytes),
               "d2h_bytes_per_step": int(uh.nbytes), "ms_per_step": e2e_ms}
    plan.close()

    # the FP64 path on the same input
    fp64 = None
    if not args.skip_fp64 and mixed:
        p64 = dmk.Plan(cfg["eps"], precision=dmk.DMK_FP64, leaf_cap=cfg["leaf_cap"])
        p64.eval(xd, qd, out=out)
        barrier()
        k64 = 2
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(k64):
            p64.eval(xd, qd, out=out)
        f1.record(stream)
        barrier()
        ms64 = max_over_ranks(f0.elapsed_time(f1) / k64, dist, "cuda")
        s64 = p64.stats()
        fp64 = {"value": job_throughput(n, world, ms64), "unit": UNIT, "ms_per_step": ms64, "steps": k64,
                "phases_ms": {k: round(s64[k], 3) for k in phase},
                "mixed_speedup": ms64 / ms}
        p64.close()

    # per-kernel times: the far-field kernels alone (near field skipped) and the
    # near field alone, outside the timed region, so that no kernel's time
    # includes another running beside it
    times = {}
    with dmk.Plan(cfg["eps"], precision=prec, leaf_cap=cfg["leaf_cap"], flags=dmk.FLAG_FAR_ONLY) as pf:
        acc = {"k_upward": [], "k_prox2pw": [], "k_incoming": [], "k_local": [], "tree": []}
        for r in range(4):
            pf.eval(xd, qd, out=out)
            sf = pf.stats()
            if r == 0:
                continue
            acc["k_upward"].append(sf["t_upward_ms"])
            acc["k_prox2pw"].append(sf["t_planewave_ms"])
            acc["k_incoming"].append(sf["t_incoming_ms"])
            acc["k_local"].append(sf["t_local_ms"])
            acc["tree"].append(sf["t_tree_ms"])
        times.update({k: statistics.median(v) for k, v in acc.items()})
    t_tree = times.pop("tree")
    if not mixed:
        # the FP64 path forms the incoming expansions inside the local pass
        times.pop("k_incoming", None)
    with dmk.Plan(cfg["eps"], precision=prec, leaf_cap=cfg["leaf_cap"], flags=dmk.FLAG_NEAR_ONLY) as pn:
        tn = []
        for r in range(4):
            pn.eval(xd, qd, out=out)
            if r:
                tn.append(pn.stats()["t_near_ms"])
        times["k_near"] = statistics.median(tn)
    barrier()
    if rank != 0:
        return
    # accuracy of the timed evaluation: the oracle's compensated FP64 direct sum
    # over all sources at 256 sampled targets, on the host
    import oracle
    oracle.build()
    u = out_timed
    sample = np.sort(np.random.default_rng(cfg["seed"] + 11).choice(n, 256, replace=False))
    ref = oracle.direct(x, q, x[sample])
    rel_l2 = float(np.linalg.norm(u[sample] - ref) / np.linalg.norm(ref))

    per_step = {k: v / args.steps for k, v in phase.items()}
    sm_mhz = clocks["sm_mhz"] if clocks and clocks.get("sm_mhz") else 1440.0
    props = torch.cuda.get_device_properties(local_rank)
    sm_count = props.multi_processor_count
    pk = measured_peaks()
    f32, f32_basis = fp32_peak(sm_count, sm_mhz)
    peaks = {"hbm": pk["hbm_gbs"], "fp32": f32,
             "tensor": pk["bf16_tflops_sustained"] * TF32_PER_BF16 / 3.0}
    peak_basis = {"hbm": "STREAM-style copy %s" % pk["basis"],
                  "fp32": f32_basis,
                  "tensor": "3xTF32 (three TF32 products per FP32 product): cuBLAS BF16 sustained %.1f TFLOP/s %s x "
                            "nominal TF32/BF16 ratio 1.1/2.25 / 3" % (pk["bf16_tflops_sustained"], pk["basis"])}
    work = kernel_work(stats, prm, n, n)
    if not mixed:
        # the FP64 path runs every contraction in double precision on the CUDA cores
        peaks["fp64"] = DFMA_MEASURED_TFLOPS * sm_mhz / FFMA_MEASURED_MHZ
        peak_basis["fp64"] = "DFMA probe %.2f TFLOP/s at %.0f MHz, scaled to %.0f MHz" % (
            DFMA_MEASURED_TFLOPS, FFMA_MEASURED_MHZ, sm_mhz)
        work = {k: [(nm, a, "hbm" if kd == "hbm" else "fp64") for nm, a, kd in v] for k, v in work.items()}
    kernels = rooflines(work, times, peaks)
    # the traffic captured by ncu for the kernel whose source it was taken on,
    # scaled by the kernel's units of work in this evaluation
    units = {"near_pairs_screened": stats["near_pairs_screened"], "local_flops": stats["local_flops"],
             "n_points": n, "hbm_bytes": sum(a for nm, a, kd in work.get("k_incoming", []) if kd == "hbm")}
    for k in TRAFFIC:
        if k in kernels and mixed:  # the captures are of the single-precision kernels
            tpu = traffic_per_unit(k)
            kernels[k]["traffic"] = tpu * units[TRAFFIC[k][3]] if tpu is not None else None
    dom = max(kernels, key=lambda k: kernels[k]["ms_per_eval"])
    roofline = {"kernel": dom, "bound": kernels[dom]["bound"], "achieved": kernels[dom]["achieved"],
                "peak": kernels[dom]["peak"], "unit": kernels[dom]["unit"], "frac": kernels[dom]["frac"],
                "traffic": kernels[dom].get("traffic"), "ms_per_eval": kernels[dom]["ms_per_eval"],
                "peak_basis": peak_basis[kernels[dom]["bound"] if kernels[dom]["bound"] != "alu"
                                         else ("fp32" if mixed else "fp64")],
                "timing": "CUDA events the library records on each kernel's stream, the kernel alone "
                          "(far-field or near-field-only evaluations, median of 3)"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64acc" if mixed else "f64", "data": "synthetic",
            "config": config_dict(args, cfg), "rel_l2": rel_l2,
            # the phases of the paper's timing breakdown (Table 2): tree, plane-wave
            # (Fourier) work, residual near field (direct), each kernel alone
            "paper_phases_ms": {"t_tree": t_tree,
                                "t_fourier": times.get("k_prox2pw", 0.0) + times.get("k_incoming", 0.0),
                                "t_direct": times.get("k_near", 0.0),
                                "t_other_far": times.get("k_upward", 0.0) + times.get("k_local", 0.0)},
            "rel_l2_basis": "256 sampled targets against the oracle's compensated FP64 direct sum over all sources",
            "e2e": e2e, "gpu_launches": launches,
            "roofline": roofline, "kernels": kernels, "peaks": peaks, "peak_basis": peak_basis,
            "sm_count": sm_count, "clocks": clocks,
            "phases_ms": {k: round(v, 3) for k, v in per_step.items()},
            "fp64_path": fp64,
            "tree": {"levels": stats["n_levels"], "boxes": stats["n_boxes"], "leaves": stats["n_leaves"],
                     "fout": stats["n_fout"], "fin": stats["n_fin"], "near_pairs": stats["near_pairs"],
                     "near_pairs_inside": stats["near_pairs_inside"],
                     "near_pairs_screened": stats["near_pairs_screened"], "incoming_reads": stats["incoming_reads"],
                     "balance_rounds": stats["balance_rounds"]}}
    if not args.skip_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg, args.cpu_sample)
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.grad:
        run_grad(args)
    elif args.batch:
        run_batch(args)
    elif args.yukawa:
        run_yukawa(args)
    elif args.log2d:
        run_log2d(args)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
