#!/usr/bin/env python3
"""Benchmark: even/odd CG solves/s to an FP64 true residual of 1e-10 (mixed precision vs
FP64) and the hopping kernel's bandwidth against the measured HBM roofline.

Headline workload (default): the 48^3 x 96 lattice, random SU(3) links exp(i eps H) with
eps = 0.6, kappa = 0.1615, mu = 0.0015 (mu~ = 2 kappa mu), Gaussian source -- the largest of
the single-GPU workloads.  One step = one complete solve of M x = b through the C ABI: packing,
source preparation, CG on Qhat+ Qhat- with the sloppy operator in FP16 storage with 8-real
links (the workload's named form) and FP32 arithmetic, reliable updates (FP32 recomputations
between FP64 ones),
reconstruction and the FP64 true-residual check.  The L2 cache is flushed (a 512 MB write)
before every step.  Beside the headline the line carries the same solve with 12-real links
(`link_form_12`, the faster form on GB300), the 16^3 x 32 throughput baseline
(FP64 and FP32 hopping kernels, FP64 CG), the 32^3 x 64 precision form, the batched workload
and the other solvers as extra objects.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun each rank solves its own system (a different
source) with no collective on the data path: weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Dslash GB/s & % HBM roofline; CG solves/sec to 1e-10 FP64 residual, mixed vs FP64"
HOP_FLOPS = 1320  # per output site per hopping application (8 hops x 168 flops - 24)
REF_TOTAL_SECONDS = 90.0  # host time of the reference arm's timed steps together
# Solver settings of the mixed solve per workload: sloppy storage:links, reliable-update delta and
# the arithmetic of the residual recomputations between FP64 ones.  FP16 storage keeps the
# iterated residual trustworthy over a factor ~0.3 only; FP32 storage over ~1e-5 on 16^3 x 32
# (88 iterations) and ~1e-3 on the longer solves.  48^3 x 96 is named with 8-real links; the
# 12-real form is measured beside it (LINK_FORM_12): both kernels are bound by the FP32 pipe and
# the 12-real one does fewer operations per site (no 8-real reconstruction), so its 64 more bytes
# a site cost nothing.
SOLVER_DEFAULTS = {"48^3x96": ("f16:8", 0.3, "f32"), "32^3x64": ("f32:12", 1e-3, "f64"),
                   "24^3x48": ("f32:12", 1e-3, "f64"), "16^3x32": ("f32:12", 1e-5, "f64")}
# Iterations of the FP64 CG to 1e-10 on each workload's first Gaussian source, measured on GB300
# by this library's FP64 CG (the same count the oracle's CG reaches up to rounding): the reference
# arm extrapolates its bounded sample to them where one complete oracle solve would take longer
# than the run may (48^3 x 96: about 50 minutes on 16 Grace cores).
LINK_FORM_12_DELTA = 0.2  # FP16/12 on 48^3 x 96: delta 0.2 0.719, 0.3 0.717, 0.5 0.702 solves/s
FP64_CG_ITERS = {"48^3x96": 522, "32^3x64": 437, "16^3x32": 88}
HOP_VARIANT = {1: "1 thread per site", 2: "2 threads per site", 4: "4 threads per site",
               3: "1 thread per site, pipelined loads"}


def hop_bytes_per_site(prec: int, nreal: int) -> int:
    """Algorithmic bytes per output site of one half-lattice hopping application: one input
    spinor, eight links (4 forward + 4 backward), one output spinor."""
    spinor = {0: 192, 1: 96, 2: 52, 3: 192}[prec]
    elem = {0: 8, 1: 4, 2: 2, 3: 8}[prec]
    return 2 * spinor + 8 * nreal * elem


def hop_naive_bytes_per_site(prec: int, nreal: int) -> int:
    """Bytes per output site without any neighbour reuse: eight neighbour spinors and eight links
    read, one spinor written (the naive count, printed beside the algorithmic one)."""
    spinor = {0: 192, 1: 96, 2: 52, 3: 192}[prec]
    elem = {0: 8, 1: 4, 2: 2, 3: 8}[prec]
    return 9 * spinor + 8 * nreal * elem


def parse_sloppy(s: str):
    p, l = s.split(":")
    return {"f32": 1, "f16": 2}[p], int(l)


def kernel_sources_hash(prec: int) -> str:
    """Digest of the sources of the one-flavour hopping kernel in storage precision `prec` (the
    kernel template, the shared device helpers and the precision's instantiation unit): an ncu
    traffic figure is reported only while the kernel it was taken of is unchanged."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_0905_3331_gb300", "csrc")
    unit = {0: "tm_dslash_f64.cu", 1: "tm_dslash_f32.cu", 2: "tm_dslash_f16.cu", 3: "tm_dslash_df64.cu"}[prec]
    pair_unit = {1: "tm_dslash_pair_f32.cu", 2: "tm_dslash_pair_f16.cu"}.get(prec, unit)
    h = hashlib.sha256()
    for f in ("tm_dslash.cuh", "tm_dslash_pair.cuh", "tm_internal.cuh", unit, pair_unit):
        path = os.path.join(csrc, f)
        if os.path.exists(path):
            with open(path, "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:12]


def ncu_traffic(form: str, lattice: str, variant: int, prec: int):
    """DRAM bytes (read + write) of one launch of the hopping kernel from a committed ncu summary:
    a line `bench-traffic: form=F lattice=L kernel=K sources=H bytes=N` in one of the files under
    profiles/, for this form, lattice, kernel choice and the current kernel sources.  Returns
    (bytes, file) or (None, None)."""
    import glob
    import re
    want = kernel_sources_hash(prec)
    pat = re.compile(r"bench-traffic: form=(\S+) lattice=(\S+) kernel=(\d+) sources=([0-9a-f]+) bytes=(\d+)")
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as fh:
            for line in fh:
                m = pat.search(line)
                if m and (m.group(1), m.group(2), int(m.group(3)), m.group(4)) == (form, lattice, variant, want):
                    return float(m.group(5)), os.path.relpath(path, ROOT)
    return None, None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.file, stderr=subprocess.DEVNULL)
            # nvidia-smi takes a moment to start: begin the timed region once it samples
            t0 = time.time()
            while time.time() - t0 < 3.0 and os.path.getsize(self.file.name) == 0:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.file is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.file.flush()
        rows = []
        with open(self.file.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[4 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# -------------------------------------------------------- multi-rank logic ---
def trimmed_mean(ts, frac: float = 0.1) -> float:
    """Mean of the launch times without the lowest and highest `frac` (a stray launch that the
    host or another process delays by 50-150 us would otherwise dominate a ~14 us average)."""
    ts = sorted(ts)
    k = int(len(ts) * frac)
    core = ts[k:len(ts) - k] if len(ts) > 2 * k else ts
    return statistics.mean(core)


def reduce_max(v: float, world: int, device) -> float:
    """Max of a per-rank value over all ranks (the slowest rank's time)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, t_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / t_max


# ------------------------------------------------------------------ GPU arm ---
def hop_launch_time(lat, dev, prec, nreal, half, n, flush, clean, cold=True):
    """Mean time of one tm_apply_hopping_eo launch on `lat` in (prec, nreal) storage, from per-launch
    CUDA events on the launching stream.  Cold: before each launch L2 is flushed (512 MB write) and
    cleaned (a read pass over another buffer twice the size of L2, so that the flush's dirty lines
    are written back first: the cold state ncu measures in); mean of the middle 80% of launches.
    Warm: n launches back to back."""
    import torch
    stream = torch.cuda.current_stream()
    nb = lat.half_field_bytes(prec)
    din = torch.empty(nb, dtype=torch.uint8, device=dev)
    dout = torch.empty(nb, dtype=torch.uint8, device=dev)
    lat.pack_half(prec, din, half)
    lat.apply_hopping_eo(1, dout, din, prec, nreal)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if cold:
        ts = []
        for k in range(n):
            flush.zero_()
            clean.sum()
            e0.record(stream)
            lat.apply_hopping_eo(k & 1, dout, din, prec, nreal)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        return trimmed_mean(ts)
    e0.record(stream)
    for k in range(n):
        lat.apply_hopping_eo(k & 1, dout, din, prec, nreal)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / n


def hop_entry(prec, nreal, h, t_cold, t_warm, peak):
    by = hop_bytes_per_site(prec, nreal) * h
    e = {"bytes_per_site": hop_bytes_per_site(prec, nreal), "us_cold": t_cold * 1e6,
         "gbs_cold": by / t_cold / 1e9,
         "gbs_naive_count_cold": hop_naive_bytes_per_site(prec, nreal) * h / t_cold / 1e9,
         "frac_hbm_cold": by / t_cold / 1e9 / peak, "gflops_cold": HOP_FLOPS * h / t_cold / 1e9}
    if t_warm is not None:
        e.update({"us_l2_resident": t_warm * 1e6, "gbs_l2_resident": by / t_warm / 1e9,
                  "gflops_l2_resident": HOP_FLOPS * h / t_warm / 1e9})
    return {k: (round(v, 4) if isinstance(v, float) else v) for k, v in e.items()}


def run_gpu(args):
    import numpy as np
    import torch

    from paper_0905_3331_gb300 import CG_FP64, CG_RELIABLE, F32, F64, Lattice, inputs, launch_count
    from paper_0905_3331_gb300 import build as libbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    libbuild.build()

    w = inputs.WORKLOADS[args.workload]
    d_sloppy, d_delta, d_upd = SOLVER_DEFAULTS.get(w.name, ("f32:12", 1e-3, "f64"))
    args.sloppy = args.sloppy or d_sloppy
    args.delta = args.delta if args.delta is not None else d_delta
    args.update_prec = args.update_prec or d_upd
    sp, sl = parse_sloppy(args.sloppy)
    upd = {"f64": F64, "f32": F32}[args.update_prec]
    U = w.gauge()
    phi = w.source(rank)
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    lat.set_gauge(torch.from_numpy(U).to(dev))
    b = torch.from_numpy(phi).to(dev)
    x = torch.zeros_like(b)
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    mixed_kw = dict(mode=CG_RELIABLE, sloppy_prec=sp, sloppy_link=sl, delta=args.delta, update_prec=upd)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(v: float) -> float:
        return reduce_max(v, world, dev)

    def timed_solves(n, kw, host=False):
        """n solves, each after an L2 flush, timed with CUDA events (device side)."""
        infos = []
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * n)]
        if host:
            bh = torch.from_numpy(phi).pin_memory()
            xh = torch.zeros_like(bh).pin_memory()
        total = 0.0
        for k in range(n):
            flush.zero_()
            barrier()
            torch.cuda.synchronize()
            ev[2 * k].record(stream)
            if host:
                infos.append(lat.solve_cg(xh, bh, tol=1e-10, **kw))
            else:
                infos.append(lat.solve_cg(x, b, tol=1e-10, **kw))
            ev[2 * k + 1].record(stream)
            torch.cuda.synchronize()
            total += ev[2 * k].elapsed_time(ev[2 * k + 1]) / 1e3
        return total, infos

    # warm-up (allocations, gauge copies of every form used, tuning, stage graphs)
    for _ in range(args.warmup):
        timed_solves(1, mixed_kw)

    # ---- timed region: K mixed-precision solves
    launches0 = launch_count()
    torch.cuda.nvtx.range_push("timed_region")  # ncu --nvtx --nvtx-include "timed_region/"
    with ClockSampler(local) as clk:
        t_mixed, infos = timed_solves(args.steps, mixed_kw)
    torch.cuda.nvtx.range_pop()
    launches = launch_count() - launches0
    clocks = clk.summary()
    t_mixed = max_over_ranks(t_mixed)
    worst_res = max(i.true_rel_residual for i in infos)

    # ---- FP64 CG on the same system (the comparison the metric asks for); its stage graphs are
    # captured in the first solve, a few ms against seconds per solve at this size
    n64 = max(1, min(args.steps, args.fp64_steps))
    t64, infos64 = timed_solves(n64, dict(mode=CG_FP64))
    t64 = max_over_ranks(t64)

    # ---- end to end: same solve through the C ABI with pinned HOST buffers
    n_e2e = max(1, min(args.steps, args.e2e_steps))
    timed_solves(1, mixed_kw, host=True)
    t_e2e, _ = timed_solves(n_e2e, mixed_kw, host=True)
    t_e2e = max_over_ranks(t_e2e)

    # ---- the sloppy hopping kernel of the headline solve: launches back to back as in the solve
    # (one launch reads more than the 129 MB L2 on this lattice, so each starts without reuse), and
    # per launch after an L2 flush and clean
    h = w.V // 2
    peak, peak_kind = peaks()
    clean = torch.ones(256 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    half = torch.from_numpy(np.ascontiguousarray(phi.reshape(-1, 4, 3)[:h])).to(dev)
    t_cold = hop_launch_time(lat, dev, sp, sl, half, args.hop_iters, flush, clean)
    bytes_per_launch = hop_bytes_per_site(sp, sl) * h
    back_to_back = bytes_per_launch > 2 * 129 * 2 ** 20
    t_hop = hop_launch_time(lat, dev, sp, sl, half, args.hop_iters, flush, clean, cold=False) if back_to_back else t_cold
    variant_id = lat.hop_threads(sp, sl)
    top = hop_entry(sp, sl, h, t_hop, None, peak)
    traffic, traffic_file = ncu_traffic(args.sloppy, w.name, variant_id, sp)
    if args.traffic is not None:
        traffic, traffic_file = args.traffic, "--traffic"
    variant = HOP_VARIANT.get(variant_id, str(variant_id))
    roofline = {"bound": "hbm", "kernel": f"hop_kernel ({args.sloppy} sloppy form, {variant}) on {w.name}",
                "achieved": round(top["gbs_cold"], 1), "peak": peak, "unit": "GB/s",
                "frac": round(top["gbs_cold"] / peak, 4), "traffic": traffic,
                "traffic_source": traffic_file, "peak_kind": peak_kind,
                "bytes_per_launch": bytes_per_launch, "us_per_launch": round(t_hop * 1e6, 3),
                "us_per_launch_cold": round(t_cold * 1e6, 3),
                "frac_cold": round(bytes_per_launch / t_cold / 1e9 / peak, 4),
                "timing": (f"{args.hop_iters} launches back to back (alternating parity; one launch reads "
                           f"{bytes_per_launch / 1e6:.0f} MB, more than twice the L2), CUDA events around them; "
                           if back_to_back else "") +
                          f"cold: {args.hop_iters} launches, per-launch CUDA events, mean of the middle 80%, before "
                          "each launch L2 flushed (512 MB write) and cleaned (256 MB read)"}
    # ---- the same solve with 12-real links (where the headline form has 8), timed the same way
    link12 = None
    if sl == 8 and not args.no_link_form:
        kw12 = dict(mixed_kw, sloppy_link=12, delta=LINK_FORM_12_DELTA)
        timed_solves(1, kw12)
        n12 = max(1, min(args.steps, 3))
        t12, inf12 = timed_solves(n12, kw12)
        t12 = max_over_ranks(t12)
        t12_hop = hop_launch_time(lat, dev, sp, 12, half, args.hop_iters, flush, clean, cold=False)
        b12 = hop_bytes_per_site(sp, 12) * h
        tr12, tr12_file = ncu_traffic(f"f{16 if sp == 2 else 32}:12", w.name, lat.hop_threads(sp, 12), sp)
        link12 = {"sloppy": f"{'f16' if sp == 2 else 'f32'}:12", "delta": LINK_FORM_12_DELTA,
                  "solves_per_s": round(n12 * world / t12, 5), "s_per_solve": round(t12 / n12, 4),
                  "iters": inf12[-1].iters, "reliable_updates": inf12[-1].reliable_updates,
                  "true_rel_residual": max(i.true_rel_residual for i in inf12),
                  "speedup_vs_fp64": round((n12 * world / t12) / (n64 * world / t64), 3),
                  "roofline": {"bound": "hbm", "kernel": f"hop_kernel ({'f16' if sp == 2 else 'f32'}:12, "
                               f"{HOP_VARIANT.get(lat.hop_threads(sp, 12), '?')}) on {w.name}",
                               "achieved": round(b12 / t12_hop / 1e9, 1), "peak": peak, "unit": "GB/s",
                               "frac": round(b12 / t12_hop / 1e9 / peak, 4), "traffic": tr12,
                               "traffic_source": tr12_file, "bytes_per_launch": b12,
                               "us_per_launch": round(t12_hop * 1e6, 3),
                               "timing": f"{args.hop_iters} launches back to back, CUDA events around them"},
                  "timing": f"{n12} solves after one warm-up, CUDA events, L2 flushed before each"}
    del half, clean

    n_units = args.steps * world
    value = whole_job_rate(args.steps, world, t_mixed)
    result = {
        "metric": METRIC, "value": round(value, 5), "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(t_mixed / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f16 storage, f32 arithmetic, f64 residuals" if sp == 2 else "f32+f64", "data": "synthetic",
        "config": {"workload": f"{w.name} lattice (V = {w.V}), random SU(3) links eps {w.eps}, kappa {w.kappa}, "
                               f"mu {w.mu}, Gaussian source; even/odd CG to FP64 true residual 1e-10",
                   "lattice": w.name, "solver": f"reliable-update CG, sloppy {args.sloppy} (FP32 arithmetic), "
                   f"delta {args.delta}, {args.update_prec.upper()} recomputations between FP64 ones",
                   "l2": "flushed (512 MB write) before every step; inputs also larger than L2",
                   "parallelism": f"replicas x{world} (independent systems)"},
        "mixed_cg": {"solves_per_s": round(value, 5), "s_per_solve": round(t_mixed / args.steps, 4),
                     "iters": infos[-1].iters, "reliable_updates": infos[-1].reliable_updates,
                     "true_rel_residual": worst_res},
        "fp64_cg": {"solves_per_s": round(n64 * world / t64, 5), "s_per_solve": round(t64 / n64, 4),
                    "iters": infos64[-1].iters, "true_rel_residual": infos64[-1].true_rel_residual},
        "speedup_mixed_vs_fp64": round((n_units / t_mixed) / (n64 * world / t64), 3),
        "roofline": roofline,
        "e2e": {"value": round(n_e2e * world / t_e2e, 5), "unit": "solves/s",
                "h2d_bytes_per_step": int(phi.nbytes), "d2h_bytes_per_step": int(phi.nbytes)},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if link12 is not None:
        result["link_form_12"] = link12
    lat.close()
    del b, x
    torch.cuda.empty_cache()
    if not args.no_extras:
        result["throughput_baseline"] = throughput_baseline(args, dev, flush)
    if not args.no_precision_form:
        result["precision_form"] = precision_form_measurement(args, dev)
    if not args.no_batched:
        result["batched"] = batched_measurement(args, dev)
    if not args.no_extras:
        result["solver_variants"] = extra_measurements(args, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(w, U, phi, infos64[-1].iters, args.cpu_seconds)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result))


# ----------------------------------------------------- 16^3 x 32 baseline ---
def throughput_baseline(args, dev, flush):
    """The 16^3 x 32 throughput baseline (eps 0.5, kappa 0.1632, mu 0.004): the hopping operator
    in FP64 and FP32 with 18-real links, 1000 applications back to back (L2-resident: the whole
    working set fits in the 129 MB L2) and per launch with L2 flushed and cleaned; FP64 CG to 1e-10
    on one Gaussian source; the mixed solve (FP32 storage, 12-real links, delta 1e-5); and the
    oracle's FP64 hopping on the host beside the FP64 kernel."""
    import numpy as np
    import torch

    from paper_0905_3331_gb300 import CG_FP64, CG_RELIABLE, F32, F64, Lattice, inputs
    w = inputs.WORKLOADS["16^3x32"]
    U, phi = w.gauge(), w.source()
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    lat.set_gauge(torch.from_numpy(U).to(dev))
    h = w.V // 2
    peak, _ = peaks()
    clean = torch.ones(256 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    half = torch.from_numpy(np.ascontiguousarray(phi.reshape(-1, 4, 3)[:h])).to(dev)
    dslash = {}
    for name, (prec, nreal) in {"f64_18": (F64, 18), "f32_18": (F32, 18), "f32_12": (F32, 12)}.items():
        tc = hop_launch_time(lat, dev, prec, nreal, half, 200, flush, clean)
        tw = hop_launch_time(lat, dev, prec, nreal, half, 1000, flush, clean, cold=False)
        dslash[name] = {**hop_entry(prec, nreal, h, tc, tw, peak), "threads_per_site": lat.hop_threads(prec, nreal)}
    b = torch.from_numpy(phi).to(dev)
    x = torch.zeros_like(b)
    out = {"workload": f"{w.name} lattice, eps {w.eps}, kappa {w.kappa}, mu {w.mu}, Gaussian source",
           "dslash": dslash,
           "dslash_timing": "cold: 200 launches, per-launch CUDA events, L2 flushed and cleaned before each, "
                            "mean of the middle 80%; l2_resident: 1000 launches back to back"}
    for name, kw, n in (("fp64_cg", dict(mode=CG_FP64), 3),
                        ("mixed_cg_f32_12", dict(mode=CG_RELIABLE, sloppy_prec=F32, sloppy_link=12, delta=1e-5), 20)):
        lat.solve_cg(x, b, tol=1e-10, **kw)  # warm-up (gauge copy, tuning, graphs)
        t, infos = _timed(lambda: lat.solve_cg(x, b, tol=1e-10, **kw), n, dev)
        out[name] = {"solves_per_s": round(n / t, 3), "iters": infos[-1].iters,
                     "reliable_updates": infos[-1].reliable_updates,
                     "true_rel_residual": infos[-1].true_rel_residual}
    out["speedup_mixed_vs_fp64"] = round(out["mixed_cg_f32_12"]["solves_per_s"] / out["fp64_cg"]["solves_per_s"], 3)
    lat.close()
    if not args.no_cpu_baseline:
        out["cpu_oracle_operator"] = cpu_oracle_operator(w, U, phi, dslash["f64_18"]["us_cold"])
    return out


# --------------------------------------------------------------- batched ---
def batched_measurement(args, dev):
    """The batched workload (12 spin-colour point sources on 24^3 x 48 plus 8^4, 12^3 x 24 and
    16^3 x 32 lattices with 4 Gaussian sources for each mu in {0.002, 0.005, 0.01}: 48 systems on
    4 gauge fields) in one batched solve, against the same systems solved one at a time; the 12
    point sources alone against one FP64 CG solve on their lattice; and the meson contraction of
    the 12 point-source solutions.  FP32 storage with 12-real links, delta --batched-delta (the
    24^3 x 48 systems run several hundred iterations, and the FP32 recursion drifts below delta ~
    1e-4 there).  CUDA events on the launching stream; L2 flushed before each timed call."""
    import torch

    from paper_0905_3331_gb300 import CG_FP64, CG_RELIABLE, F32, Lattice, inputs, solve_cg_batch
    defs = inputs.batched_workload()
    lats, systems = {}, []
    for d in defs:
        wl = d.workload
        if wl.name not in lats:
            lats[wl.name] = Lattice(wl.T, wl.L, wl.kappa, wl.mu)
            lats[wl.name].set_gauge(wl.gauge())
        b = torch.from_numpy(d.source()).to(dev)
        systems.append((lats[wl.name], d.mu, torch.zeros_like(b), b))
    kw = dict(sloppy_prec=F32, sloppy_link=12, delta=args.batched_delta)
    solve_cg_batch(systems, **kw)  # warm-up (gauge copies, allocations, tuning)
    t_batch, (infos,) = _timed(lambda: solve_cg_batch(systems, **kw), 1, dev)
    pts = systems[:12]
    solve_cg_batch(pts, **kw)
    t_pts, _ = _timed(lambda: solve_cg_batch(pts, **kw), 1, dev)
    big = defs[0].workload
    lat0, _, x0, b0 = pts[0]
    lat0.set_params(big.kappa, big.mu)
    x64 = torch.zeros_like(b0)
    t64, (i64,) = _timed(lambda: lat0.solve_cg(x64, b0, tol=1e-10, mode=CG_FP64), 1, dev)
    del x64
    point_sources = {"workload": f"12 point sources on {big.name}", "batched_s_per_solve": round(t_pts / 12, 4),
                     "fp64_s_per_solve": round(t64, 4), "fp64_iters": i64.iters,
                     "speedup_vs_fp64": round(t64 / (t_pts / 12), 2)}
    # meson contraction of the 12 point-source solutions (the correlators' building block)
    props = torch.stack([systems[k][2] for k in range(12)])
    Aout = torch.empty((big.T, 12, 12, 2), dtype=torch.float64, device=dev)
    lat0.meson_contract(props, Aout)
    t_con, _ = _timed(lambda: lat0.meson_contract(props, Aout), 5, dev)
    t_con /= 5
    con_bytes = props.numel() * props.element_size() + Aout.numel() * Aout.element_size()
    hbm, _ = peaks()
    # FP64 flops: 78 hermitian pairs x 12 components x 8 flop per site (conj(a) b accumulated)
    con_flops = 78 * 12 * 8 * big.T * big.L ** 3
    contraction = {"workload": f"12 point-source propagators on {big.name} ({con_bytes / 1e9:.2f} GB)",
                   "ms": round(t_con * 1e3, 4), "gbs": round(con_bytes / t_con / 1e9, 1),
                   "frac_hbm": round(con_bytes / t_con / 1e9 / hbm, 4),
                   "fp64_tflops": round(con_flops / t_con / 1e12, 4), "bytes": int(con_bytes),
                   "flops": int(con_flops), "bound": "fp64 alu (about 3.3 flop per byte)",
                   "timing": "mean of 5 calls, CUDA events, L2 flushed before each"}
    del props
    t_single, iters_single = 0.0, 0
    for lat_, mu, x, b in systems:
        lat_.set_params(lat_.kappa, mu)
        x.zero_()
        t, (info,) = _timed(lambda: lat_.solve_cg(x, b, mode=CG_RELIABLE, **kw), 1, dev)
        t_single += t
        iters_single += info.iters
    for lat_ in lats.values():
        lat_.close()
    n = len(systems)
    return {"workload": "12 point sources on 24^3x48 + {8^4, 12^3x24, 16^3x32} x 3 mu x 4 sources",
            "sloppy": "f32:12", "delta": args.batched_delta, "systems": n,
            "systems_per_s": round(n / t_batch, 3), "unbatched_systems_per_s": round(n / t_single, 3),
            "speedup": round(t_single / t_batch, 3),
            "max_true_rel_residual": max(i.true_rel_residual for i in infos),
            "iters_batched": sum(i.iters for i in infos), "iters_unbatched": iters_single,
            "timing": "CUDA events around one batched call / the sum of the single solves, L2 flushed before each",
            "point_sources": point_sources,
            "meson_contract": contraction}


# -------------------------------------------------- the precision-form size ---
def precision_form_measurement(args, dev):
    """The 32^3 x 64 workload (eps 0.6, kappa 0.1615, mu 0.003): per-launch roofline of the
    FP32 and FP16 hopping kernels with 12-real links (L2 flushed and cleaned before each launch)
    and reliable-update mixed solves with FP32 and FP16 storage against one FP64 CG solve, all
    to 1e-10."""
    import numpy as np
    import torch

    from paper_0905_3331_gb300 import CG_FP64, CG_RELIABLE, F16, F32, LINK12, Lattice, inputs
    w = inputs.WORKLOADS["32^3x64"]
    U, phi = w.gauge(), w.source()
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    lat.set_gauge(torch.from_numpy(U).to(dev))
    h = w.V // 2
    peak, _ = peaks()
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
    clean = torch.ones(256 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    half = torch.from_numpy(np.ascontiguousarray(phi.reshape(-1, 4, 3)[:h])).to(dev)
    out = {"workload": f"{w.name} lattice, eps {w.eps}, kappa {w.kappa}, mu {w.mu}"}
    for name, prec in (("f32_12", F32), ("f16_12", F16)):
        nb = lat.half_field_bytes(prec)
        din = torch.empty(nb, dtype=torch.uint8, device=dev)
        dout = torch.empty(nb, dtype=torch.uint8, device=dev)
        lat.pack_half(prec, din, half)
        lat.apply_hopping_eo(1, dout, din, prec, LINK12)
        ts = []
        for k in range(10):
            flush.zero_()
            clean.sum()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lat.apply_hopping_eo(k & 1, dout, din, prec, LINK12)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        t = trimmed_mean(ts)
        by = hop_bytes_per_site(prec, LINK12) * h
        out[name] = {"us": round(t * 1e6, 2), "gbs": round(by / t / 1e9, 1), "frac_hbm": round(by / t / 1e9 / peak, 4),
                     "bytes_per_site": hop_bytes_per_site(prec, LINK12)}
    b = torch.from_numpy(phi).to(dev)
    x = torch.zeros_like(b)
    # FP16 storage: delta 0.3 with FP32 recomputations between the FP64 ones (update_prec F32)
    for name, kw in (("mixed_f32_12", dict(mode=CG_RELIABLE, sloppy_prec=F32, sloppy_link=LINK12,
                                           delta=args.batched_delta)),
                     ("mixed_f16_12", dict(mode=CG_RELIABLE, sloppy_prec=F16, sloppy_link=LINK12,
                                           delta=0.3, update_prec=F32)),
                     ("fp64", dict(mode=CG_FP64))):
        if name != "fp64":
            lat.solve_cg(x, b, tol=1e-10, **kw)  # warm-up (sloppy gauge copy, tuning, graphs)
        t, infos = _timed(lambda: lat.solve_cg(x, b, tol=1e-10, **kw), 1, dev)
        out[name] = {"s_per_solve": round(t, 4), "iters": infos[-1].iters,
                     "reliable_updates": infos[-1].reliable_updates,
                     "true_rel_residual": infos[-1].true_rel_residual}
    out["speedup_mixed_vs_fp64"] = round(out["fp64"]["s_per_solve"] / out["mixed_f32_12"]["s_per_solve"], 2)
    out["speedup_mixed_f16_vs_fp64"] = round(out["fp64"]["s_per_solve"] / out["mixed_f16_12"]["s_per_solve"], 2)
    out["timing"] = ("hopping: 10 launches, CUDA events, mean of the middle 80%, L2 flushed and cleaned "
                     "before each; solves: CUDA events")
    lat.close()
    return out


# ------------------------------------------------------ the other solvers ---
def _timed(fn, n, dev):
    """n calls of fn, each after an L2 flush, CUDA events on the current stream; (seconds, infos)."""
    import torch
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    total, infos = 0.0, []
    for _ in range(n):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos.append(fn())
        e1.record(stream)
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1) / 1e3
    return total, infos


def extra_measurements(args, dev):
    """On the 16^3 x 32 workload's gauge field and source: BiCGstab and MR on Mhat against CG on
    the normal equations, the chronological guess along a sequence of slowly varying sources, and
    the non-degenerate doublet solve (FP32 sloppy storage with 12-real links, delta 1e-5)."""
    import numpy as np
    import torch

    from paper_0905_3331_gb300 import CG_FP64, CG_RELIABLE, F32, F64, Lattice, inputs
    w = inputs.WORKLOADS["16^3x32"]
    U, phi = w.gauge(), w.source()
    sp, sl, delta = F32, 12, 1e-5
    out = {}
    b = torch.from_numpy(phi).to(dev)
    x = torch.zeros_like(b)
    # ---- BiCGstab vs CG.  BiCGstab needs the spectrum of Mhat in Re > 0: kappa 0.13 on this
    # gauge field; at the workload's kappa it stagnates (shown with a bounded run).
    kb = 0.13
    lat = Lattice(w.T, w.L, kb, w.mu)
    lat.set_gauge(torch.from_numpy(U).to(dev))
    mixed = dict(mode=CG_RELIABLE, sloppy_prec=sp, sloppy_link=sl, delta=delta)
    rows = {}
    mixed_mr = dict(mode=CG_RELIABLE, sloppy_link=sl, delta=delta)
    for name, fn, kw in (("cg_fp64", lat.solve_cg, dict(mode=CG_FP64)),
                         ("bicgstab_fp64", lat.solve_bicgstab, dict(mode=CG_FP64)),
                         ("mr_fp64", lat.solve_mr, dict(mode=CG_FP64)),
                         ("cg_mixed", lat.solve_cg, mixed),
                         ("bicgstab_mixed", lat.solve_bicgstab, mixed),
                         ("mr_mixed", lat.solve_mr, mixed_mr)):
        fn(x, b, tol=1e-10, **kw)  # warm-up
        t, infos = _timed(lambda: fn(x, b, tol=1e-10, **kw), 3, dev)
        rows[name] = {"solves_per_s": round(3 / t, 3), "iters": infos[-1].iters,
                      "reliable_updates": infos[-1].reliable_updates,
                      "true_rel_residual": infos[-1].true_rel_residual}
    lat.set_params(w.kappa, w.mu)
    info = lat.solve_bicgstab(x, b, tol=1e-10, max_iter=500, check=False)
    rows["bicgstab_fp64_at_workload_kappa"] = {
        "kappa": w.kappa, "converged": info.status == 0, "iters": info.iters,
        "schur_rel_residual": info.schur_rel_residual}
    lat.close()
    out["bicgstab"] = {"workload": f"{w.name} gauge field and source at kappa {kb} "
                                   "(spectrum of Mhat in Re > 0), mu " + str(w.mu),
                       "sloppy": f"f32:{sl}, delta {delta}", **rows,
                       "timing": "3 solves each, CUDA events, L2 flushed before each"}
    # ---- chronological guess: 8 sources phi_k = phi + 0.02 k eta1 + 0.0005 k^2 eta2, normal
    # equations solved cold and from the guess of the last 4 solutions
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    lat.set_gauge(torch.from_numpy(U).to(dev))
    hb = lat.half_field_bytes(F64) // 8
    base, d1, d2 = (inputs.gaussian_spinor(w.T, w.L, s_) for s_ in (51, 52, 53))
    odd = ((np.indices((w.T, w.L, w.L, w.L)).sum(axis=0) & 1) == 1).reshape(-1)
    srcs = []
    for k in range(8):
        full = (base + 0.02 * k * d1 + 0.0005 * k * k * d2).reshape(-1, 4, 3)[odd]
        h = torch.from_numpy(np.ascontiguousarray(full).view(np.float64).reshape(-1)).to(dev)
        dsrc = torch.empty(hb, dtype=torch.float64, device=dev)
        lat.pack_half(F64, dsrc, h)
        srcs.append(dsrc)
    X = torch.zeros(hb, dtype=torch.float64, device=dev)
    lat.solve_normal(X, srcs[0], tol=1e-10)  # warm-up
    cold_iters = warm_iters = 0
    t_cold = t_warm = 0.0
    history = []
    for dsrc in srcs:
        X.zero_()
        t, (i,) = _timed(lambda: lat.solve_normal(X, dsrc, tol=1e-10), 1, dev)
        t_cold += t
        cold_iters += i.iters

        def warm():
            lat.chrono_guess(X, history[-4:], dsrc)
            return lat.solve_normal(X, dsrc, tol=1e-10, use_x0=True)
        t, (i,) = _timed(warm, 1, dev)
        t_warm += t
        warm_iters += i.iters
        history.append(X.clone())
    lat.close()
    # ---- non-degenerate doublet (eq. Dh): mubar 0.15, epsbar 0.19 on the same gauge field
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    lat.set_gauge(torch.from_numpy(U).to(dev))
    bd = torch.from_numpy(np.stack([phi, inputs.gaussian_spinor(w.T, w.L, 3)])).to(dev)
    xd = torch.zeros_like(bd)
    drows = {}
    for name, kw in (("fp64", dict(mode=CG_FP64)),
                     ("mixed", dict(mode=CG_RELIABLE, sloppy_link=sl, delta=delta))):
        lat.solve_doublet(xd, bd, 0.15, 0.19, tol=1e-10, **kw)  # warm-up
        t, infos = _timed(lambda: lat.solve_doublet(xd, bd, 0.15, 0.19, tol=1e-10, **kw), 3, dev)
        drows[name] = {"solves_per_s": round(3 / t, 3), "iters": infos[-1].iters,
                       "reliable_updates": infos[-1].reliable_updates,
                       "true_rel_residual": infos[-1].true_rel_residual}
    od = torch.empty_like(bd)
    lat.apply_Dh(od, bd, 0.15, 0.19)
    t, _ = _timed(lambda: lat.apply_Dh(od, bd, 0.15, 0.19), 5, dev)
    lat.close()
    out["doublet"] = {"workload": f"{w.name} gauge field, mubar 0.15, epsbar 0.19, kappa {w.kappa}, two "
                                  "Gaussian flavour sources; even/odd CG to 1e-10",
                      "sloppy": f"f32:{sl}, delta {delta}", **drows,
                      "apply_Dh_ms": round(t / 5 * 1e3, 4),
                      "timing": "3 solves / 5 applications, CUDA events, L2 flushed before each"}
    out["chrono_guess"] = {"workload": f"{w.name}, 8 slowly varying sources, N_CSG = 4, FP64 CG on "
                                       "Qhat^+ Qhat^- to 1e-10",
                           "iters_cold": cold_iters, "iters_with_guess": warm_iters,
                           "seconds_cold": round(t_cold, 4), "seconds_with_guess": round(t_warm, 4),
                           "speedup": round(t_cold / t_warm, 3)}
    return out


# -------------------------------------------------------------- CPU oracle ---
class OracleSample:
    """The oracle's even/odd FP64 CG on one workload, as it stands, timed in bounded samples: the
    source preparation and the reconstruction once (`fixed`), then CG iterations in samples of
    about `seconds` (at least one iteration each).  The oracle's CG applies the operator once for
    its initial residual and once more for the final check: one application (`t_A`, timed once) is
    taken off each sample, and a solve is modelled as fixed + 2 t_A + iterations x (time per
    iteration)."""

    def __init__(self, w, U, phi):
        import numpy as np

        import oracle
        self.w, self.U = w, U
        self.lat = oracle.Lattice.cubic(w.T, w.L)
        t0 = time.perf_counter()
        varphi = oracle.eo_prepare(self.lat, U, phi, w.kappa, w.mu)
        t1 = time.perf_counter()
        odd = self.lat.parity_mask()[..., None, None]
        self.b = np.where(odd, varphi, 0) * np.array([1, 1, -1, -1])[:, None]
        t2 = time.perf_counter()
        oracle.eo_reconstruct(self.lat, U, varphi, np.where(odd, self.b, 0), w.kappa, w.mu)
        t3 = time.perf_counter()
        oracle.normal_op(self.lat, U, self.b, w.kappa, w.mu)
        self.t_A = time.perf_counter() - t3
        # one preparation, one reconstruction (whose x_o = Qhat^- X costs as much again), and the
        # CG's initial and final operator applications
        self.fixed = (t1 - t0) + 2 * (t3 - t2) + 2 * self.t_A

    def iterations(self, seconds: float):
        """Runs CG iterations for about `seconds` (at least one); returns (seconds per iteration,
        iterations run)."""
        import oracle
        w = self.w
        n, t, k = 0, 0.0, 1
        while n == 0 or t < seconds:
            t1 = time.perf_counter()
            res = oracle.cg(self.lat, self.U, self.b, w.kappa, w.mu, tol=1e-30, max_iter=k)
            t += max(0.0, time.perf_counter() - t1 - self.t_A)
            n += res.iters
            k = min(2 * k, 64)
        return t / n, n


def cpu_baseline(w, U, phi, iters, seconds):
    import oracle
    smp = OracleSample(w, U, phi)
    t_it, n = smp.iterations(seconds)
    per_solve = t_it * iters + smp.fixed
    return {"value": round(1.0 / per_solve, 8), "unit": "solves/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"oracle FP64 CG on {w.name}: {n} iterations timed ({t_it:.3f} s each), extrapolated "
                      f"to the {iters} iterations of the GPU FP64 CG, plus one source preparation, "
                      f"reconstruction and the CG's initial and final residuals ({smp.fixed:.2f} s, timed)"}


def cpu_oracle_operator(w, U, phi, gpu_us, seconds: float = 2.0):
    """The oracle's H_oe (FP64, full 4x4 (1 +- gamma) matrices, OpenMP site loop) timed on the host
    for about `seconds`, beside the FP64 GPU hopping kernel on the same lattice."""
    import oracle
    olat = oracle.Lattice.cubic(w.T, w.L)
    oracle.hopping(olat, U, phi, out_parity=1)
    n, t0 = 0, time.perf_counter()
    while True:
        oracle.hopping(olat, U, phi, out_parity=1)
        n += 1
        dt = time.perf_counter() - t0
        if dt >= seconds:
            break
    per = dt / n
    h = w.V // 2
    return {"kernel": "oracle hopping H_oe, FP64", "workload": w.name, "applications": n,
            "ms_per_application": round(per * 1e3, 3), "cores": oracle.num_threads(),
            "gbs_algorithmic": round(hop_bytes_per_site(0, 18) * h / per / 1e9, 2),
            "gflops": round(HOP_FLOPS * h / per / 1e9, 2),
            "gpu_fp64_kernel_speedup": round(per / (gpu_us * 1e-6), 1)}


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, each step a bounded sample of the workload
    (CG iterations), extrapolated to one complete solve."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_0905_3331_gb300 import inputs
    w = inputs.WORKLOADS[args.workload]
    U, phi = w.gauge(), w.source()
    iters, how = args.ref_iters, "given"
    if iters <= 0 and w.name in FP64_CG_ITERS:
        iters, how = FP64_CG_ITERS[w.name], "of the FP64 CG to 1e-10 on this system, measured on GB300"
    elif iters <= 0:  # small workloads: one complete oracle solve gives the iteration count
        res = oracle.solve(oracle.Lattice.cubic(w.T, w.L), U, phi, w.kappa, w.mu, tol=1e-10)
        iters, how = res.iters, "of the oracle's own complete FP64 solve to 1e-10"
    smp = OracleSample(w, U, phi)
    for _ in range(args.warmup):
        smp.iterations(0.0)
    # each step's sample: --ref-seconds, shortened so that all steps together take about
    # REF_TOTAL_SECONDS of host time (at least one CG iteration per step)
    step_seconds = min(args.ref_seconds, max(0.5, REF_TOTAL_SECONDS / max(1, args.steps)))
    per_step, n_it = [], 0
    t_host = time.perf_counter()
    for _ in range(args.steps):
        t_it, n = smp.iterations(step_seconds)
        n_it += n
        per_step.append(t_it * iters + smp.fixed)
    t_host = time.perf_counter() - t_host
    tot = sum(per_step)
    value = args.steps / tot
    cb = {"value": round(value, 8), "unit": "solves/s", "cores": oracle.num_threads(),
          "kind": "oracle",
          "sample": f"each step: oracle FP64 CG iterations on {w.name} for ~{step_seconds:.2g} s (at least one; "
                    f"{n_it} in all), extrapolated to {iters} iterations per solve ({how}), plus one source "
                    f"preparation, reconstruction and the CG's initial and final residuals ({smp.fixed:.2f} s, "
                    "timed once)"}
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 8), "unit": "solves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(tot / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{w.name} lattice (V = {w.V}), random SU(3) links eps {w.eps}, kappa {w.kappa}, "
                               f"mu {w.mu}, Gaussian source; even/odd CG to FP64 true residual 1e-10",
                   "lattice": w.name},
        "cpu_baseline": cb,
        # ms_per_step is the modelled time of one complete solve; the host time a step's sample took:
        "sample_ms_per_step": round(t_host / max(1, args.steps) * 1e3, 3),
        "e2e": {"value": round(value, 8), "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="48^3x96")
    ap.add_argument("--sloppy", default=None, help="sloppy storage:links, e.g. f32:12, f16:8 (default per workload)")
    ap.add_argument("--delta", type=float, default=None, help="reliable-update delta (default per workload)")
    ap.add_argument("--update-prec", default=None, choices=["f64", "f32"],
                    help="arithmetic of the residual recomputations between FP64 ones (default per workload)")
    ap.add_argument("--batched-delta", type=float, default=1e-3,
                    help="reliable-update delta of the batched measurement (24^3x48 systems)")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--hop-iters", type=int, default=50)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-solve measurement")
    ap.add_argument("--no-link-form", action="store_true",
                    help="skip the 12-real-link solve beside an 8-real headline")
    ap.add_argument("--no-precision-form", action="store_true",
                    help="skip the 32^3x64 roofline and mixed-vs-FP64 solve measurement")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the 16^3x32 baseline and the BiCGstab, chronological-guess and doublet measurements")
    ap.add_argument("--ref-seconds", type=float, default=8.0)
    ap.add_argument("--ref-iters", type=int, default=0,
                    help="CG iterations per solve used to scale the reference arm's sample (0: the table of "
                         "measured FP64 CG counts, else one complete oracle solve)")
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu dram bytes per launch of the sloppy hopping kernel, if measured")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)  # at least 3 warm-up steps, always
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
