#!/usr/bin/env python3
"""Benchmark of the even-odd Wilson-Dirac operator on one GB300 (or N replicas).

Metric: "Dirac-op GB/s & % HBM peak at 48^4 SU(2); mixed vs FP64 CG time to
1e-10".  One step is one even-odd Dirac application of the whole 48^4 lattice
in the SU(2) fundamental representation, FP64: out_e = D_eo in_o and
out_o = D_oe in_e (two launches of the hop kernel, every site once).  Its
throughput counts the compulsory bytes of the hop (per output site: the input
spinor once, the output spinor once and 8 quaternion links = 512 B in FP64).
The CG half of the metric (32^4, FP64 vs FP32/FP16-inner mixed precision,
true residual 1e-10) and the other precisions/representations are measured
after the timed region and reported under "extras".

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun every rank runs an independent replica (the single-GPU hot path
has no data exchange); value = the bytes all ranks processed / max rank time.
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
sys.path.insert(0, ROOT)

METRIC = "Dirac-op GB/s & % HBM peak at 48^4 SU(2); mixed vs FP64 CG time to 1e-10"
DIMS = (48, 48, 48, 48)
GAUGE_SEED, SPINOR_SEED = 1003, 2003
HBM_FALLBACK = 6800.0
HBM_NOMINAL_GBS = 8000.0  # the HBM3e figure the target is quoted against
# Wilson hopping-term flops per output site, 8*16*Nc^2 + 7*4*Nc*2 (fund 624,
# adjoint with real 3x3 links 744), the convention of the paper's field
HOP_FLOPS = {"fund": 624, "adj": 744}
# FP32-pipe roofline of GB300: 152 SMs x 128 FP32 lanes x 2.07 GHz (maximum SM clock)
FP32_PEAK_GOPS = 152 * 128 * 2.070
# Essential FP32-pipe operations per output site of the double-float fundamental hop
# (TwoSum = 6, TwoProduct with cross terms = 4, double-float add = 8): per direction
# 8 projection adds (64) + 8 colour-product outputs of 4 products and 3 adds each
# (320) = 384, and 16 reconstruction adds (128) for every direction but the first
# (which assigns); the epilogue scales (32) and renormalises (96) the 16 reals.
DF_OPS_PER_SITE_FUND = 8 * 384 + 7 * 128 + 32 + 96
# kernel symbol of each hop variant (the tuner's index)
HOP_KERNELS = ["k_hop", "k_hop_staged", "k_hop_loop", "k_hop_loop", "k_hop_sw", "k_hop_sw", "k_hop_pf",
               "k_hop_r96", "k_hop_tile", "k_hop_tile_r96", "k_hop_x2", "k_hop_x2s", "k_hop_x2_r96",
               "k_hop_x2s_r96", "k_hop_h16", "k_hop_h16_r64", "k_hop_p2", "k_hop_p2_r96",
               "k_hop_h16s", "k_hop_h16s_r64"]
HOP_VARIANT_NAMES = ["unrolled", "unrolled cp.async staged", "generic loop", "generic loop staged",
                     "switched loop", "switched loop staged", "unrolled register prefetch",
                     "unrolled, 96 registers", "bulk-copy tiled", "bulk-copy tiled, 96 registers",
                     "paired f32x2", "paired f32x2, cp.async staged",
                     "paired f32x2, 96 registers", "paired f32x2, cp.async staged, 96 registers",
                     "binary16, half2 projection", "binary16, half2 projection, 64 registers",
                     "two sites per thread (f32x2 lanes)", "two sites per thread (f32x2 lanes), 96 registers",
                     "binary16, half2 projection, cp.async staged",
                     "binary16, half2 projection, cp.async staged, 64 registers",
                     "2 right-hand sides per thread", "4 right-hand sides per thread",
                     "binary16, half2 projection, register prefetch, 80 registers",
                     "binary16, half2 projection, register prefetch two directions ahead, 96 registers"]


def variant_name(rep, variant):
    """The tuned kernel's name; variant 12 of the adjoint FP64 hop is the paired
    kernel with 168 registers (96 for the fundamental)."""
    if variant == 12 and rep != 0:
        return "paired f32x2, 168 registers"
    return HOP_VARIANT_NAMES[variant] if 0 <= variant < len(HOP_VARIANT_NAMES) else str(variant)


def roofline(pname, vh, bytes_site, launch_ms, achieved_gbs, peak_gbs, peak_kind, traffic, kernel, fma=None):
    """The dominant kernel's roofline against HBM: compulsory bytes per launch
    over the launch time, against the measured copy peak.  For the FP64 class
    an "alu" view sits beside it: the double-float hop needs 4096 FP32-pipe
    lane operations per site (the implementation's count, not the method's
    624 flops), against the FP32 FMA rate measured on this GPU (fma: the
    library's calibration, scalar and packed lane ops per second)."""
    out = {"bound": "hbm", "achieved": round(achieved_gbs, 2), "peak": peak_gbs, "unit": "GB/s",
           "frac": round(achieved_gbs / peak_gbs, 4), "peak_kind": f"{peak_kind} HBM copy (burst), of measured",
           "traffic": traffic, "kernel": kernel, "bytes_per_launch": vh * bytes_site,
           "avg_launch_ms": round(launch_ms, 5)}
    if pname == "f64":
        sites_per_s = vh / (launch_ms * 1e-3)
        gops = sites_per_s * DF_OPS_PER_SITE_FUND / 1e9
        alu = {"achieved": round(gops, 1), "unit": "Gop/s (FP32 lane ops)", "ops_per_site": DF_OPS_PER_SITE_FUND,
               "ops_note": "the double-float implementation's FP32-pipe operations per site (the method: 624 flops)",
               "nominal_peak": round(FP32_PEAK_GOPS, 1), "nominal_kind": "152 SMs x 128 FP32 lanes x 2.07 GHz",
               "frac_of_nominal": round(gops / FP32_PEAK_GOPS, 4)}
        if fma:
            peak = max(fma) / 1e9
            alu.update({"peak": round(peak, 1), "peak_kind": "measured FP32 FMA rate (hr_fp32_fma_rate, best of "
                        "scalar / packed, operand-reuse best case)", "frac": round(gops / peak, 4),
                        "measured_scalar": round(fma[0] / 1e9, 1), "measured_paired": round(fma[1] / 1e9, 1)})
        out["alu"] = alu
    return out


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-extras", action="store_true", help="skip the CG and precision sweep")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-autotune", action="store_true", help="use the default hop launch shape")
    ap.add_argument("--lattice", type=int, default=48,
                    help="L of the L^4 lattice (48 is the benchmark workload; smaller for profiling)")
    ap.add_argument("--prec", choices=["f64", "f32", "f16"], default="f64",
                    help="hop precision of the timed step (f64 is the benchmark workload)")
    ap.add_argument("--rep", choices=["fund", "adj", "adjmat"], default="fund",
                    help="representation of the timed step (fund is the benchmark workload; adj: quaternion "
                         "links, adjoint matrices rebuilt in registers; adjmat: stored 3x3 links)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks_fn(dist, device):
    """x -> the maximum of x over the ranks of the default process group (the
    slowest replica's time); the identity without one."""
    def max_over_ranks(x: float) -> float:
        if dist is None:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return max_over_ranks


def replica_value(world: int, units_per_step: float, ms_per_step: float) -> float:
    """Whole-job throughput of `world` replicas that each process units_per_step
    per step, timed by the slowest rank: units per second."""
    return world * units_per_step / (ms_per_step * 1e-3)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK, "fallback"


def hop_bytes_per_site(rep: str, prec: str) -> int:
    """Compulsory bytes per output site of one hop: 1 spinor in, 1 out, 8 links."""
    spinor = {"f64": 16 * 8, "f32": 16 * 4, "f16": 16 * 2 + 4}
    link = {"f64": 32, "f32": 16, "f16": 8}
    nspin = {"fund": 1.0, "adj": 1.5}[rep]
    return int(2 * spinor[prec] * nspin + 8 * link[prec])


def neighbour_bytes_per_site(rep: str, prec: str) -> int:
    spinor = {"f64": 16 * 8, "f32": 16 * 4, "f16": 16 * 2 + 4}
    link = {"f64": 32, "f32": 16, "f16": 8}
    nspin = {"fund": 1.0, "adj": 1.5}[rep]
    return int(9 * spinor[prec] * nspin + 8 * link[prec])


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2411_18511_gb300", "csrc")
    for f in ("hr_internal.cuh", "hr_clover.cuh", "hr_host.h", "hr_hop_dev.cuh", "hr_hop_fam.h", "hr_hop_x2.cuh",
              "hr_hop.cu", "hr_hop_staged.cu", "hr_hop_loop.cu", "hr_hop_tile.cu", "hr_hop_x2.cu", "hr_hop_half.cu",
              "hr_hop_p2.cu", "hr_hop_chunk.cu"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(name: str, variant: int, block: int):
    """Per-launch DRAM bytes of the hop kernel in launch shape (variant, block)
    from a committed ncu summary ('traffic_bytes_per_launch v<variant> b<block>:'
    lines), if it was taken on the current kernel source (its 'source_hash:'
    line must match); else None."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        txt = open(path).read()
    except OSError:
        return None
    vals = {}
    for line in txt.splitlines():
        if ":" in line and line.strip().startswith(("traffic_bytes_per_launch", "source_hash")):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_hash") != kernel_source_hash():
        return None
    try:
        return float(vals[f"traffic_bytes_per_launch v{variant} b{block}"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock/throttle samples taken while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return

        def reader():
            for line in self.proc.stdout:
                self.lines.append(line.strip())

        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_smi_id(torch, dev: int) -> str:
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev)


# ----------------------------------------------------------------------------- ours

def run_ours(args):
    import torch
    from paper_2411_18511_gb300 import hr, fields
    import synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    max_over_ranks = max_over_ranks_fn(dist, "cuda")

    ctx = hr.Context(local)
    L4 = args.lattice
    dims = (L4,) * 4
    V = int(np.prod(dims))
    Vh = V // 2
    pname = args.prec
    rname = args.rep
    rep = {"fund": hr.HR_FUND, "adj": hr.HR_ADJ, "adjmat": hr.HR_ADJ_MAT}[rname]
    prec = {"f64": hr.HR_F64, "f32": hr.HR_F32, "f16": hr.HR_F16}[pname]
    q = synth.haar_links(dims, GAUGE_SEED)
    psi = synth.gaussian_spinor(dims, 2, SPINOR_SEED) if rname == "fund" else synth.gaussian_spinor(dims, 3, 2004)
    gauge = fields.pack_gauge(ctx, dims, rep, prec, fields.gauge_to_device(q))
    src = fields.pack_spinor(ctx, dims, rep, prec, hr.HR_FULL, fields.spinor_to_device(psi))
    dst = fields.empty_spinor(dims, rep, prec, hr.HR_FULL)
    half = hr.hr_spinor_packed_bytes(dims, rep, prec, hr.HR_EVEN, 1)
    stream = torch.cuda.current_stream()
    s_ptr = stream.cuda_stream
    L = hr.lib()
    lat = hr.lattice(dims)
    p_g, p_s, p_d = gauge.data_ptr(), src.data_ptr(), dst.data_ptr()
    tuned = None
    if not args.no_autotune:
        # pick the hop kernel's launch shape for this configuration (untimed set-up)
        res = hr.hr_autotune_hop(ctx, dims, rep, prec, hr.HR_EVEN, 1, gauge, p_s + half, p_d, reps=20)
        tuned = {"variant": variant_name(rep, res.variant),
                 "block": res.block,
                 "tuned_ms": round(res.best_ms, 5), "default_ms": round(res.default_ms, 5),
                 "shapes_timed": res.candidates}

    def step():
        # out_e = D_eo in_o ; out_o = D_oe in_e   (two hop launches)
        rc = L.hr_dirac_eo(ctx.handle, lat, 0.0, rep, prec, hr.HR_EVEN, hr.HR_OP_HOP, 1, p_g,
                           p_s + half, p_d, None, 0, s_ptr)
        rc |= L.hr_dirac_eo(ctx.handle, lat, 0.0, rep, prec, hr.HR_ODD, hr.HR_OP_HOP, 1, p_g,
                            p_s, p_d + half, None, 0, s_ptr)
        if rc:
            ctx.check(rc)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_smi_id(torch, local))
    sampler.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms_step = max_over_ranks(e0.elapsed_time(e1)) / args.steps
    fma = hr.hr_fp32_fma_rate(ctx) if pname == "f64" else None  # the FP32 pipe's measured rate (untimed)
    hr.hr_ctx_status(ctx)  # every packed value was in range
    variant, block = hr.hr_tune_lookup(ctx, dims, rep, prec)
    kname = HOP_KERNELS[variant] if 0 <= variant < len(HOP_KERNELS) else str(variant)
    if pname != "f64" and kname in ("k_hop_x2", "k_hop_x2s"):
        kname = kname.replace("x2", "f2")  # the FP32-arithmetic paired kernels
    kernel = f"{kname}<{rname},{pname}> x{block}"
    bytes_site = hop_bytes_per_site("fund" if rname == "fund" else "adj", pname)
    if rname == "adjmat":  # stored 3x3 real links instead of quaternions
        bytes_site += 8 * ({"f64": 72, "f32": 36, "f16": 18}[pname] - {"f64": 32, "f32": 16, "f16": 8}[pname])
    bytes_step = 2 * Vh * bytes_site
    value = replica_value(world, bytes_step, ms_step) / 1e9
    launch_ms = ms_step / 2.0  # the step is exactly two launches of the hop kernel
    achieved = Vh * bytes_site / (launch_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()

    e2e = None
    if not args.no_e2e and rname == "fund":
        e2e = run_e2e(args, ctx, torch, hr, dims, rep, prec, psi, src, dst, step, stream,
                      max_over_ranks, world, bytes_step)
    extras, sols = {}, None
    if not args.no_extras and rank == 0:
        extras, sols = run_extras(ctx, torch, hr, fields, synth, q, psi)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and rname == "fund":
        cpu = cpu_baseline(q, psi, dims, sols)
        attach_oracle_checks(extras, cpu)

    gauge_mb = hr.hr_gauge_packed_bytes(dims, rep, prec) / 1e6
    result = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"f64": "df64", "f32": "f32", "f16": "f16"}[pname],
        "data": "synthetic (Haar-random SU(2) links, Gaussian complex source, Philox seeds 1003/2003)",
        "config": {
            "workload": (f"even-odd Wilson-Dirac hop pair D_eo+D_oe, {L4}^4 SU(2) "
                         f"{ {'fund': 'fundamental', 'adj': 'adjoint', 'adjmat': 'adjoint (3x3 links)'}[rname]}, "
                         f"{pname.upper()}"),
            "lattice": list(dims), "rep": rname, "prec": pname,
            "arithmetic": ("double-float: each real an unevaluated pair of fp32 (hi + lo), TwoSum/"
                           "TwoProduct on the FP32 pipes, ~2^-48 relative" if pname == "f64" else pname),
            "launch": tuned,
            "bytes_per_site": bytes_site,
            "byte_convention": "compulsory (1 spinor in + 1 out + 8 quaternion links)",
            "neighbour_counted_gbs": round(value * (neighbour_bytes_per_site("fund" if rname == "fund" else "adj", pname)
                                                    + bytes_site - hop_bytes_per_site(
                                                        "fund" if rname == "fund" else "adj", pname)) / bytes_site, 2),
            "gflops": round(value * HOP_FLOPS["fund" if rname == "fund" else "adj"] / bytes_site, 1),
            "pct_of_nominal_8000": round(100 * value / HBM_NOMINAL_GBS, 1),
            "l2": f"inputs larger than L2 (gauge {gauge_mb:.0f} MB + spinor half {half / 1e6:.0f} MB per launch)",
            "parallelism": f"replicas{world}",
        },
        "roofline": roofline(pname if rname == "fund" else "", Vh, bytes_site, launch_ms, achieved, peak,
                             peak_kind, profiled_traffic(f"hop_{rname}_{pname}_{L4}x{L4}x{L4}x{L4}.md", variant, block),
                             kernel, fma),
        "e2e": e2e,
        "gpu_launches": 2 * args.steps,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "extras": extras,
    }
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_e2e(args, ctx, torch, hr, dims, rep, prec, psi, src, dst, step, stream, max_over_ranks, world,
            bytes_step, nbuf=3):
    """The same step through the public API from pinned host memory: H2D of the
    canonical spinor, pack, the two hops, unpack, D2H; all inside the timing.
    Steps are pipelined over three streams with three device buffer sets, so
    the H2D copy of step k+1 and the D2H copy of step k-1 overlap step k's
    kernels (the link carries both directions at once); every step still moves
    its whole input to the device and its whole result back.  Beside it, the
    same H2D and D2H copies alone (host_link): the ceiling the link sets."""
    host_in = torch.view_as_real(torch.from_numpy(psi)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    dev_in = [torch.empty(host_in.shape, dtype=torch.float64, device="cuda") for _ in range(nbuf)]
    dev_out = [torch.empty_like(dev_in[0]) for _ in range(nbuf)]
    s_h2d, s_d2h = torch.cuda.Stream(), torch.cuda.Stream()
    h2d_done = [torch.cuda.Event() for _ in range(nbuf)]
    comp_done = [torch.cuda.Event() for _ in range(nbuf)]
    d2h_done = [torch.cuda.Event() for _ in range(nbuf)]
    used = [False] * nbuf

    def e2e_step(k):
        b = k % nbuf
        if used[b]:
            s_h2d.wait_event(comp_done[b])  # step k-nbuf has read dev_in[b]
        with torch.cuda.stream(s_h2d):
            dev_in[b].copy_(host_in, non_blocking=True)
        h2d_done[b].record(s_h2d)
        stream.wait_event(h2d_done[b])
        hr.hr_spinor_pack(ctx, dims, rep, prec, hr.HR_FULL, 1, dev_in[b], src, stream)
        step()
        if used[b]:
            stream.wait_event(d2h_done[b])  # step k-nbuf's result has left dev_out[b]
        hr.hr_spinor_unpack(ctx, dims, rep, prec, hr.HR_FULL, 1, dst, dev_out[b], stream)
        comp_done[b].record(stream)
        s_d2h.wait_event(comp_done[b])
        with torch.cuda.stream(s_d2h):
            host_out.copy_(dev_out[b], non_blocking=True)
        d2h_done[b].record(s_d2h)
        used[b] = True

    # warm-up: a whole untimed pass (the first pass through freshly pinned
    # buffers runs about 10 % slower than the ones after it)
    n_e2e = max(6, min(50, args.steps // 20))
    for k in range(n_e2e):
        e2e_step(k)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s_h2d.wait_event(e0)
    s_d2h.wait_event(e0)
    for k in range(n_e2e):
        e2e_step(n_e2e + k)
    stream.wait_event(d2h_done[(2 * n_e2e - 1) % nbuf])
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / n_e2e)
    # the host link's ceiling for this traffic: the same H2D and D2H copies
    # alone, concurrent on their two streams, no kernels
    for k in range(2):
        with torch.cuda.stream(s_h2d):
            dev_in[0].copy_(host_in, non_blocking=True)
        with torch.cuda.stream(s_d2h):
            host_out.copy_(dev_out[0], non_blocking=True)
    torch.cuda.synchronize()
    e0.record(stream)
    s_h2d.wait_event(e0)
    s_d2h.wait_event(e0)
    for k in range(n_e2e):
        with torch.cuda.stream(s_h2d):
            dev_in[0].copy_(host_in, non_blocking=True)
        with torch.cuda.stream(s_d2h):
            host_out.copy_(dev_out[0], non_blocking=True)
    h2d_done[0].record(s_h2d)
    d2h_done[0].record(s_d2h)
    stream.wait_event(h2d_done[0])
    stream.wait_event(d2h_done[0])
    e1.record(stream)
    torch.cuda.synchronize()
    copy_ms = max_over_ranks(e0.elapsed_time(e1) / n_e2e)
    link_bytes = 2 * host_in.numel() * 8
    return {"value": round(world * bytes_step / (e2e_ms * 1e-3) / 1e9, 2), "unit": "GB/s",
            "h2d_bytes_per_step": int(host_in.numel() * 8), "d2h_bytes_per_step": int(host_out.numel() * 8),
            "ms_per_step": round(e2e_ms, 4),
            "host_link": {"copies_only_ms_per_step": round(copy_ms, 4),
                          "copies_only_gbs": round(link_bytes / (copy_ms * 1e-3) / 1e9, 1),
                          "e2e_link_gbs": round(link_bytes / (e2e_ms * 1e-3) / 1e9, 1),
                          "frac_of_copies_only": round(copy_ms / e2e_ms, 3)},
            "path": "pinned host canonical spinor -> H2D -> hr_spinor_pack -> 2x hr_dirac_eo -> "
                    "hr_spinor_unpack -> D2H, pipelined over 3 streams (H2D, kernels, D2H)"}


def time_hop(ctx, torch, hr, fields, dims, rep, prec, q, psi, steps=100, peak=None):
    """Average GB/s of one hop launch (compulsory bytes) for a rep/prec, with
    the autotuner's launch shape for the configuration."""
    gauge = fields.pack_gauge(ctx, dims, rep, prec, fields.gauge_to_device(q))
    src = fields.pack_spinor(ctx, dims, rep, prec, hr.HR_ODD, psi)
    dst = fields.empty_spinor(dims, rep, prec, hr.HR_EVEN)
    res = hr.hr_autotune_hop(ctx, dims, rep, prec, hr.HR_EVEN, 1, gauge, src, dst, reps=10)
    for _ in range(20):
        hr.hr_dirac_eo(ctx, dims, 0.0, rep, prec, hr.HR_EVEN, hr.HR_OP_HOP, 1, gauge, src, dst)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        hr.hr_dirac_eo(ctx, dims, 0.0, rep, prec, hr.HR_EVEN, hr.HR_OP_HOP, 1, gauge, src, dst)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    Vh = int(np.prod(dims)) // 2
    rname = "fund" if rep == hr.HR_FUND else "adj"
    pname = {hr.HR_F64: "f64", hr.HR_F32: "f32", hr.HR_F16: "f16"}[prec]
    b = hop_bytes_per_site(rname, pname)
    nb = neighbour_bytes_per_site(rname, pname)
    if rep == hr.HR_ADJ_MAT:
        extra = 8 * ({"f64": 72, "f32": 36, "f16": 18}[pname] - {"f64": 32, "f32": 16, "f16": 8}[pname])
        b += extra
        nb += extra
    gbs = Vh * b / (ms * 1e-3) / 1e9
    out = {"ms": round(ms, 5), "gbs": round(gbs, 1), "bytes_per_site": b,
           "gbs_neighbour_counted": round(Vh * nb / (ms * 1e-3) / 1e9, 1),
           "gflops": round(Vh * HOP_FLOPS[rname] / (ms * 1e-3) / 1e9, 1),
           "pct_of_nominal_8000": round(100 * gbs / HBM_NOMINAL_GBS, 1),
           "launch": {"variant": variant_name(rep, res.variant), "block": res.block}}
    if peak:
        out["pct_of_measured_copy"] = round(100 * gbs / peak, 1)
    return out


def run_extras(ctx, torch, hr, fields, synth, q48, psi48):
    out = {}
    dims = DIMS
    dq = None
    # precision / representation sweep of the hop at 48^4 (config: adjoint FP64 and FP32, 200 applications)
    fund_psi = fields.spinor_to_device(psi48)
    for prec in (hr.HR_F32, hr.HR_F16):
        out[f"hop_fund_{ {1: 'f32', 2: 'f16'}[prec]}_48"] = time_hop(ctx, torch, hr, fields, dims, hr.HR_FUND, prec, q48,
                                                                      fund_psi, peak=measured_peaks()[0])
    del fund_psi
    adj_psi = fields.spinor_to_device(synth.gaussian_spinor(dims, 3, 2004))
    for rep, rn in ((hr.HR_ADJ, "adj"), (hr.HR_ADJ_MAT, "adjmat")):
        for prec in (hr.HR_F64, hr.HR_F32):
            out[f"hop_{rn}_{ {0: 'f64', 1: 'f32'}[prec]}_48"] = time_hop(
                ctx, torch, hr, fields, dims, rep, prec, q48, adj_psi, steps=200, peak=measured_peaks()[0])
    del adj_psi
    torch.cuda.empty_cache()
    # CG time to solution at 32^4 (smeared links, plaquette ~0.6, m0 = -0.2, tol 1e-10)
    d32 = (32, 32, 32, 32)
    t0 = time.time()
    q32, nsm, plaq = synth.ape_smear_to_plaquette(synth.haar_links(d32, 1002), d32, 0.6)
    b = synth.gaussian_spinor(d32, 2, 2002)
    gauge = fields.pack_gauge(ctx, d32, hr.HR_FUND, hr.HR_F64, fields.gauge_to_device(q32))
    bp = fields.pack_spinor(ctx, d32, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, fields.spinor_to_device(b))
    cg = {"lattice": list(d32), "m0": -0.2, "tol": 1e-10, "plaquette": round(plaq, 4), "ape_steps": nsm,
          "setup_s": round(time.time() - t0, 1)}
    # the solvers use the context's tuned hop shapes: tune every precision they use at this size
    bdev = fields.spinor_to_device(b)
    for prec in (hr.HR_F64, hr.HR_F32, hr.HR_F16):
        gp = fields.pack_gauge(ctx, d32, hr.HR_FUND, prec, fields.gauge_to_device(q32))
        src = fields.pack_spinor(ctx, d32, hr.HR_FUND, prec, hr.HR_ODD, bdev)
        dst = fields.empty_spinor(d32, hr.HR_FUND, prec, hr.HR_EVEN)
        hr.hr_autotune_hop(ctx, d32, hr.HR_FUND, prec, hr.HR_EVEN, 1, gp, src, dst, reps=10)
        del gp, src, dst
    xp = fields.zeros_spinor(d32, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN)
    sols = {"cg_32": {"dims": d32, "q": q32, "b": b, "x": {}}}
    for name, inner, deltas in (("fp64", hr.HR_F64, (0.1,)),
                                ("mixed_f32", hr.HR_F32, (0.1, 1e-2, 1e-3, 1e-4, 1e-5)),
                                ("mixed_f16", hr.HR_F16, (0.1, 3e-2, 1e-2, 3e-3))):
        sweep = {}
        best = None
        for delta in deltas:
            opts = hr.hr_solver_default_opts()
            opts.inner_prec = inner
            opts.reliable_delta = delta
            work = fields.empty_bytes(hr.hr_cg_workspace_bytes(d32, hr.HR_FUND, opts))
            times = []
            info = rc = None
            for rep_i in range(6):  # one warm-up solve (it also captures the solve graph), five timed
                rc, info = hr.hr_cg_solve(ctx, d32, -0.2, hr.HR_FUND, opts, gauge, bp, xp, work)
                times.append(info.seconds)
            rec = {"status": hr.STATUS_NAMES.get(rc, rc), "seconds_median": round(statistics.median(times[1:]), 4),
                   "first_solve_s": round(times[0], 4), "timed_solves": len(times) - 1, "iters": info.iters,
                   "reliable_updates": info.n_reliable_updates, "true_rel_residual": info.true_rel_residual,
                   "reliable_delta": delta}
            sweep[str(delta)] = rec["seconds_median"]
            if rc == hr.HR_OK and (best is None or rec["seconds_median"] < best["seconds_median"]):
                best = rec
                sols["cg_32"]["x"][name] = fields.unpack_spinor(ctx, d32, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN,
                                                                xp).cpu().numpy()
            del work
        cg[name] = dict(best or rec)
        if len(deltas) > 1:
            cg[name]["delta_sweep_s"] = sweep
    if "fp64" in cg and cg["fp64"]["seconds_median"] > 0:
        for k in ("mixed_f32", "mixed_f16"):
            cg[k]["speedup_vs_fp64"] = round(cg["fp64"]["seconds_median"] / cg[k]["seconds_median"], 3)
    out["cg_32"] = cg
    out["cg_32_clover"] = run_cg_clover(ctx, hr, fields, d32, q32, gauge, bp, xp, cg)
    del gauge, bp
    torch.cuda.empty_cache()
    out["clover_48"] = run_clover_48(ctx, torch, hr, fields, q48, psi48)
    torch.cuda.empty_cache()
    out["twist_48"] = run_twist_48(ctx, torch, hr, fields, q48, psi48)
    torch.cuda.empty_cache()
    out["dd_48"] = run_dd_48(ctx, torch, hr, fields, q48, psi48)
    torch.cuda.empty_cache()
    out["diff_solve_16"] = run_diff_solve(torch, synth)
    torch.cuda.empty_cache()
    out["multi_rhs_24"], sols["multi_rhs_24"] = run_multi_rhs(ctx, torch, hr, fields, synth)
    torch.cuda.empty_cache()
    out["batch_12"] = run_batch(ctx, torch, hr, fields, synth)
    torch.cuda.empty_cache()
    out["hmc_16"] = run_hmc(ctx, torch, hr, fields, synth)
    return out, sols


def run_hmc(ctx, torch, hr, fields, synth):
    """16^4 HMC with two flavours of Wilson fermions (beta = 2.2, m0 = -0.2,
    antiperiodic time, tau = 1): wall time of one trajectory (MD through
    hr_hmc_trajectory, with its CG solves), Delta H, force evaluations, for
    leapfrog and Omelyan at the same number of force evaluations, FP64 /
    FP16-inner solvers, Hasenbusch's two pseudofermions (heavy m0 = 0.2), and
    two time scales (6 outer Omelyan steps on the pseudofermion force, 3 gauge
    steps per outer link update: half the fermion forces); a short chain from a
    thermalised start for the acceptance, and clover fermions (c_sw = 1) on two
    time scales.  force_evaluations counts pseudofermion forces (each one or
    two solves)."""
    from paper_2411_18511_gb300.hmc import HMC
    lat = hr.Lattice((16, 16, 16, 16), 1)
    beta, m0 = 2.2, -0.2
    q0, _, plaq = synth.ape_smear_to_plaquette(synth.haar_links(lat, 1006), lat, 0.6)
    qd0 = fields.gauge_to_device(q0)
    # thermalisation: molecular dynamics from fresh momenta, kept without a Metropolis test
    warm = HMC(ctx, lat, beta=beta, m0=m0, fermions=True, n_steps=12, tau=1.0, seed=3006)
    for _ in range(30):
        eta = warm.draw_pseudofermion(qd0)
        info = hr.hr_hmc_trajectory(ctx, lat, warm.prm, qd0, warm.draw_momenta(), eta, warm.work)
    del warm
    out = {"lattice": list(lat), "beta": beta, "m0": m0, "tau": 1.0, "bc": "antiperiodic in time",
           "smeared_start_plaquette": round(plaq, 4), "thermalised_plaquette": round(info.plaquette, 4),
           "thermalisation": "30 Omelyan trajectories of 12 steps without accept/reject"}
    om = hr.HR_INTEGRATOR_OMELYAN
    for name, integ, steps, inner, mh, m in (("leapfrog_f64", hr.HR_INTEGRATOR_LEAPFROG, 24, hr.HR_F64, None, 1),
                                             ("omelyan_f64", om, 12, hr.HR_F64, None, 1),
                                             ("omelyan_f16_inner", om, 12, hr.HR_F16, None, 1),
                                             ("omelyan_f16_inner_hasenbusch", om, 12, hr.HR_F16, 0.2, 1),
                                             ("omelyan_f16_inner_2scales", om, 6, hr.HR_F16, None, 3),
                                             ("omelyan_f16_inner_hasenbusch_2scales", om, 6, hr.HR_F16, 0.2, 3),
                                             ("omelyan_f16_inner_clover_2scales", om, 6, hr.HR_F16, None, 3),
                                             ("omelyan_f16_inner_clover_hasenbusch_2scales", om, 6, hr.HR_F16, 0.2,
                                              3)):
        solver = hr.hr_solver_default_opts()
        solver.inner_prec = inner
        solver.reliable_delta = 0.01 if inner != hr.HR_F64 else 0.1
        chain = HMC(ctx, lat, beta=beta, m0=m0, fermions=True, n_steps=steps, tau=1.0, integrator=integ,
                    solver=solver, seed=2006, m0_hasenbusch=mh, n_steps_gauge=m,
                    c_sw=1.0 if "clover" in name else None)
        q = qd0.clone()
        secs, dhs, iters = [], [], []
        for _ in range(4):
            torch.cuda.synchronize()
            acc, info = chain.step(q)
            secs.append(info.seconds)
            dhs.append(info.dH)
            iters.append(info.cg_iters)
        forces = steps + 1 if integ == hr.HR_INTEGRATOR_LEAPFROG else 2 * steps + 1
        out[name] = {"n_steps": steps, "force_evaluations": forces, "hasenbusch_m0": mh, "n_steps_gauge": m,
                     "c_sw": 1.0 if "clover" in name else None,
                     "trajectory_s_median": round(statistics.median(secs[1:]), 4),
                     "dH": [round(float(x), 4) for x in dhs], "accepted": f"{chain.accepted}/{chain.trajectories}",
                     "cg_iters_per_trajectory": int(statistics.median(iters)), "end_plaquette": round(info.plaquette, 4)}
        del chain, q
    return out



def run_cg_clover(ctx, hr, fields, d32, q32, gauge, bp, xp, cg_wilson):
    """The 32^4 solves of cg_32 with the clover term (c_sw = 1, m0 = -0.2):
    FP64 and mixed precision (each at the reliable_delta that won for the
    Wilson operator), median of five solves after one warm-up."""
    m0, csw = -0.2, 1.0
    t0 = time.perf_counter()
    clov = fields.build_clover(ctx, d32, hr.HR_FUND, hr.HR_F64, hr.HR_CLOVER_SW, m0, csw,
                               fields.gauge_to_device(q32))
    out = {"c_sw": csw, "m0": m0, "kind": "clover (Sheikholeslami-Wohlert)",
           "build_s": round(time.perf_counter() - t0, 3)}
    for name, inner in (("fp64", hr.HR_F64), ("mixed_f32", hr.HR_F32), ("mixed_f16", hr.HR_F16)):
        opts = hr.hr_solver_default_opts()
        opts.inner_prec = inner
        opts.reliable_delta = cg_wilson.get(name, {}).get("reliable_delta", 0.1)
        work = fields.empty_bytes(hr.hr_cg_clover_workspace_bytes(d32, hr.HR_FUND, opts))
        times = []
        rc = info = None
        for _ in range(6):
            rc, info = hr.hr_cg_solve_clover(ctx, d32, hr.HR_FUND, opts, gauge, clov, bp, xp, work)
            times.append(info.seconds)
        out[name] = {"status": hr.STATUS_NAMES.get(rc, rc), "seconds_median": round(statistics.median(times[1:]), 4),
                     "iters": info.iters, "reliable_updates": info.n_reliable_updates,
                     "true_rel_residual": info.true_rel_residual, "reliable_delta": opts.reliable_delta}
        del work
    if out["fp64"]["seconds_median"] > 0:
        for k in ("mixed_f32", "mixed_f16"):
            out[k]["speedup_vs_fp64"] = round(out["fp64"]["seconds_median"] / out[k]["seconds_median"], 3)
    return out


def run_clover_48(ctx, torch, hr, fields, q48, psi48, reps=30):
    """48^4 fund FP64: one Schur operator application Mhat (two hops) with and
    without the clover site term (clover and exponential clover), the cost of
    the diagonal term the paper measures (Sec. 2.2, Fig. 3), and the one-off
    build of the field.  Bytes per even site: Wilson 1152 (two hops of 512 +
    the aux spinor 128); with the term + 2 x 256 (A_oo^-1 and A_ee blocks)."""
    dims = DIMS
    m0, csw = -0.2, 1.0
    qd = fields.gauge_to_device(q48)
    gauge = fields.pack_gauge(ctx, dims, hr.HR_FUND, hr.HR_F64, qd)
    src = fields.pack_spinor(ctx, dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, fields.spinor_to_device(psi48))
    dst = fields.empty_spinor(dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN)
    work = fields.empty_bytes(hr.hr_dirac_workspace_bytes(dims, hr.HR_FUND, hr.HR_F64, hr.HR_OP_SCHUR))
    Vh = int(np.prod(dims)) // 2
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(5):
            fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {"lattice": list(dims), "m0": m0, "c_sw": csw, "applications": reps}
    ms_w = timed(lambda: hr.hr_dirac_eo(ctx, dims, m0, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, hr.HR_OP_SCHUR, 1,
                                        gauge, src, dst, work))
    out["wilson"] = {"ms": round(ms_w, 4), "gbs": round(Vh * 1152 / (ms_w * 1e-3) / 1e9, 1)}
    for name, kind in (("clover", hr.HR_CLOVER_SW), ("exp_clover", hr.HR_CLOVER_EXP)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        clov = fields.build_clover(ctx, dims, hr.HR_FUND, hr.HR_F64, kind, m0, csw, qd)
        torch.cuda.synchronize()
        build_s = time.perf_counter() - t0
        ms = timed(lambda: hr.hr_dirac_eo_clover(ctx, dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, hr.HR_OP_SCHUR, 1,
                                                 gauge, clov, src, dst, work))
        out[name] = {"ms": round(ms, 4), "gbs": round(Vh * (1152 + 512) / (ms * 1e-3) / 1e9, 1),
                     "time_vs_wilson": round(ms / ms_w, 3), "build_s": round(build_s, 3)}
        del clov
    del gauge, src, dst, work, qd
    return out


def run_twist_48(ctx, torch, hr, fields, q48, psi48, reps=30):
    """48^4 fund FP64 hop with twisted boundaries (theta in time only, and in
    all four directions): the twisted kernel (paired double-float, one launch
    shape, the phase on the projected doublets of boundary-crossing hops),
    against the tuned untwisted hop on the same fields (512 B per site)."""
    dims = DIMS
    Vh = int(np.prod(dims)) // 2
    qd = fields.gauge_to_device(q48)
    pd = fields.spinor_to_device(psi48)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"lattice": list(dims), "applications": reps}
    for name, lat in (("untwisted", hr.Lattice(dims, 1)), ("twist_t", hr.Lattice(dims, 1, (0.5, 0, 0, 0))),
                      ("twist_all", hr.Lattice(dims, 1, (0.5, 0.3, -0.7, 1.1)))):
        gauge = fields.pack_gauge(ctx, lat, hr.HR_FUND, hr.HR_F64, qd)
        src = fields.pack_spinor(ctx, lat, hr.HR_FUND, hr.HR_F64, hr.HR_ODD, pd)
        dst = fields.empty_spinor(lat, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN)

        def hop():
            hr.hr_dirac_eo(ctx, lat, 0.0, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, hr.HR_OP_HOP, 1, gauge, src, dst)

        for _ in range(5):
            hop()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            hop()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"ms": round(ms, 4), "gbs": round(Vh * 512 / (ms * 1e-3) / 1e9, 1)}
        del gauge, src, dst
    for k in ("twist_t", "twist_all"):
        out[k]["time_vs_untwisted"] = round(out[k]["ms"] / out["untwisted"]["ms"], 3)
    del qd, pd
    return out


def run_dd_48(ctx, torch, hr, fields, q48, psi48, reps=20):
    """48^4 fund FP64 split along time into 4 slabs of 12 x 48^3 on this one
    GPU (the multi-GPU data flow, the exchange a device copy on a second
    stream): one D_eo + D_oe application (per parity: face pack, exchange,
    the 4 local hops, the boundary kernels) against the tuned whole-lattice
    hop pair, 512 B per site.  The slabs run one after another on the one
    GPU, so this is the decomposition's overhead, not a scaling figure."""
    from paper_2411_18511_gb300 import dd
    dims, n = DIMS, 4
    Vh = int(np.prod(dims)) // 2
    slabs = dd.TimeSlabs(dims, n)
    op = dd.SlabHop(ctx, slabs, hr.HR_FUND, hr.HR_F64, q48)
    src = {p: op.pack_input(psi48, 1 - p) for p in (hr.HR_EVEN, hr.HR_ODD)}
    out = {p: [fields.empty_spinor(slabs.local(r), hr.HR_FUND, hr.HR_F64, p) for r in range(n)]
           for p in (hr.HR_EVEN, hr.HR_ODD)}
    # the local hops with the shape the tuner picks for a slab
    loc = slabs.local(0)
    g0, s0, d0 = op.gauge[0], src[hr.HR_EVEN][0], out[hr.HR_EVEN][0]
    res = hr.hr_autotune_hop(ctx, loc, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, 1, g0, s0, d0, reps=10)

    def step():
        op.apply(hr.HR_EVEN, src[hr.HR_EVEN], out[hr.HR_EVEN])
        op.apply(hr.HR_ODD, src[hr.HR_ODD], out[hr.HR_ODD])

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    face_mb = hr.hr_dd_face_bytes(loc, hr.HR_FUND, hr.HR_F64) / 1e6
    return {"lattice": list(dims), "slabs": n, "slab": list(loc), "ms_per_hop_pair": round(ms, 4),
            "gbs": round(2 * Vh * 512 / (ms * 1e-3) / 1e9, 1), "face_mb_each": round(face_mb, 2),
            "faces_per_slab_per_hop": 2, "local_hop_launch": {"variant": res.variant, "block": res.block},
            "note": "all slabs on one GPU, run in turn; multi-GPU runs untested here (one GPU per call)"}


def run_diff_solve(torch, synth):
    """16^4 fund FP64: S = Re<eta, (Mhat^+ Mhat)^-1 eta> through the autograd
    solve; forward (one solve) and backward (one adjoint solve and the link
    gradient) wall times."""
    from paper_2411_18511_gb300 import autograd as ag
    d = (16, 16, 16, 16)
    m0 = -0.2
    q, nsm, plaq = synth.ape_smear_to_plaquette(synth.haar_links(d, 1005), d, 0.6)
    eta = synth.gaussian_spinor(d, 2, 2005)
    eta[(np.indices(d).sum(axis=0).reshape(-1) & 1) == 1] = 0  # even source
    qt = torch.tensor(q, device="cuda")
    et = torch.tensor(eta, device="cuda")
    fwd, bwd = [], []
    for _ in range(4):
        qg = qt.clone().requires_grad_(True)
        eg = et.clone().requires_grad_(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x = ag.EoSolve.apply(qg, eg, d, m0, 1e-10)
        S = torch.sum(eg.conj() * x).real
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        S.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        fwd.append(t1 - t0)
        bwd.append(t2 - t1)
    return {"lattice": list(d), "m0": m0, "tol": 1e-10, "plaquette": round(plaq, 4),
            "forward_s": round(statistics.median(fwd[1:]), 4), "backward_s": round(statistics.median(bwd[1:]), 4),
            "backward_over_forward": round(statistics.median(bwd[1:]) / statistics.median(fwd[1:]), 2),
            "note": "wall times incl. packing; backward = adjoint solve + link gradient kernels"}


def run_batch(ctx, torch, hr, fields, synth):
    """12 lattices of 8^4..24^4 (Haar links, own seeds): one batched persistent
    FP64 CG against the 12 single-lattice solves one after the other."""
    sizes = [8, 8, 10, 12, 12, 14, 16, 16, 18, 20, 22, 24]
    dims = [(L,) * 4 for L in sizes]
    m0 = -0.2
    gauges, bs = [], []
    for k, d in enumerate(dims):
        q = synth.haar_links(d, 1100 + k)
        b = synth.gaussian_spinor(d, 2, 2100 + k)
        gauges.append(fields.pack_gauge(ctx, d, hr.HR_FUND, hr.HR_F64, fields.gauge_to_device(q)))
        bs.append(fields.pack_spinor(ctx, d, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, fields.spinor_to_device(b)))
    opts = hr.hr_solver_default_opts()
    work = fields.empty_bytes(hr.hr_cg_batch_workspace_bytes(dims, hr.HR_FUND))
    tb, infos = [], None
    for _ in range(3):
        xs = [fields.zeros_spinor(d, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN) for d in dims]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, infos = hr.hr_cg_solve_batch(ctx, dims, m0, hr.HR_FUND, opts, gauges, bs, xs, work)
        torch.cuda.synchronize()
        tb.append(time.perf_counter() - t0)
    ts = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k, d in enumerate(dims):
            x = fields.zeros_spinor(d, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN)
            w = fields.empty_bytes(hr.hr_cg_workspace_bytes(d, hr.HR_FUND, opts))
            hr.hr_cg_solve(ctx, d, m0, hr.HR_FUND, opts, gauges[k], bs[k], x, w)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    return {"lattices": sizes, "m0": m0, "tol": opts.tol, "status": hr.STATUS_NAMES.get(rc, rc),
            "batch_wall_s": round(statistics.median(tb), 4), "sequential_wall_s": round(statistics.median(ts), 4),
            "speedup": round(statistics.median(ts) / statistics.median(tb), 3),
            "iters": [i.iters for i in infos], "max_true_rel_residual": max(i.true_rel_residual for i in infos)}


def run_multi_rhs(ctx, torch, hr, fields, synth):
    """24^4 fundamental: N_rhs Gaussian sources sharing one smeared gauge field,
    FP32-inner / FP64-outer CG to 1e-10, and the FP32 multi-RHS hop's GB/s."""
    d = (24, 24, 24, 24)
    Vh = int(np.prod(d)) // 2
    q, nsm, plaq = synth.ape_smear_to_plaquette(synth.haar_links(d, 1004), d, 0.6)
    gauge = fields.pack_gauge(ctx, d, hr.HR_FUND, hr.HR_F64, fields.gauge_to_device(q))
    g32 = fields.pack_gauge(ctx, d, hr.HR_FUND, hr.HR_F32, fields.gauge_to_device(q))
    res = {"lattice": list(d), "m0": -0.2, "tol": 1e-10, "plaquette": round(plaq, 4), "inner": "f32",
           "reliable_delta": 1e-5}
    sols = {"dims": d, "q": q, "n": {}}
    t1 = None
    for n in (1, 4, 8, 16, 32):
        bs = synth.gaussian_spinor(d, 2, 2004, n_rhs=n)
        dev = fields.spinor_to_device(bs if n > 1 else bs[0])
        bp = fields.pack_spinor(ctx, d, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, dev)
        opts = hr.hr_solver_default_opts()
        opts.inner_prec = hr.HR_F32
        opts.reliable_delta = 1e-5  # the FP32-inner setting that wins at 32^4 (cg_32): fewer FP64 updates
        opts.n_rhs = n
        # the solver's hop shapes (FP32 inner, FP64 reliable updates) tuned for this N
        tuned = {}
        for tp, gp in ((hr.HR_F32, g32), (hr.HR_F64, gauge)):
            ts = fields.pack_spinor(ctx, d, hr.HR_FUND, tp, hr.HR_ODD, dev)
            td = fields.empty_spinor(d, hr.HR_FUND, tp, hr.HR_EVEN, n)
            tr = hr.hr_autotune_hop(ctx, d, hr.HR_FUND, tp, hr.HR_EVEN, n, gp, ts, td, reps=10)
            tuned[{hr.HR_F32: "f32", hr.HR_F64: "f64"}[tp]] = [tr.variant, tr.block]
            del ts, td
        work = fields.empty_bytes(hr.hr_cg_workspace_bytes(d, hr.HR_FUND, opts))
        times = []
        info = rc = None
        for _ in range(6):  # one warm-up solve (it also captures the solve graph), five timed
            xp = fields.zeros_spinor(d, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, n)
            rc, info = hr.hr_cg_solve(ctx, d, -0.2, hr.HR_FUND, opts, gauge, bp, xp, work)
            times.append(info.seconds)
        t = statistics.median(times[1:])
        if n == 1:
            t1 = t
        if n in (1, 32):  # the solutions the oracle checks (cpu_baseline)
            xs = fields.unpack_spinor(ctx, d, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, xp, n).cpu().numpy()
            sols["n"][n] = (bs if n > 1 else bs[0][None], xs if n > 1 else xs[None])
        # multi-RHS FP32 hop: each link load serves n spinors
        src = fields.pack_spinor(ctx, d, hr.HR_FUND, hr.HR_F32, hr.HR_ODD, dev)
        dst = fields.empty_spinor(d, hr.HR_FUND, hr.HR_F32, hr.HR_EVEN, n)
        for _ in range(3):
            hr.hr_dirac_eo(ctx, d, 0.0, hr.HR_FUND, hr.HR_F32, hr.HR_EVEN, hr.HR_OP_HOP, n, g32, src, dst)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(50):
            hr.hr_dirac_eo(ctx, d, 0.0, hr.HR_FUND, hr.HR_F32, hr.HR_EVEN, hr.HR_OP_HOP, n, g32, src, dst)
        e1.record()
        torch.cuda.synchronize()
        hop_ms = e0.elapsed_time(e1) / 50
        hop_bytes = Vh * (n * 2 * 64 + 8 * 16)  # n spinors in and out, links once
        res[f"n{n}"] = {"status": hr.STATUS_NAMES.get(rc, rc), "solve_s": round(t, 5),
                        "first_solve_s": round(times[0], 5),
                        "per_rhs_s": round(t / n, 5), "per_rhs_speedup_vs_n1": round(t1 / (t / n), 3),
                        "iters": info.iters, "reliable_updates": info.n_reliable_updates,
                        "true_rel_residual": info.true_rel_residual,
                        "hop_ms": round(hop_ms, 5), "hop_gbs": round(hop_bytes / (hop_ms * 1e-3) / 1e9, 1),
                        "tuned_hop_shapes": tuned}
        del work, bp, src, dst, dev
        torch.cuda.empty_cache()
    return res, sols


def cpu_baseline(q, psi, dims, sols=None):
    """The FP64 oracle as it stands on the host cores: one hop pair over the
    whole lattice (every site once), OpenMP over sites; and, given the GPU
    solutions of the extras (sols), the oracle's CG at 32^4 timed beside them
    (the CPU baseline of the metric's CG half) with every GPU solution's true
    residual recomputed by the oracle and its distance to the oracle's
    solution, the same for the 24^4 multi-RHS solves (residual of every
    right-hand side at N = 1 and 32, distance for the first and last)."""
    import oracle
    try:
        L = oracle.expand_links(dims, 2, q)
        V = int(np.prod(dims))
        t0 = time.perf_counter()
        out = oracle.hop(dims, L, psi, parity=-1)
        dt = time.perf_counter() - t0
        gbs = (V // 2) * 2 * hop_bytes_per_site("fund", "f64") / dt / 1e9
        # the same oracle on one core, over a sample of 1/16 of the sites
        rng = np.random.default_rng(7)
        sites = np.sort(rng.choice(V, V // 16, replace=False)).astype(np.int64)
        prev = oracle.set_num_threads(1)
        try:
            t0 = time.perf_counter()
            oracle.hop_sites(dims, L, psi, sites)
            dt1 = time.perf_counter() - t0
        finally:
            oracle.set_num_threads(prev)
        gbs1 = len(sites) * hop_bytes_per_site("fund", "f64") / dt1 / 1e9
        del out, L
        res = {"value": round(gbs, 3), "unit": "GB/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"one D_eo+D_oe application over all {V} sites of {dims[0]}^4 ({dt:.2f} s)",
               "single_core": {"value": round(gbs1, 3), "unit": "GB/s", "cores": 1,
                               "sample": f"{len(sites)} random sites, one hop each ({dt1:.2f} s)"},
               "cpu": _cpu_model()}
    except Exception as exc:  # the baseline is informative only
        return {"value": None, "unit": "GB/s", "cores": None, "kind": "oracle", "sample": f"failed: {exc}"}
    if sols:
        try:
            res["solver_checks"] = oracle_solver_checks(oracle, sols)
        except Exception as exc:
            res["solver_checks"] = {"failed": str(exc)}
    return res


def oracle_solver_checks(oracle, sols, m0=-0.2):
    """The oracle's view of the GPU's CG solutions (see cpu_baseline)."""
    out = {}
    c = sols.get("cg_32")
    if c:
        d = c["dims"]
        even = (np.indices(d).sum(axis=0).reshape(-1) & 1) == 0
        b = c["b"].copy()
        b[~even] = 0
        L = oracle.expand_links(d, 2, c["q"])
        t0 = time.perf_counter()
        xo, it, tr, ok = oracle.cg(d, L, m0, b, tol=1e-10)
        cg_s = time.perf_counter() - t0
        rec = {"oracle_cg": {"seconds": round(cg_s, 2), "iters": it, "true_rel_residual": tr, "converged": ok,
                             "cores": oracle.num_threads()}}
        nb, nxo = np.linalg.norm(b), np.linalg.norm(xo[even])
        for name, x in c["x"].items():
            r = np.linalg.norm(b - oracle.normal(d, L, m0, x)) / nb
            rec[name] = {"oracle_true_rel_residual": float(r),
                         "rel_error_vs_oracle_x": float(np.linalg.norm((x - xo)[even]) / nxo)}
        out["cg_32"] = rec
        del L
    m = sols.get("multi_rhs_24")
    if m:
        d = m["dims"]
        even = (np.indices(d).sum(axis=0).reshape(-1) & 1) == 0
        L = oracle.expand_links(d, 2, m["q"])
        rec = {}
        for n, (bs, xs) in m["n"].items():
            worst = 0.0
            errs = []
            for r in range(n):
                b = bs[r].copy()
                b[~even] = 0
                worst = max(worst, float(np.linalg.norm(b - oracle.normal(d, L, m0, xs[r])) / np.linalg.norm(b)))
                if r in (0, n - 1) and (r == 0 or n > 1):
                    xo, it, tr, ok = oracle.cg(d, L, m0, b, tol=1e-10)
                    errs.append(float(np.linalg.norm((xs[r] - xo)[even]) / np.linalg.norm(xo[even])))
            rec[f"n{n}"] = {"max_oracle_true_rel_residual": worst, "rel_error_vs_oracle_x": errs,
                            "rhs_checked": n, "x_compared_for_rhs": sorted({0, n - 1})}
        out["multi_rhs_24"] = rec
    return out


def attach_oracle_checks(extras, cpu):
    """Each CG result of the extras states its error against the FP64 oracle."""
    chk = (cpu or {}).get("solver_checks") or {}
    for key in ("cg_32", "multi_rhs_24"):
        if key not in extras or key not in chk:
            continue
        for name, v in chk[key].items():
            if name in extras[key] and isinstance(extras[key][name], dict):
                extras[key][name]["vs_oracle"] = v
            else:
                extras[key][name] = v


def _cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return os.uname().machine


# ----------------------------------------------------------------------------- reference

def run_reference(args):
    """The FP64 CPU oracle on the same workload and metric, on the host cores."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    import oracle
    import synth
    q = synth.haar_links(DIMS, GAUGE_SEED)
    psi = synth.gaussian_spinor(DIMS, 2, SPINOR_SEED)
    L = oracle.expand_links(DIMS, 2, q)
    V = int(np.prod(DIMS))
    rng = np.random.default_rng(0)
    # size each step's sample so that warmup + steps take about two minutes
    probe = rng.choice(V, 20000, replace=False)
    t0 = time.perf_counter()
    oracle.hop_sites(DIMS, L, psi, probe)
    per_site = (time.perf_counter() - t0) / probe.size
    n_sites = int(min(V, max(2000, 120.0 / max(1, args.steps + args.warmup) / per_site)))
    sites = [rng.choice(V, n_sites, replace=False) for _ in range(4)]
    for w in range(args.warmup):
        oracle.hop_sites(DIMS, L, psi, sites[w % 4])
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle.hop_sites(DIMS, L, psi, sites[k % 4])
    dt = time.perf_counter() - t0
    bps = hop_bytes_per_site("fund", "f64")
    value = n_sites * args.steps * bps / dt / 1e9
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GB/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "even-odd Wilson-Dirac hop pair D_eo+D_oe, 48^4 SU(2) fundamental, FP64",
                   "lattice": list(DIMS)},
        "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": f"{n_sites} random sites of 48^4 per step (hop at each site)"},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
