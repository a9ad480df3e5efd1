#!/usr/bin/env python3
"""Throughput of one quasi-cylindrical arbitrary-order PSATD PIC cycle on GB300.

Workload (default): the 2048 x 256 grid, 2 azimuthal modes, stencil order 32, FP64,
1e17 cm^-3 plasma at 2 macroparticles per cell plus a 200k-particle drive beam and a
100k-particle witness beam (1,348,576 particles): the plain FP64 beam-driven wakefield
configuration.  A step is one full cycle: gather + push + current deposit, cell sort,
charge deposit, z-FFT + DHT, PSATD update, inverse DHT + z-FFT.

Prints ONE JSON line (rank 0).  Under torchrun each rank runs its own independent
simulation (weak scaling; no collective on the data path), and the time is the max
over ranks.  ``--impl reference`` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12   # 152 SMs x 2 DFMA/clk x 2070 MHz (nominal 1.25)


def fp64_particle_flops(Nm):
    """Algorithmic float64 operations of one particle's pass in the FP64 form (gather, push,
    J at x^{n+1/2}, rho at x^{n+1}), each multiply, add, divide and square root counted once:
      polar decomposition 7 (x^2, y^2, add, sqrt, 2 divides) and stencil 7 at each of the
      three positions; 4 node weights (gather) and 8 node weights / V_j (each deposit);
      phases e^{-+i m theta}: 6 per mode m >= 2 in the gather and each deposit;
      interpolation + mode sum of 6 components: 8 (mode 0, real part) + 21 per mode m >= 1
      (4 complex node terms 16, real part of the phase product 3, x 2 and accumulate 2);
      (r, theta) -> (x, y) of E and B 12; Boris 58; 1/gamma and v 11; two half moves 12;
      J: q w and its phases 1 + 2 (Nm - 1), q w e^{i m theta} v_k 3 (2 Nm - 1), node products
      and adds 24 (2 Nm - 1); rho: 1 + 2 (Nm - 1) and 8 (2 Nm - 1)."""
    ph = 6 * max(Nm - 2, 0)
    gather = 7 + 7 + 4 + ph + 6 * (8 + 21 * (Nm - 1)) + 12
    push = 58 + 11 + 12
    dep_j = 7 + 7 + 8 + ph + 1 + 2 * (Nm - 1) + 3 * (2 * Nm - 1) + 24 * (2 * Nm - 1)
    dep_rho = 7 + 7 + 8 + ph + 1 + 2 * (Nm - 1) + 8 * (2 * Nm - 1)
    return gather + push + dep_j + dep_rho
FP64_PROBE_TFLOPS = 1.1947                     # FMA-loop probe on this machine's GB300 at 1987 MHz
# DRAM bytes per FP64 DHT launch (k_gemm<double>) on this workload, from one ncu capture of
# the current kernel (forward 71.42 + 27.50 MB, inverse 106.87 + 60.50 MB, mean of the two)
DHT_F64_TRAFFIC_BYTES = (71.424 + 27.501568 + 106.872064 + 60.499968) / 2 * 1e6
# DRAM bytes of one k_gather_push_f32<2, false, true> launch at cfg2 (dram__bytes_read.sum +
# dram__bytes_write.sum, profiles/k_gather_push_f32__wake_2048x256_m2_mixed.md)
PUSH_F32_TRAFFIC_BYTES = (148.361984 + 45.164544) * 1e6
TF32_PER_BF16 = 1.1 / 2.25                     # nominal dense TF32 / BF16 tensor rates


def peaks():
    """Roofline denominators: the driver's measurements on this machine (MEASURED_PEAKS.json:
    STREAM-style copy bandwidth, cuBLAS BF16 burst and sustained), else the fallback figures
    of one earlier GB300 measurement.  Kernels timed inside the cycle loop take the
    sustained tensor figure."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_burst": float(d["bf16_tflops"]),
                "bf16_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), "source": "of measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_burst": 1900.0, "bf16_sustained": 1700.0, "source": "of fallback"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--order", type=int, default=32)
    ap.add_argument("--precision", choices=["fp64", "mixed", "bf16"], default="fp64",
                    help="fp64: every stage in float64; mixed: float grids and particles, "
                         "3-term TF32 DHT on tcgen05; bf16: the same with the 6-product BF16 DHT")
    ap.add_argument("--e2e-steps", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-form comparison")
    ap.add_argument("--accuracy-cycles", type=int, default=2000,
                    help="cycles after which the mixed form's fields and beam quality are "
                         "compared with the FP64 form (0: skip)")
    ap.add_argument("--sort-interval", type=int, default=4,
                    help="sort particles by cell on every k-th cycle (pic_set_sort_interval), all forms: "
                         "the order only serves memory locality; results change by rounding only")
    ap.add_argument("--workload", choices=["wake", "scan", "large", "crop", "guard", "order_sweep", "window",
                                           "fft_lengths"],
                    default="wake",
                    help="wake: the 2048x256 wakefield run; scan: many uneven simulations "
                         "(order / resolution scan) advanced by one CUDA graph per launch; "
                         "large: the 8192x1024 3-mode run with ~103M particles, mixed form; "
                         "crop: its 1024x128 crop (1.6M particles), a small case of the same kernels")
    ap.add_argument("--sims", type=int, default=64, help="simulations in the scan workload")
    ap.add_argument("--no-extra", action="store_true",
                    help="wake workload: skip the large run and the scan that the 1-GPU line also reports")
    ap.add_argument("--large-accuracy-cycles", type=int, default=20,
                    help="cycles after which the large run's mixed forms are compared with its FP64 form (0: skip)")
    ap.add_argument("--sweep-steps", type=int, default=2000, help="cycles per order in the order sweep")
    ap.add_argument("--window-cycles", type=int, default=8192,
                    help="cycles of the moving-window propagation after the timed cycles")
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket each timed region with cudaProfilerStart/Stop (for "
                         "ncu --profile-from-start off); no work is skipped")
    return ap.parse_args()


E2E_MAX_SLICES = 256   # slice values read back per end-to-end cycle (the witness has ~25)


def workload(order, rank=0):
    from paper_1611_05712_gb300 import workloads as W
    return W.wake_2048x256(order_p=order, seed=2 + rank)


def config_of(w, n, precision="fp64", sort_interval=None):
    c = {"workload": w.name, "Nz": w.Nz, "Nr": w.Nr, "Nm": w.Nm, "order_p": w.order_p,
         "particles": n, "dz_m": w.dz, "dt_s": w.dt, "precision": precision,
         "l2": "no flush: working set (fields + particles, ~0.8 GB) exceeds the 129 MB L2"}
    if sort_interval is not None:
        c["sort_interval"] = sort_interval
    return c


# ------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------- multi-rank
def reduce_max(x, dist=None, device=None):
    """Max of a per-rank time over all ranks (a timing reduction, not a data-path exchange)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_throughput(steps, world, max_ms):
    """Whole-job cycles/s: every rank advances its own simulation `steps` cycles."""
    return world * steps / (max_ms * 1e-3)


# ------------------------------------------------------------------------- CPU oracle
def oracle_steps_per_s(w, P, npl, beams, n_steps):
    """Time the FP64 oracle as it stands on the host cores: n_steps full cycles."""
    from oracle import psatd_rz as O
    g = O.Grid(w.Nz, w.Nr, w.Nm, w.dz, w.dr, w.dt)
    st = O.make_state(g, w.order_p, True, P, npl, beams)
    t0 = time.perf_counter()
    O.pic_step(st, n_steps)
    dt = time.perf_counter() - t0
    return n_steps / dt, dt


def oracle_crop_baseline(args):
    """The oracle beside the large run: one cycle of its 1024 x 128 x 3 crop (a full cycle
    of the 8192 x 1024 x 3 grid with 102.7M particles does not fit a bounded host sample)."""
    from paper_1611_05712_gb300 import workloads as W
    wc = W.large_crop_1024x128(order_p=args.order)
    Pc, nplc, beamsc = W.particles(wc)
    v, secs = oracle_steps_per_s(wc, Pc, nplc, beamsc, 1)
    return {"value": v, "unit": "steps/s", "cores": os.cpu_count(), "kind": "oracle",
            "particle_updates_per_s": v * len(Pc["x"]),
            "sample": f"1 full cycle of the 1024x128x3 crop of this workload ({len(Pc['x'])} particles, "
                      f"{secs:.1f} s; numpy FP64 oracle): cycles/s of the crop, not scaled to the full grid"}


def oracle_scan_baseline(n_sample=4):
    """The oracle beside the scan: one cycle of each of n_sample members taken evenly through
    the 64 members ordered by cell count; value = the sample's member-cycles per second."""
    from paper_1611_05712_gb300 import workloads as W
    members = [W.scan_member(s) for s in range(64)]
    order = sorted(range(64), key=lambda i: members[i].Nz * members[i].Nr)
    step = len(order) // n_sample
    pick = [order[step // 2 + k * step] for k in range(n_sample)]
    total = 0.0
    names = []
    for i in pick:
        m = members[i]
        Pm, nplm, beamsm = W.particles(m)
        _, secs = oracle_steps_per_s(m, Pm, nplm, beamsm, 1)
        total += secs
        names.append(f"{m.Nz}x{m.Nr}x{m.Nm}")
    return {"value": n_sample / total, "unit": "sim-steps/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"1 cycle each of {n_sample} members spread evenly over the cell-count order "
                      f"({', '.join(names)}; {total:.1f} s; numpy FP64 oracle)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_1611_05712_gb300 import workloads as W
    w = workload(args.order)
    P, npl, beams = W.particles(w)
    from oracle import psatd_rz as O
    g = O.Grid(w.Nz, w.Nr, w.Nm, w.dz, w.dr, w.dt)
    st = O.make_state(g, w.order_p, True, P, npl, beams)
    O.pic_step(st, args.warmup)
    t0 = time.perf_counter()
    O.pic_step(st, args.steps)
    el = time.perf_counter() - t0
    v = args.steps / el
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": "pic_steps_per_s", "value": v, "unit": "steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_of(w, len(P["x"])),
        "particle_updates_per_s": v * len(P["x"]),
        "cpu_baseline": {"value": v, "unit": "steps/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} full cycles of the workload (numpy FP64 oracle)"},
        "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------- GPU

def measure(args, w, P, npl, beams, prec, dist, dev, world, local):
    """Set one simulation up (untimed), warm up, time args.steps cycles with CUDA events
    between the stages, then time args.e2e_steps cycles end to end through the C ABI."""

    import numpy as np
    import torch

    from paper_1611_05712_gb300 import binding as bd
    n = len(P["x"])
    mixed = prec != bd.PIC_FP64
    sim = bd.Sim.from_workload(w, P, npl, beams, device=f"cuda:{local}", precision=prec)
    wit_lo, wit_hi = beams[-1][0], beams[-1][1]
    # the sort interval first: the chunk tuning times that many cycles' particle passes
    sim.set_sort_interval(args.sort_interval)
    tuning = sim.autotune() if mixed else {}   # untimed: tile sizes for this workload
    tuning["sort_interval"] = args.sort_interval
    sim.step(args.warmup)
    sim.sync()
    torch.cuda.synchronize(dev)

    # timed region: K cycles, CUDA events between stages on the library's stream
    l0 = sim.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        if args.profile_range:
            torch.cuda.profiler.start()
        stage_ms, total_ms = sim.step_timed(args.steps)
        if args.profile_range:
            torch.cuda.synchronize(dev)
            torch.cuda.profiler.stop()
    torch.cuda.synchronize(dev)
    launches = sim.launch_count() - l0
    el_ms = reduce_max(total_ms, dist, dev)
    steps_per_s = weak_throughput(args.steps, world, el_ms)

    # end to end through the C ABI with host buffers: every cycle takes a particle set
    # copied from pinned host memory, steps once and reads the witness-beam diagnostics
    # back; the copy of the next cycle's set is staged on the library's copy stream while
    # the current cycle computes (pic_stage_particles / pic_take_particles)
    pinned = {k: torch.from_numpy(np.ascontiguousarray(P[k])).pin_memory() for k in bd.SOA}
    pinned["id"] = torch.from_numpy(np.ascontiguousarray(P["id"], dtype=np.int32)).pin_memory()
    n_slices = 0
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    sim.stage_particles(pinned)
    for k in range(args.e2e_steps):
        sim.take_particles()
        if k + 1 < args.e2e_steps:
            sim.stage_particles(pinned)
        sim.step(1)
        d = sim.diagnostics(wit_lo, wit_hi, max_slices=E2E_MAX_SLICES)
        n_slices = d["n_slices"]
    e2e_s = time.perf_counter() - t0
    e2e_s = reduce_max(e2e_s, dist, dev)
    e2e = {"value": weak_throughput(args.e2e_steps, world, 1e3 * max(e2e_s, 1e-12)), "unit": "steps/s",
           # the staged copy of the particle set; the diagnostics' header and slice values
           "h2d_bytes_per_step": n * (7 * 8 + 4),
           "d2h_bytes_per_step": 8 * (64 + E2E_MAX_SLICES),
           "steps": args.e2e_steps, "witness_slices_read": n_slices}

    # roofline of the dominant kernel: the DHT (two launches per cycle)
    dht_flops_per_step = 10 * w.Nm * 4.0 * w.Nz * w.Nr ** 2
    dht_ms = stage_ms["dht_fwd"] + stage_ms["dht_inv"]
    launches_dht = 2 * args.steps
    achieved = (dht_flops_per_step * args.steps / launches_dht) / (dht_ms * 1e-3 / launches_dht) / 1e12
    share = dht_ms / sum(stage_ms.values())
    pk = peaks()
    if prec == bd.PIC_MIXED_TF32X3:
        # 3 TF32 products per algorithmic multiply-add; the TF32 peak is the measured BF16
        # figure x the recipe's nominal TF32/BF16 ratio (sustained: timed inside the cycle loop)
        tf32_peak = pk["bf16_sustained"] * TF32_PER_BF16
        roofline = {"bound": "tensor", "achieved": achieved, "peak": tf32_peak, "unit": "TFLOP/s",
                    "frac": achieved / tf32_peak, "traffic": None,
                    "executed_tflops": 3 * achieved, "executed_frac": 3 * achieved / tf32_peak,
                    "frac_of_burst": achieved / (pk["bf16_burst"] * TF32_PER_BF16),
                    "kernel": "k_dht_tc<TF32x3> (3-term TF32 on tcgen05)",
                    "peak_source": f"{pk['source']}: bf16 sustained {pk['bf16_sustained']} TFLOP/s x nominal "
                                   "tf32/bf16 1.1/2.25",
                    "share_of_step": share}
    elif prec == bd.PIC_MIXED_BF16X6:
        # 6 BF16 products per algorithmic multiply-add against the measured BF16 peak
        roofline = {"bound": "tensor", "achieved": achieved, "peak": pk["bf16_sustained"], "unit": "TFLOP/s",
                    "frac": achieved / pk["bf16_sustained"], "traffic": None,
                    "executed_tflops": 6 * achieved, "executed_frac": 6 * achieved / pk["bf16_sustained"],
                    "frac_of_burst": achieved / pk["bf16_burst"],
                    "kernel": "k_dht_tc<BF16x6> (6 BF16 split products on tcgen05)",
                    "peak_source": f"{pk['source']}: bf16 sustained {pk['bf16_sustained']} TFLOP/s",
                    "share_of_step": share}
    elif w.Nr <= 256:
        # FP64 form, sliced path: 28 BF16 slice products per algorithmic multiply-add on the
        # tensor cores (executed against the measured BF16 peak), FP64-equivalent rate beside
        roofline = {"bound": "tensor", "achieved": 28 * achieved, "peak": pk["bf16_sustained"], "unit": "TFLOP/s",
                    "frac": 28 * achieved / pk["bf16_sustained"], "traffic": None,
                    "fp64_equivalent_tflops": achieved,
                    "fp64_equivalent_vs_fp64_peak": achieved / FP64_PEAK_TFLOPS,
                    "kernel": "k_f64s_colmax + k_f64s_panel + k_dht_f64s (FP64 DHT from exact BF16 slices on tcgen05)",
                    "peak_source": f"{pk['source']}: bf16 sustained {pk['bf16_sustained']} TFLOP/s; FP64 SIMT peak "
                                   "derived 152 SMs x 4 FP64 flop/clk x 2070 MHz",
                    "share_of_step": share}
    else:
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_PEAK_TFLOPS, "traffic": DHT_F64_TRAFFIC_BYTES,
                    "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, mean of the "
                                      "forward and inverse launch (profiles/k_gemm_f64__wake_2048x256_m2_fp64.md)",
                    "kernel": "k_gemm<double> (forward and inverse DHT, FP64 SIMT)",
                    "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x 2070 MHz (recipe nominal "
                                   "1.25 TFLOP/s); FMA probe measured 1.195 TFLOP/s",
                    "share_of_step": share}
    roofline_particles = None
    if not mixed:
        # the FP64 particle kernel against the derived FP64 peak, algorithmic operations of
        # fp64_particle_flops per particle (rho^{n+1} fused when the window is off)
        gp_s = stage_ms["gather_push"] / args.steps * 1e-3
        flops = n * fp64_particle_flops(w.Nm)
        ach = flops / gp_s / 1e12
        roofline_particles = {
            "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
            "algorithmic_flops": flops, "flops_per_particle": fp64_particle_flops(w.Nm),
            "kernel": "k_gather_push<false, true> (gather in double words, Boris push, J at x^{n+1/2}, "
                      "rho at x^{n+1}; FP64)",
            "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x 2070 MHz (recipe nominal 1.25 TFLOP/s)",
            "share_of_step": stage_ms["gather_push"] / sum(stage_ms.values()),
            "note": "operations counted in float64 as the algorithm states them; the kernel runs the gather's "
                    "interpolation and mode sum in double words on the FP32 units and the rest on the FP64 "
                    "pipe, the binding unit (profiles/k_gather_push__wake_2048x256_m2_fp64.md)"}
    if mixed:
        # the particle kernel (gather, push, J and rho deposits) against the survey's
        # algorithmic bytes: 56 B per particle (FP32 cell-relative state read and written,
        # 4 B key) + 10 complex-float grid passes (6 Nm field planes gathered, 4 Nm deposit
        # planes written); the copy of E and B into the gather layout is reported apart
        G = w.Nm * w.Nr * w.Nz
        bytes_alg = n * 56 + 10 * G * 8
        gp_s = stage_ms["gather_push"] / args.steps * 1e-3
        ach = bytes_alg / gp_s / 1e9
        lay_s = stage_ms["gather_layout"] / args.steps * 1e-3
        lay_bytes = 2 * 6 * G * 8
        full = (w.Nz, w.Nr, w.Nm, n) == (2048, 256, 2, 1348576)
        roofline_particles = {
            "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": ach / pk["hbm_gbs"],
            "algorithmic_bytes": bytes_alg,
            "traffic": PUSH_F32_TRAFFIC_BYTES if full else None,
            "kernel": "k_gather_push_f32 (gather, push, J and rho deposits)",
            "peak_source": f"{pk['source']}: hbm copy {pk['hbm_gbs']} GB/s",
            "share_of_step": stage_ms["gather_push"] / sum(stage_ms.values()),
            "state_bytes_per_particle": 96,
            "gather_layout": {"kernel": "k_nodes_rz", "ms_per_step": lay_s * 1e3,
                              "achieved": lay_bytes / max(lay_s, 1e-12) / 1e9, "unit": "GB/s",
                              "frac": lay_bytes / max(lay_s, 1e-12) / 1e9 / pk["hbm_gbs"]},
            "note": "bound by instruction issue and L1 latency (profiles/k_gather_push_f32__wake_2048x256_m2_mixed.md), "
                    "not by DRAM"}
    # `roofline` is the kernel with the largest share of the cycle; the other one beside it
    dominant = roofline
    if roofline_particles is not None and roofline_particles["share_of_step"] > roofline["share_of_step"]:
        dominant = roofline_particles
    out = {"steps_per_s": steps_per_s, "ms_per_step": el_ms / args.steps,
           "stage_ms_per_step": {k: v / args.steps for k, v in stage_ms.items()},
           "roofline": dominant, "roofline_dht": roofline, "roofline_particles": roofline_particles,
           "e2e": e2e, "gpu_launches": launches, "clocks": clk.summary(),
           "dtype": {bd.PIC_FP64: "f64", bd.PIC_MIXED_TF32X3: "f32+tf32x3",
                     bd.PIC_MIXED_BF16X6: "f32+bf16x6"}[prec]}
    if tuning is not None:
        out["tuning"] = tuning
    sim.close()
    del sim
    torch.cuda.empty_cache()
    return out


def accuracy_vs_fp64(w, P, npl, beams, n_cycles, local, sort_interval=1):
    """Error of both mixed forms against the FP64 form, run in lockstep from the same initial
    state, at checkpoints up to n_cycles: per field max |mixed - fp64| / max |fp64| over all
    components and modes, each beam's relative differences of normalised emittances and
    slice energy spread, and the worst of those beam differences."""
    import numpy as np
    import torch

    from paper_1611_05712_gb300 import binding as bd
    forms = (("fp64", bd.PIC_FP64), ("tf32x3", bd.PIC_MIXED_TF32X3), ("bf16x6", bd.PIC_MIXED_BF16X6))
    sims = {name: bd.Sim.from_workload(w, P, npl, beams, device=f"cuda:{local}", precision=pr) for name, pr in forms}
    for name, s in sims.items():
        s.set_sort_interval(sort_interval)   # as in the timed runs

    def rel(x, y):
        return float(np.abs(y - x).max() / max(np.abs(x).max(), 1e-300))

    names = ["drive" if bi == 0 and len(beams) > 1 else ("witness" if bi == len(beams) - 1 else f"beam{bi}")
             for bi in range(len(beams))]
    out = {"tf32x3": {}, "bf16x6": {}}
    done = 0
    for cp in sorted({c for c in (100, 500, 1000, n_cycles) if c <= n_cycles}):
        for s in sims.values():
            s.step(cp - done)
            s.sync()
        done = cp
        a = sims["fp64"]
        dep_a, E_a, B_a = a.get("DEP"), a.get("E"), a.get("B")
        ref = [a.diagnostics(lo, hi) for lo, hi, _ in beams]
        for form in ("tf32x3", "bf16x6"):
            b = sims[form]
            dep_b = b.get("DEP")
            row = {"E": rel(E_a, b.get("E")), "B": rel(B_a, b.get("B")), "J": rel(dep_a[1:], dep_b[1:]),
                   "rho": rel(dep_a[:1], dep_b[:1])}
            worst = 0.0
            for name, (lo, hi, _), da in zip(names, beams, ref):
                db = b.diagnostics(lo, hi)
                row[name] = {k: abs(db[k] - da[k]) / max(abs(da[k]), 1e-300)
                             for k in ("emit_nx", "emit_ny", "sigma_gamma_mean", "gamma_mean")}
                worst = max(worst, *(row[name][k] for k in ("emit_nx", "emit_ny", "sigma_gamma_mean")))
            row["worst_beam_metric"] = worst
            out[form][str(cp)] = row
    for s in sims.values():
        s.close()
    del sims
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import numpy as np
    import torch

    from paper_1611_05712_gb300 import binding as bd
    from paper_1611_05712_gb300 import workloads as W
    from paper_1611_05712_gb300.build import build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if rank == 0:
        build()
    if dist:
        dist.barrier()
    build()   # no-op once built; every rank needs the library loaded
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    w = workload(args.order, rank)
    P, npl, beams = W.particles(w)
    n = len(P["x"])
    head_prec = {"fp64": bd.PIC_FP64, "mixed": bd.PIC_MIXED_TF32X3, "bf16": bd.PIC_MIXED_BF16X6}[args.precision]
    head = measure(args, w, P, npl, beams, head_prec, dist, dev, world, local)
    line = {
        "metric": "pic_steps_per_s", "value": head["steps_per_s"], "unit": "steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": head["dtype"], "data": "synthetic", "config": config_of(w, n, args.precision, args.sort_interval),
        "particle_updates_per_s": head["steps_per_s"] * n,
        "stage_ms_per_step": head["stage_ms_per_step"],
        "roofline": head["roofline"], "roofline_dht": head["roofline_dht"],
        "roofline_particles": head["roofline_particles"],
        "e2e": head["e2e"], "gpu_launches": head["gpu_launches"], "clocks": head["clocks"],
    }
    if args.precision == "fp64" and not args.no_mixed:
        # the two mixed-precision forms on the same workload (3-term TF32 and 6-product BF16
        # DHT), their accuracy against the FP64 form, and the chosen one
        acc = (accuracy_vs_fp64(w, P, npl, beams, args.accuracy_cycles, local, args.sort_interval)
               if args.accuracy_cycles > 0 else {})
        for key, form, prec in (("mixed_form", "tf32x3", bd.PIC_MIXED_TF32X3),
                                ("mixed_form_bf16", "bf16x6", bd.PIC_MIXED_BF16X6)):
            mx = measure(args, w, P, npl, beams, prec, dist, dev, world, local)
            line[key] = {
                "value": mx["steps_per_s"], "unit": "steps/s", "dtype": mx["dtype"],
                "ms_per_step": mx["ms_per_step"], "particle_updates_per_s": mx["steps_per_s"] * n,
                "speedup_vs_fp64": mx["steps_per_s"] / head["steps_per_s"],
                "stage_ms_per_step": mx["stage_ms_per_step"], "roofline": mx["roofline"],
                "roofline_dht": mx["roofline_dht"], "roofline_particles": mx["roofline_particles"], "e2e": mx["e2e"],
                "gpu_launches": mx["gpu_launches"], "clocks": mx["clocks"], "tuning": mx.get("tuning")}
            if acc:
                line[key]["accuracy_vs_fp64"] = acc[form]
        if acc:
            # the chosen form: the fastest whose beam emittances and slice energy spreads stay
            # within 1e-4 of the FP64 form at the configuration's full length, with a factor 2
            # of margin: the float atomics that add the deposit bands to the grids run in a
            # varying order, and the wake amplifies the rounding differences, so one form's
            # worst metric scatters by about that factor from run to run
            last = str(args.accuracy_cycles)
            margin = 2.0
            ok = [(line[k]["value"], k) for k, f in (("mixed_form", "tf32x3"), ("mixed_form_bf16", "bf16x6"))
                  if acc[f][last]["worst_beam_metric"] * margin <= 1e-4]
            if ok:
                v, k = max(ok)
                line["chosen_form"] = {"form": k, "value": v, "unit": "steps/s",
                                       "speedup_vs_fp64": v / head["steps_per_s"],
                                       "worst_beam_metric_vs_fp64": acc["tf32x3" if k == "mixed_form" else "bf16x6"][last]
                                       ["worst_beam_metric"],
                                       "criterion": f"beam emittances and slice energy spreads within 1e-4 of the "
                                                    f"FP64 form after {last} cycles, with a factor {margin:g} of margin "
                                                    f"for run-to-run scatter"}
            else:
                line["chosen_form"] = {"form": None, "criterion": f"no mixed form within 1e-4 / {margin:g} after {last} "
                                                                  f"cycles"}
    if world == 1 and args.precision == "fp64" and not args.no_extra:
        # the configurations the metric also names: the large single run (8192 x 1024, 3 modes,
        # mixed form, with its accuracy against the FP64 form) and the batched scan
        large = measure_large(args, local, None, 1, args.large_accuracy_cycles)
        line["large"] = {k: large[k] for k in ("value", "unit", "ms_per_step", "particle_updates_per_s", "dtype",
                                               "stage_ms_per_step", "roofline", "roofline_dht", "roofline_particles", "e2e",
                                               "clocks", "tuning", "config")}
        if "accuracy_vs_fp64" in large:
            line["large"]["accuracy_vs_fp64"] = large["accuracy_vs_fp64"]
        scan = measure_scan(args, local)
        line["scan"] = {k: scan[k] for k in ("value", "unit", "ms_per_step", "particle_updates_per_s", "dtype",
                                             "gpu_launches", "graph_launches", "clocks", "config")}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, secs = oracle_steps_per_s(w, P, npl, beams, 1)
        line["cpu_baseline"] = {"value": v, "unit": "steps/s", "cores": os.cpu_count(),
                                "kind": "oracle",
                                "sample": f"1 full cycle of the same workload ({secs:.1f} s; numpy FP64 "
                                          "oracle, BLAS threads = host cores)"}
        if "large" in line:
            line["large"]["cpu_baseline"] = oracle_crop_baseline(args)
        if "scan" in line:
            line["scan"]["cpu_baseline"] = oracle_scan_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def measure_scan(args, local, dist=None, rank=0, world=1):
    """Batched order / resolution scan: args.sims independent simulations (Nz 7-smooth in
    [512, 4096], Nr in [64, 512], Nm in {1,2,3}, p in {8..64, inf}, c dt/dz in {0.5, 1}),
    mixed form, each on its own stream, advanced together by one captured CUDA graph
    (2 cycles per launch).  value = sum over simulations of cycles / s."""
    import concurrent.futures as cf

    import torch

    from paper_1611_05712_gb300 import binding as bd
    from paper_1611_05712_gb300 import workloads as W
    dev = torch.device("cuda", local)
    members = [W.scan_member(rank * args.sims + s) for s in range(args.sims)]
    parts = [W.particles(w) for w in members]
    streams = [torch.cuda.Stream(dev) for _ in members]
    t0 = time.perf_counter()

    def init(i):
        P, npl, beams = parts[i]
        return bd.Sim.from_workload(members[i], P, npl, beams, precision=bd.PIC_MIXED_TF32X3,
                                    device=f"cuda:{local}", stream=streams[i])

    with cf.ThreadPoolExecutor(max_workers=16) as ex:
        sims = list(ex.map(init, range(len(members))))
    init_s = time.perf_counter() - t0
    # tile sizes per member, one at a time so that the timings do not overlap
    # each graph launch runs 2 cycles: sort on one of them (sort interval 2)
    for s in sims:
        s.set_sort_interval(min(args.sort_interval, 2))
    tunings = [s.autotune() for s in sims]
    setup_s = time.perf_counter() - t0
    batch = bd.Batch(sims, cycles=2)
    batch.launch(max(1, args.warmup // 2 + 1))
    batch.origin.synchronize()
    launches = max(1, args.steps // 2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        if args.profile_range:
            torch.cuda.profiler.start()
        e0.record(batch.origin)
        batch.launch(launches)
        e1.record(batch.origin)
        e1.synchronize()
        if args.profile_range:
            torch.cuda.profiler.stop()
    ms = reduce_max(e0.elapsed_time(e1), dist, dev)
    cycles = 2 * launches
    n_tot = sum(len(p[0]["x"]) for p in parts)
    value = weak_throughput(cycles * len(sims), world, ms)
    line = {
        "metric": "pic_steps_per_s", "value": value, "unit": "sim-steps/s", "n_gpus": world,
        "steps": cycles, "warmup": 2 * max(1, args.warmup // 2 + 1), "ms_per_step": ms / cycles,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+tf32x3",
        "data": "synthetic",
        "config": {"workload": f"scan_{len(sims)}_uneven_sims", "sims": len(sims),
                   "cells": int(sum(w.Nz * w.Nr * w.Nm for w in members)), "particles": n_tot,
                   "Nz": [w.Nz for w in members], "Nr": [w.Nr for w in members],
                   "Nm": [w.Nm for w in members], "order_p": [w.order_p for w in members],
                   "cdt_over_dz": [round(299792458.0 * w.dt / w.dz, 3) for w in members],
                   "cycles_per_graph_launch": 2, "init_s": init_s, "setup_s": setup_s,
                   "dht_n_tile": [t["dht_n_tile"] for t in tunings],
                   "band_chunk": [t["band_chunk"] for t in tunings]},
        "particle_updates_per_s": world * cycles * n_tot / (ms * 1e-3),
        "gpu_launches": batch.kernels_per_launch * launches, "graph_launches": launches,
        "clocks": clk.summary(),
    }
    batch.close()
    for s in sims:
        s.close()
    del sims, batch
    torch.cuda.empty_cache()
    return line


def run_scan(args):
    import torch

    from paper_1611_05712_gb300.build import build
    build()
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    line = measure_scan(args, local, dist, rank, world)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def accuracy_large(w, P, npl, beams, n_cycles, local, sort_interval):
    """The mixed forms against the FP64 form on the large workload after n_cycles cycles from
    one initial state: per field max |mixed - fp64| / max |fp64| over all components and
    modes, and each beam's relative differences of normalised emittances and slice energy
    spread."""
    import numpy as np
    import torch

    from paper_1611_05712_gb300 import binding as bd

    def rel(x, y):
        return float(np.abs(y - x).max() / max(np.abs(x).max(), 1e-300))

    ref = bd.Sim.from_workload(w, P, npl, beams, device=f"cuda:{local}", precision=bd.PIC_FP64)
    ref.set_sort_interval(sort_interval)
    t0 = time.perf_counter()
    ref.step(n_cycles)
    ref.sync()
    fp64_s = time.perf_counter() - t0
    dep_a, E_a, B_a = ref.get("DEP"), ref.get("E"), ref.get("B")
    d_a = [ref.diagnostics(lo, hi) for lo, hi, _ in beams]
    ref.close()
    del ref
    torch.cuda.empty_cache()
    names = ["drive", "witness"] if len(beams) == 2 else [f"beam{i}" for i in range(len(beams))]
    keys = ("emit_nx", "emit_ny", "sigma_gamma_mean", "gamma_mean")
    # the beams start cold (u_perp = 0): their emittances grow from zero, so early relative
    # differences divide by a small quantity; the FP64 values and absolute differences are
    # reported beside them
    out = {"cycles": n_cycles, "fp64_s_per_cycle": fp64_s / n_cycles,
           "fp64_values": {name: {k: da[k] for k in keys} for name, da in zip(names, d_a)}}
    for form, prec in (("tf32x3", bd.PIC_MIXED_TF32X3), ("bf16x6", bd.PIC_MIXED_BF16X6)):
        s = bd.Sim.from_workload(w, P, npl, beams, device=f"cuda:{local}", precision=prec)
        s.set_sort_interval(sort_interval)
        s.step(n_cycles)
        s.sync()
        dep_b = s.get("DEP")
        row = {"E": rel(E_a, s.get("E")), "B": rel(B_a, s.get("B")), "J": rel(dep_a[1:], dep_b[1:]),
               "rho": rel(dep_a[:1], dep_b[:1])}
        for name, (lo, hi, _), da in zip(names, beams, d_a):
            db = s.diagnostics(lo, hi)
            row[name] = {k: abs(db[k] - da[k]) / max(abs(da[k]), 1e-300) for k in keys}
            row[name + "_abs"] = {k: abs(db[k] - da[k]) for k in keys}
        out[form] = row
        s.close()
        del s
        torch.cuda.empty_cache()
    return out


def measure_large(args, local, dist=None, world=1, accuracy_cycles=0, crop=False):
    """The large single run: 8192 x 1024, 3 modes, p = 32, 12 plasma macroparticles per cell
    plus 1M-particle drive and witness beams (~102.7M particles), mixed form; with
    accuracy_cycles > 0 also both mixed forms against the FP64 form after that many cycles.
    crop: its 1024 x 128 crop (same plasma, scaled beams; 1.6M particles) instead."""
    import torch

    from paper_1611_05712_gb300 import binding as bd
    from paper_1611_05712_gb300 import workloads as W
    dev = torch.device("cuda", local)
    w = W.large_crop_1024x128(order_p=args.order) if crop else W.large_8192x1024(order_p=args.order)
    t0 = time.perf_counter()
    P, npl, beams = W.particles(w)
    gen_s = time.perf_counter() - t0
    n = len(P["x"])
    e2e_steps = args.e2e_steps
    args.e2e_steps = min(args.e2e_steps, 2)   # each end-to-end cycle uploads 5.8 GB of particles
    t0 = time.perf_counter()
    try:
        mx = measure(args, w, P, npl, beams, bd.PIC_MIXED_TF32X3, dist, dev, world, local)
    finally:
        args.e2e_steps = e2e_steps
    run_s = time.perf_counter() - t0
    cfg = config_of(w, n, "mixed")
    cfg["l2"] = ("no flush: working set (fields + particles, ~0.3 GB) exceeds the 129 MB L2" if crop else
                 "no flush: working set (fields + particles, ~21 GB) exceeds the 129 MB L2")
    cfg["host_generation_s"] = gen_s
    cfg["setup_and_run_s"] = run_s
    line = {
        "metric": "pic_steps_per_s", "value": mx["steps_per_s"], "unit": "steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mx["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": mx["dtype"],
        "data": "synthetic", "config": cfg, "particle_updates_per_s": mx["steps_per_s"] * n,
        "stage_ms_per_step": mx["stage_ms_per_step"], "roofline": mx["roofline"],
        "roofline_dht": mx["roofline_dht"], "roofline_particles": mx["roofline_particles"], "e2e": mx["e2e"],
        "gpu_launches": mx["gpu_launches"], "clocks": mx["clocks"], "tuning": mx.get("tuning"),
    }
    if accuracy_cycles > 0:
        line["accuracy_vs_fp64"] = accuracy_large(w, P, npl, beams, accuracy_cycles, local, args.sort_interval)
    return line


def run_large(args):
    import torch

    from paper_1611_05712_gb300.build import build
    build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    line = measure_large(args, local, dist, world, args.large_accuracy_cycles, crop=args.workload == "crop")
    if int(os.environ.get("RANK", "0")) == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_guard(args):
    """Guard-cell domain decomposition along z (FP64, no sources): max relative difference
    between four subdomains advanced with their own FFT over interior + g guard cells and
    the global field step, for stencil orders p and guard widths g."""
    import numpy as np

    from paper_1611_05712_gb300 import binding as bd
    from paper_1611_05712_gb300.build import build
    from paper_1611_05712_gb300.domains import GuardedDomains
    build()
    c_light = 299792458.0
    Nz, Nr, Nm, dz = 512, 32, 2, 0.05e-6
    table = {}
    for p in (8, 16, 32, 64, 0):
        row = {}
        for g in (0, 8, 16, 32, 48, 64, 96, 128):
            cfg = bd.make_config(Nz, Nr, Nm, dz, dz, dz / c_light, p, True, bd.PIC_FP64, 0)
            glob, out = bd.Sim(cfg), bd.Sim(cfg)
            for h in (glob, out):   # the SIMT DHT: its FP64 rounding floor shows the locality
                h.set_dht_path(bd.PIC_DHT_F64_GEMM)
            rng = np.random.default_rng(7)
            shape = (3, Nm, Nr, Nz)
            glob.set("E", rng.normal(size=shape) + 1j * rng.normal(size=shape))
            glob.set("B", (rng.normal(size=shape) + 1j * rng.normal(size=shape)) / c_light)
            for h in (glob, out):
                h.set("DEP", h.zeros("DEP"))
                h.set("RHO_PREV_H", h.zeros("RHO_PREV_H"))
            dom = GuardedDomains(cfg, 4, g, dht_path=bd.PIC_DHT_F64_GEMM)
            dom.field_step(glob, out)
            glob.fields_to_spectral()
            glob.field_step()
            err = 0.0
            for name in ("E", "B"):
                a, b = out.get(name), glob.get(name)
                err = max(err, float(np.abs(a - b).max() / np.abs(b).max()))
            row[g] = err
            for h in (dom, glob, out):
                h.close()
        table["inf" if p == 0 else str(p)] = row
    print(json.dumps({"metric": "guard_cell_decomposition_error", "unit": "max relative difference",
                      "config": {"Nz": Nz, "Nr": Nr, "Nm": Nm, "subdomains": 4, "precision": "fp64",
                                 "fields": "random E, B, no sources", "steps": 1},
                      "error_by_order_and_guard": table}), flush=True)
    return 0


def run_order_sweep(args):
    """Order study of the beam-driven wakefield (2048 x 256, 2 modes): the same initial
    state advanced args.sweep_steps cycles at each stencil order p and at infinite order;
    Err_eps, Err_sigma_gamma (witness beam) and Err_Ez of each finite order against the
    infinite-order run (numerical Cherenkov radiation measures of the paper)."""
    from paper_1611_05712_gb300 import binding as bd
    from paper_1611_05712_gb300 import ncr
    from paper_1611_05712_gb300 import workloads as W
    from paper_1611_05712_gb300.build import build
    build()
    prec = {"fp64": bd.PIC_FP64, "mixed": bd.PIC_MIXED_TF32X3, "bf16": bd.PIC_MIXED_BF16X6}[args.precision]
    w = W.wake_2048x256(order_p=0)
    P, npl, beams = W.particles(w)
    lo, hi = beams[-1][0], beams[-1][1]
    runs = {}
    t0 = time.perf_counter()
    for p in (0, 4, 8, 16, 32, 64, 128, 256):
        s = bd.Sim.from_workload(w, P, npl, beams, precision=prec, order_p=p)
        if prec != bd.PIC_FP64:
            s.autotune()
        s.step(args.sweep_steps)
        d = s.diagnostics(lo, hi)
        runs[p] = (d, ncr.ez_plane(s.get("E")), ncr.beam_of(s.read_particles(), lo, hi))
        s.close()
    ref_d, ref_ez, ref_beam = runs[0]
    res = {}
    for p in (4, 8, 16, 32, 64, 128, 256):
        d, ez, beam = runs[p]
        res[str(p)] = {"err_eps_x": ncr.err_emittance(d["emit_nx"], ref_d["emit_nx"]),
                       "err_eps_y": ncr.err_emittance(d["emit_ny"], ref_d["emit_ny"]),
                       # both runs sliced on the infinite-order run's grid
                       "err_sigma_gamma": ncr.err_sigma_gamma_runs(beam, ref_beam),
                       "err_ez": ncr.err_ez(ez, ref_ez), "err_ez_l2": ncr.err_ez_l2(ez, ref_ez)}
    print(json.dumps({"metric": "ncr_order_sweep", "unit": "relative error vs infinite order",
                      "config": {"workload": w.name, "cycles": args.sweep_steps, "precision": args.precision,
                                 "beam": "witness", "reference": "p = inf, same initial state",
                                 "wall_s": time.perf_counter() - t0},
                      "errors_by_order": res}), flush=True)
    return 0


def run_window(args):
    """The wakefield run (2048 x 256, 2 modes, p = 32) in a window moving at c, one cell per
    cycle: cycles/s with and without the window from the same initial state (the window's
    cost), then args.window_cycles further cycles checking that the beams keep their window
    coordinates and that removal and injection keep the plasma balanced."""
    import torch

    from paper_1611_05712_gb300 import binding as bd
    from paper_1611_05712_gb300 import workloads as W
    from paper_1611_05712_gb300.build import build
    build()
    prec = {"fp64": bd.PIC_FP64, "mixed": bd.PIC_MIXED_TF32X3, "bf16": bd.PIC_MIXED_BF16X6}[args.precision]
    mixed = prec != bd.PIC_FP64
    w = workload(args.order)
    P, npl, beams = W.particles(w)
    n = len(P["x"])
    # inside the wake the plasma electrons move forward and stay longer in the window, so the
    # window holds more plasma than it was loaded with until the wake fills it: keep a
    # quarter of the plasma in reserve
    reserve = npl // 4

    def timed(sim, k):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(sim.stream)
        sim.step(k)
        e1.record(sim.stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    def make():
        sim = bd.Sim.from_workload(w, P, npl, beams, precision=prec, capacity=n + reserve)
        if mixed:
            sim.set_sort_interval(args.sort_interval)
            sim.autotune()
        return sim

    s = make()
    s.step(args.warmup)
    ms_plain = timed(s, args.steps)
    s.close()

    s = make()
    s.window_setup(npl, 1, reserve)
    d0 = [s.diagnostics(lo, hi) for lo, hi, _ in beams]
    s.step(args.warmup)
    l0 = s.launch_count()
    with ClockSampler(0) as clk:
        ms_win = timed(s, args.steps)
    launches = s.launch_count() - l0
    wall = 0.0
    samples = []
    done = 0
    while done < args.window_cycles:
        k = min(1024, args.window_cycles - done)
        t0 = time.perf_counter()
        s.step(k)
        s.sync()
        wall += time.perf_counter() - t0
        done += k
        pk = s.read_particles()   # untimed: active plasma count along the propagation
        act = pk["w"] != 0
        samples.append([done, int((act & ((pk["id"] < npl) | (pk["id"] >= n))).sum()),
                        s.window_state()["dropped"]])
    info = s.window_state()
    d1 = [s.diagnostics(lo, hi) for lo, hi, _ in beams]
    parts = s.read_particles()
    active = parts["w"] != 0
    plasma_active = int((active & (parts["id"] < npl)).sum()) + int((active & (parts["id"] >= n)).sum())
    beams_out = {}
    for (lo, hi, gam), a, b in zip(beams, d0, d1):
        beams_out[f"gamma_{gam:g}"] = {
            "z_window_start_um": a["z_mean"] * 1e6, "z_window_end_um": b["z_mean"] * 1e6,
            "gamma_mean_start": a["gamma_mean"], "gamma_mean_end": b["gamma_mean"],
            "emit_nx_start": a["emit_nx"], "emit_nx_end": b["emit_nx"],
            "particles_active": int((active & (parts["id"] >= lo) & (parts["id"] < hi)).sum()), "particles": hi - lo}
    cfg = config_of(w, n, args.precision)
    cfg.update({"window": "moves one cell per cycle (c dt = dz)", "reserve": reserve,
                "propagation_cycles": args.window_cycles,
                "propagation_um": args.window_cycles * w.dz * 1e6})
    steps_win = args.steps / (ms_win * 1e-3)
    print(json.dumps({
        "metric": "pic_steps_per_s_moving_window", "value": steps_win, "unit": "steps/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_win / args.steps,
        "ms_per_step_without_window": ms_plain / args.steps,
        "window_overhead_ms_per_step": (ms_win - ms_plain) / args.steps,
        "higher_is_better": True, "dtype": {bd.PIC_FP64: "f64", bd.PIC_MIXED_TF32X3: "f32+tf32x3",
                                            bd.PIC_MIXED_BF16X6: "f32+bf16x6"}[prec],
        "data": "synthetic", "config": cfg, "gpu_launches": launches, "clocks": clk.summary(),
        "propagation": {"wall_s": wall, "cycles_per_s": args.window_cycles / wall,
                        "shifts": info["shifts"], "dropped": info["dropped"],
                        "plasma_active_start": npl, "plasma_active_end": plasma_active,
                        "plasma_active_samples": {"columns": ["cycles", "active_plasma", "dropped"],
                                                  "rows": samples},
                        "beams": beams_out}}), flush=True)
    s.close()
    return 0


def run_fft_lengths(args):
    """Cost of the z transforms at lengths that are not 7-smooth (Bluestein rows) against the
    nearest power of two: the wakefield configuration (256 r nodes, 2 modes, p = 32) at
    Nz = 2048 and at the prime Nz = 2039, per-stage device times of args.steps cycles."""
    import dataclasses

    from paper_1611_05712_gb300 import binding as bd
    from paper_1611_05712_gb300 import workloads as W
    from paper_1611_05712_gb300.build import build
    build()
    prec = {"fp64": bd.PIC_FP64, "mixed": bd.PIC_MIXED_TF32X3, "bf16": bd.PIC_MIXED_BF16X6}[args.precision]
    out = {}
    for nz in (2048, 2039):
        w = dataclasses.replace(W.wake_2048x256(order_p=args.order), Nz=nz)
        P, npl, beams = W.particles(w)
        s = bd.Sim.from_workload(w, P, npl, beams, precision=prec)
        if prec != bd.PIC_FP64:
            s.autotune()
        s.step(args.warmup)
        st, tot = s.step_timed(args.steps)
        out[str(nz)] = {"ms_per_step": tot / args.steps,
                        "fft_fwd_ms": st["fft_fwd"] / args.steps, "fft_inv_ms": st["fft_inv"] / args.steps,
                        "dht_ms": (st["dht_fwd"] + st["dht_inv"]) / args.steps}
        s.close()
    print(json.dumps({"metric": "z_transform_cost_by_length", "unit": "ms per cycle", "precision": args.precision,
                      "config": {"Nr": 256, "Nm": 2, "order_p": args.order, "steps": args.steps,
                                 "lengths": {"2048": "power of two (radix-8 rows)",
                                             "2039": "prime (Bluestein, M = 4096)"}},
                      "by_length": out}), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "scan":
        return run_scan(args)
    if args.workload in ("large", "crop"):
        return run_large(args)
    if args.workload == "guard":
        return run_guard(args)
    if args.workload == "order_sweep":
        return run_order_sweep(args)
    if args.workload == "window":
        return run_window(args)
    if args.workload == "fft_lengths":
        return run_fft_lengths(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
