#!/usr/bin/env python
"""Benchmark of the mu_ex hot path: one step = one evaluation of the cDFT
excess chemical potentials (FMT hard spheres, Rosenfeld) of a 128^3 grid with
three species of radius 1.5h, 2h, 3h (packing 0.1 each, densities rho_b x
lognormal(0, 0.1), seed 2), zero-padded to 256^3, through the C ABI
(pnp_excess_mu_device) with inputs resident in device memory.

Prints one JSON line (rank 0).  Metric: mu_ex Gpoints/s = output grid points /
time.  The headline is the FP64-accuracy path: FFT arithmetic in double-float
(pairs of FP32, ~48 bits; within 1e-10 of the FP64 oracle like plain FP64),
FMT derivatives in FP64; its dominant kernel is bound by the FP32 pipes and is
reported against their peak.  Beside it: the FP32-FFT variant (singular terms
of the derivatives in FP64) and the 3xTF32 tensor-core variant against the HBM
roofline, and the plain FP64 form, each with its error against the FP64 path.
`e2e` times pnp_excess_mu with host buffers (pinned), host->device and
device->host copies inside the timed region.  `solves` (after the timed
region) serves `--solves` independent Gummel solves of the batch recipe
concurrently and runs the same solves one at a time in plain FP64: solves/s,
speed-up, p50/p99 latency and the largest density difference.

`--impl reference` times the FP64 CPU oracle (direct real-space quadrature
sums) on a bounded sample of the same workload; it is the reference arm.

Multi-GPU: the workload does not shard, so N ranks run N independent replicas
(weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_EDGE = 128
PAD = 256
SPECIES = 3
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=40, help="edge of the oracle sample box")
    ap.add_argument("--ref-sample", type=int, default=24, help="edge of the reference-arm sample box")
    ap.add_argument("--n", type=int, default=N_EDGE, help="grid edge (profiling runs use smaller cases)")
    ap.add_argument("--pad", type=int, default=PAD, help="padded FFT length")
    ap.add_argument("--bias-points", type=int, default=11, help="film3: points of the 0..1 kT/e bias sweep")
    ap.add_argument("--film3-start", default="warm", choices=["warm", "eq"],
                    help="film3: warm-start each bias point from the previous one, or start each from its equilibrium")
    ap.add_argument("--max-iter3", type=int, default=2000, help="film3: Gummel iteration cap per bias point")
    ap.add_argument("--solve-prec", default="df64", choices=["fp64", "df64", "fp32", "tf32split"],
                    help="mu_ex precision of the batched / served solves (the sequential baseline is plain FP64)")
    ap.add_argument("--autotune", type=int, default=0,
                    help="autotune the batched / served problems' plans (timing candidates on a loaded GPU)")
    ap.add_argument("--solve-aa", type=int, default=0,
                    help="Anderson depth of the batched / served solves (0: the recipe's relaxation; > 0 with the "
                         "step-limited geometric relaxation); the sequential FP64 baseline keeps the recipe's")
    ap.add_argument("--film-aa", type=int, default=3,
                    help="film workload: Anderson depth of the solve reported beside the plain one (0: none)")
    ap.add_argument("--policy", default="smallest_first", choices=["fifo", "smallest_first"],
                    help="admission policy of the batched / served solves")
    ap.add_argument("--slots", type=int, default=4, help="concurrently resident batched / served solves")
    ap.add_argument("--variants", default="df64,fp32,tf32split,fp64", help="precisions to time, headline first")
    ap.add_argument("--solves", type=int, default=16,
                    help="mu_ex workload: solves of the batch recipe served concurrently, against the same solves "
                         "one at a time in plain FP64, reported beside the mu_ex line (0: none)")
    ap.add_argument("--workload", default="mu_ex", choices=["mu_ex", "film", "film3", "batch", "serve"],
                    help="mu_ex (headline), film (one 32^3 Gummel solve), film3 (128x128x256 bias sweep), "
                         "batch (64 solves), serve (arrivals)")
    ap.add_argument("--batch", type=int, default=64, help="solves in the batch workload")
    ap.add_argument("--seq", type=int, default=8, help="solves timed one at a time as the sequential baseline")
    ap.add_argument("--requests", type=int, default=40, help="served requests")
    ap.add_argument("--rate", type=float, default=20.0, help="request arrivals per second")
    ap.add_argument("--max-edge", type=int, default=96, help="largest served grid edge")
    return ap.parse_args()


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)     # one GPU per rank before NCCL sees a device
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(world, v):
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sub_box(spec, rho, m):
    import copy
    s2 = copy.copy(spec)
    s2.nx = s2.ny = s2.nz = m
    s2.fft_len = (0, 0, 0)
    import numpy as np
    return s2, np.ascontiguousarray(rho[:, :m, :m, :m])


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.idx), "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def stage_bytes(name, dims, cs, s):
    """Algorithmic DRAM bytes of one launch of a pipeline stage: every array
    element the pass must read plus every element it must write (complex
    element cs bytes, real FP64 fields 8 bytes), spectra octants once."""
    nx, ny, nz, Lx, Ly, Lz = dims
    Wx = Lx // 2 + 1
    A1 = nz * ny * Wx * cs           # one field, x-spectra
    B1 = nz * Ly * Wx * cs           # one field, y-spectra
    R1 = nx * ny * nz * 8            # one real field
    oct_ = (Lx // 2 + 1) * (Ly // 2 + 1) * (Lz // 2 + 1) * (cs // 2) * 5 * s
    return {
        "x_fwd": s * (R1 + A1),
        "y_fwd": s * (A1 + B1),
        "z_mac": s * B1 + 10 * B1 + oct_,
        "y_inv": 10 * (B1 + A1),
        "x_fused": 10 * (A1 + A1),
        "y_fwd_psi": 10 * (A1 + B1),
        "z_back": 10 * B1 + s * B1 + oct_,
        "y_inv_mu": s * (B1 + A1),
        "x_inv": s * (A1 + R1),
    }[name]


STAGES = ("x_fwd", "y_fwd", "z_mac", "y_inv", "x_fused", "y_fwd_psi", "z_back", "y_inv_mu", "x_inv")


def path_bytes(dims, cs, s):
    """Algorithmic bytes of one whole mu_ex: the nine stages' sum."""
    return sum(stage_bytes(n, dims, cs, s) for n in STAGES)


def pass_model_bytes(dims, s, w):
    """Bytes of the unfused pass model of one mu_ex: T = s + 10 + min(10, 1 + 4s)
    + s real 3D transforms (the densities, the ten weighted densities, the
    non-zero derivative fields, the chemical potentials), each three axis
    passes that read and write all Lx Ly Lz values of w bytes."""
    nx, ny, nz, Lx, Ly, Lz = dims
    T = s + 10 + min(10, 1 + 4 * s) + s
    return T * 3 * 2 * Lx * Ly * Lz * w


# register-FFT lengths of the library's kernels
REG_LENGTHS = (16, 20, 24, 32, 40, 48, 64, 80, 96, 128, 256)


def kernels_per_stage(name, Lx):
    """Kernel launches one timed stage makes: the derivative stage runs as
    three kernels (10-field C2R, pointwise derivatives, 10-field R2C) when the
    x length has a register FFT, as one fused kernel otherwise; every other
    stage is one kernel."""
    if name == "x_fused" and Lx in REG_LENGTHS:
        return 3
    return 1


def stage_flops(name, dims, s):
    """Algorithmic floating-point operations of one launch of a stage: 5 L log2 L
    per complex transform of length L (a pair of real lines shares one), plus
    4 flops per species per output element of each spectral multiply-add and
    about 60 per point for the ten FMT derivatives."""
    import math
    nx, ny, nz, Lx, Ly, Lz = dims
    Wx = Lx // 2 + 1
    npairs = (ny + 1) // 2
    fx, fy, fz = (5 * L * math.log2(L) for L in (Lx, Ly, Lz))
    cols = Ly * Wx
    mac = 10 * s * 4 * Lz
    return {
        "x_fwd": s * nz * npairs * fx,
        "y_fwd": s * nz * Wx * fy,
        "z_mac": cols * ((s + 10) * fz + mac),
        "y_inv": 10 * nz * Wx * fy,
        "x_fused": nz * npairs * 20 * fx + nx * ny * nz * 60,
        "y_fwd_psi": 10 * nz * Wx * fy,
        "z_back": cols * ((s + 10) * fz + mac),
        "y_inv_mu": s * nz * Wx * fy,
        "x_inv": s * nz * npairs * fx,
    }[name]


# DRAM bytes per launch measured by ncu for a kernel (profiles/), scaled to
# the 128^3 workload by the rows it moves; set to None whenever the kernel
# changes after the capture.
PROFILED_TRAFFIC = {
    ("fp64", "z_back"): 1.1299e9,     # k_zback_p_fp64_120_pad256.md
    ("fp32", "z_back"): None,
    # k_zq4_dd_120_pad256.md: 1054.9 / 1083.1 MB at 120^3, x (algorithmic
    # bytes at 128^3 / at 120^3) = 1137 / 1082 MB
    ("df64", "z_mac"): 1.1085e9,
    ("df64", "z_back"): 1.1382e9,
}
# FP32-pipe instructions (thread-level FADD + FMUL + FFMA) one launch of a
# double-float kernel executes, from ncu's per-opcode counts (profiles/): the
# work its number format costs the FP32 pipes.  A z kernel transforms every
# one of the Ly x Wx columns over the full length Lz, with the same pruned
# butterflies for any nz <= Lz / 2, so the 120^3 capture holds for 128^3 as
# it is.  None for a kernel changed since.
PROFILED_FP32_INST = {
    ("df64", "z_mac"): 4.1615e10,      # k_zq4_dd_120_pad256.md
    ("df64", "z_back"): 4.1128e10,
}

DTYPE = {"fp64": "f64",
         "df64": "df64 (FFT values and FMT derivative products as FP32 pairs, ~48-bit; "
                 "FP64 singular terms ln(1 - n3), 1/(1 - n3))",
         "fp32": "f32 FFT / f64 singular terms of the FMT derivatives",
         "tf32split": "f32 FFT with the y-axis radix-16 DFT stages as 3xTF32 tensor-core products / "
                      "f64 singular terms of the FMT derivatives"}
VARIANT_NAME = {"fp64": "fp64_plain", "df64": "df64_fft", "fp32": "fp32_fft", "tf32split": "tf32split_fft"}
# error bound each variant is tested to against the oracle (normwise per species)
ERROR_BOUND = {"fp64": 1e-10, "df64": 1e-10, "fp32": 2e-5, "tf32split": 5e-5}

# FP64 peak of the part, from its unit counts and clock: 152 SMs x 2 FP64 FMA
# per clock x 2 flops x 2.07 GHz (an FMA-chain probe measured 1.195 TFLOP/s).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP32_PEAK_TINST = 152 * 128 * 2.07e9 / 1e12


def run_reference(args, world, rank):
    if rank != 0:
        return
    import numpy as np
    from oracle import oracle
    from workloads import mu_microbench
    spec, rho = mu_microbench(N_EDGE, fft_len=PAD)
    # sub-box edge: at most --ref-sample, small enough that warm-up + timed
    # steps take about 90 s of CPU (cost measured on a 12^3 box, scaled by volume)
    sc, rc = sub_box(spec, rho, 12)
    t1 = time.perf_counter()
    oracle.excess_mu(sc, rc)
    t_cal = time.perf_counter() - t1
    m = args.ref_sample
    while m > 8 and (args.steps + args.warmup) * t_cal * (m / 12) ** 3 > 90.0:
        m -= 2
    s2, r2 = sub_box(spec, rho, m)
    for _ in range(args.warmup):
        oracle.excess_mu(s2, r2)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.excess_mu(s2, r2)
    dt = (time.perf_counter() - t0) / args.steps
    v = m ** 3 / dt / 1e9
    line = {
        "impl": "reference", "metric": "mu_ex Gpoints/s", "value": v, "unit": "Gpoints/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"mu_ex {N_EDGE}^3 x {SPECIES} species (R 1.5/2/3 h), zero-padded {PAD}^3",
                   "sample": f"{m}^3 sub-box per step", "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": v, "unit": "Gpoints/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "cpu_model": cpu_model(),
                         "sample": f"{m}^3 sub-box of the {N_EDGE}^3 workload, full mu_ex per step"},
        "e2e": {"value": v, "unit": "Gpoints/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gpu(args, world, rank, local):
    import numpy as np
    import torch
    from paper_1407_0674_gb300 import build as lb
    from paper_1407_0674_gb300 import pnp
    from workloads import mu_microbench

    torch.cuda.set_device(local)
    lb.build()
    spec, rho = mu_microbench(args.n, fft_len=args.pad)
    npts = spec.npoints
    variants = args.variants.split(",")
    P = pnp.Problem(spec)
    info = P.info()
    d_rho = torch.from_numpy(rho).cuda()
    d_mu = torch.empty_like(d_rho)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    # a dedicated stream: the library, the L2 flush and the timing events all
    # run on it (handle 0 would mean the library's own stream)
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream
    torch.cuda.set_stream(stream)

    def step(prec):
        P.excess_mu_device(d_rho, d_mu, precision=prec, stream=sh)

    for prec in variants:
        for _ in range(args.warmup):
            step(prec)
    torch.cuda.synchronize()
    rc = P.status()
    if rc != 0:
        raise RuntimeError(f"device status {rc} after warm-up")

    results = {}
    clocks = None
    for prec in variants:
        P.stage_times()                      # reset the record
        P.stage_timing(True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        sampler = ClockSampler(local) if prec == variants[0] else None
        if sampler:
            sampler.start()
            time.sleep(0.3)
        barrier(world)
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.zero_()                    # evict L2 between steps (outside the events)
            ev[k][0].record(stream)
            step(prec)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        if sampler:
            clocks = sampler.stop()
        P.stage_timing(False)
        st = P.stage_times()
        rc = P.status()
        if rc != 0:
            raise RuntimeError(f"device status {rc}")
        ms = [a.elapsed_time(b) for a, b in ev]
        ms_step = reduce_max(world, sum(ms) / len(ms))
        results[prec] = {"ms": ms_step, "stages": st}

    # each variant's error against the FP64 path (itself within 1e-10 of the
    # oracle in the parity tests): max over species of ||mu - mu64|| / ||mu64||
    errs = {}
    if rank == 0:
        P.excess_mu_device(d_rho, d_mu, precision="fp64", stream=sh)
        torch.cuda.synchronize()
        mu64 = d_mu.cpu().numpy().reshape(SPECIES, -1)
        for prec in variants:
            if prec == "fp64":
                continue
            P.excess_mu_device(d_rho, d_mu, precision=prec, stream=sh)
            torch.cuda.synchronize()
            m = d_mu.cpu().numpy().reshape(SPECIES, -1)
            errs[prec] = max(float(abs(m[i] - mu64[i]).max() / abs(mu64[i]).max()) for i in range(SPECIES))

    # end to end through the host-pointer entry point, pinned host buffers
    h_rho = torch.from_numpy(rho).pin_memory().numpy()
    h_mu = torch.empty(rho.shape, dtype=torch.float64).pin_memory().numpy()
    lib = pnp.lib()
    import ctypes
    dp = ctypes.POINTER(ctypes.c_double)
    for _ in range(2):
        lib.pnp_excess_mu(P.h, h_rho.ctypes.data_as(dp), h_mu.ctypes.data_as(dp), pnp.PREC[variants[0]])
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = lib.pnp_excess_mu(P.h, h_rho.ctypes.data_as(dp), h_mu.ctypes.data_as(dp), pnp.PREC[variants[0]])
        if r != 0:
            raise RuntimeError(f"pnp_excess_mu {r}")
    e2e_ms = reduce_max(world, (time.perf_counter() - t0) / args.steps * 1e3)
    barrier(world)

    # roofline of the dominant FP64 kernel and of the FP32 variant's
    peak, peak_kind = measured_peaks()
    dims = (spec.nx, spec.ny, spec.nz) + tuple(info["fft_len"])

    def roof(prec):
        st = results[prec]["stages"]
        cs = 8 if prec in ("fp32", "tf32split") else 16
        name = max(st, key=lambda k: st[k][0])
        tot, n = st[name]
        avg = tot / max(n, 1)
        share = tot / sum(v[0] for v in st.values())
        b = stage_bytes(name, dims, cs, SPECIES)
        f = stage_flops(name, dims, SPECIES)
        hbm = {"achieved_gbs": b / (avg * 1e-3) / 1e9, "bytes_per_launch": b}
        hbm["frac"] = hbm["achieved_gbs"] / peak
        if prec == "df64":
            # FP32-pipe instructions the double-float kernel executes (ncu
            # count) per second against the pipes' issue rate; without a count
            # for the current kernel no fraction is claimed
            ni = PROFILED_FP32_INST.get((prec, name))
            ach = ni / (avg * 1e-3) / 1e12 if ni else None
            return {"kernel": name, "bound": "alu", "achieved": ach, "peak": FP32_PEAK_TINST,
                    "unit": "T FP32-pipe instructions/s (FADD+FMUL+FFMA of the double-float arithmetic)",
                    "frac": ach / FP32_PEAK_TINST if ach else None,
                    "traffic": PROFILED_TRAFFIC.get((prec, name)), "fp32_inst_per_launch": ni,
                    "fp64_equivalent_flops_per_launch": f, "fp64_equivalent_tflops": f / (avg * 1e-3) / 1e12,
                    "avg_launch_ms": avg, "share_of_step": share,
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz, one instruction per lane "
                                   "per clock", "hbm": hbm}
        if prec == "fp64":
            ach = f / (avg * 1e-3) / 1e12
            return {"kernel": name, "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": ach / FP64_PEAK_TFLOPS, "traffic": PROFILED_TRAFFIC.get((prec, name)), "flops_per_launch": f,
                    "avg_launch_ms": avg, "share_of_step": share,
                    "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2.07 GHz", "hbm": hbm}
        ach = b / (avg * 1e-3) / 1e9
        return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "traffic": PROFILED_TRAFFIC.get((prec, name)), "bytes_per_launch": b, "avg_launch_ms": avg,
                "share_of_step": share, "peak_source": peak_kind,
                "fp32_tflops": f / (avg * 1e-3) / 1e12}

    def path_roof(prec):
        # the whole step against the copy bandwidth: this design's algorithmic
        # bytes, and the unfused pass model of the same transforms
        sec = results[prec]["ms"] * 1e-3
        wide = prec in ("fp64", "df64")
        b = path_bytes(dims, 16 if wide else 8, SPECIES)
        m = pass_model_bytes(dims, SPECIES, 8 if wide else 4)
        return {"bound": "hbm", "peak": peak, "unit": "GB/s", "peak_source": peak_kind,
                "bytes_per_step": b, "achieved": b / sec / 1e9, "frac": b / sec / 1e9 / peak,
                "pass_model_bytes": m, "pass_model_gbs": m / sec / 1e9, "pass_model_frac": m / sec / 1e9 / peak}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        m = args.cpu_sample
        v, used, dt = oracle_mu_rate(spec, rho, m)
        m1 = max(8, m // 2)
        v1, _, dt1 = oracle_mu_rate(spec, rho, m1, threads=1)
        cpu = {"value": v, "unit": "Gpoints/s", "cores": used, "kind": "oracle", "cpu_model": cpu_model(),
               "sample": f"{m}^3 sub-box of the {N_EDGE}^3 workload (same radii and densities), one full mu_ex, "
                         f"{dt:.1f} s",
               "single_core": {"value": v1, "unit": "Gpoints/s", "cores": 1,
                               "sample": f"{m1}^3 sub-box, one full mu_ex, {dt1:.1f} s"}}

    if rank == 0:
        head = variants[0]
        vals = {p: world * npts / (results[p]["ms"] * 1e-3) / 1e9 for p in variants}
        launches = sum(n * kernels_per_stage(k, info["fft_len"][0]) for k, (_, n) in results[head]["stages"].items())
        line = {
            "metric": "mu_ex Gpoints/s", "value": vals[head], "unit": "Gpoints/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": results[head]["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[head],
            "data": "synthetic",
            "config": {"workload": f"mu_ex {args.n}^3 x {SPECIES} species (R 1.5/2/3 h, packing 0.1 each, "
                                   f"lognormal(0,0.1) seed 2), zero-padded {args.pad}^3",
                       "fft_len": list(info["fft_len"]), "parallelism": f"replicas x{world}",
                       "l2": "flushed before each step (256 MB write)"},
            "e2e": {"value": world * npts / (e2e_ms * 1e-3) / 1e9, "unit": "Gpoints/s",
                    "h2d_bytes_per_step": int(rho.nbytes), "d2h_bytes_per_step": int(rho.nbytes),
                    "ms_per_step": e2e_ms},
            "roofline": roof(head),
            "path_roofline": path_roof(head),
            "max_rel_err_vs_fp64": errs.get(head), "error_bound_vs_oracle": ERROR_BOUND[head],
            "cpu_baseline": cpu,
            "gpu_launches": launches,
            "clocks": clocks,
            "variants": {VARIANT_NAME[p]: {
                "value": vals[p], "unit": "Gpoints/s", "ms_per_step": results[p]["ms"],
                "dtype": DTYPE[p], "roofline": roof(p), "path_roofline": path_roof(p),
                "max_rel_err_vs_fp64": errs.get(p),
                "error_bound_vs_oracle": ERROR_BOUND[p]}
                for p in variants[1:]},
            "stages_ms": {p: {k: v[0] / max(v[1], 1) for k, v in results[p]["stages"].items()}
                          for p in results},
        }
    P.close()
    torch.cuda.synchronize()
    if rank == 0 and args.solves > 0:
        from workloads import batch_specs
        line["solves"] = batch_record(batch_specs(args.solves), args.solve_prec, args.autotune, args.solves,
                                      aa=args.solve_aa, policy=args.policy, slots=args.slots)
    barrier(world)
    if rank == 0:
        print(json.dumps(line), flush=True)


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the
    architecture), for the CPU baselines' records."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name:"):
                return line.split(":", 1)[1].strip() + f" ({os.uname().machine})"
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip() + f" ({os.uname().machine})"
    except OSError:
        pass
    return os.uname().machine


def _pct(v, q):
    import numpy as np
    return float(np.percentile(np.asarray(v), q)) if len(v) else None


def oracle_mu_rate(spec, rho, m, threads=None):
    """The CPU oracle's mu_ex rate (Gpoints/s) on an m^3 sub-box of the
    workload, with `threads` OpenMP threads (None: as configured).  Returns
    (rate, threads used, seconds)."""
    from oracle import oracle
    prev = oracle.num_threads()
    if threads is not None:
        oracle.set_num_threads(threads)
    try:
        s2, r2 = sub_box(spec, rho, m)
        t0 = time.perf_counter()
        oracle.excess_mu(s2, r2)
        dt = time.perf_counter() - t0
        used = oracle.num_threads()
    finally:
        oracle.set_num_threads(prev)
    return m ** 3 / dt / 1e9, used, dt


def oracle_sweep_seconds(spec, sweeps):
    """Mean wall time of one relaxed Gummel sweep of the CPU oracle on `spec`,
    over its first `sweeps` sweeps from the default start (the oracle as it
    stands, all host cores).  Returns (seconds per sweep, threads)."""
    import dataclasses
    from oracle import oracle
    s = dataclasses.replace(spec, max_iter=sweeps, tol=0.0)
    t0 = time.perf_counter()
    oracle.gummel(s)
    return (time.perf_counter() - t0) / sweeps, oracle.num_threads()


def served_variant(spec, autotune, aa):
    """The served form of a request: autotuned plan and, with aa > 0, the
    relaxed iteration accelerated by Anderson mixing of depth aa on the
    step-limited geometric relaxation (same fixed point as the recipe's)."""
    s = dataclasses.replace(spec, autotune=autotune)
    if aa > 0:
        s = dataclasses.replace(s, anderson=aa, rho_mix=2)
    return s


def batch_record(specs, solve_prec, autotune, seq_count, aa=0, policy="fifo", slots=64, log=sys.stderr):
    """Independent Gummel solves of the batch recipe served concurrently
    (mu_ex in `solve_prec`, FP64 Gummel update and linear solves, Anderson
    depth `aa`, admission `policy`) against the first `seq_count` of the same
    solves one at a time in plain FP64 with the recipe's relaxation.
    Latency of a served solve = submission (all at t = 0) to poll-ready."""
    import numpy as np
    from paper_1407_0674_gb300 import pnp
    served = [served_variant(s, autotune, aa) for s in specs]
    seq = []
    seq_res = {}
    for k, s in enumerate(specs[:seq_count]):
        with pnp.Problem(s) as P:
            t0 = time.perf_counter()
            phi, rho, st = P.gummel_solve(raise_on_error=False)
            seq.append(time.perf_counter() - t0)
            seq_res[k] = (rho, st)
        print(f"sequential fp64 {k} ({s.nx}x{s.ny}x{s.nz}): status {st['status']} it {st['iterations']} "
              f"{seq[-1]:.1f} s", file=log, flush=True)
    srv = pnp.Server(max_slots=slots, policy=policy)
    t0 = time.perf_counter()
    tickets = []
    for s in served:
        rc, t = srv.submit(s, precision=solve_prec)
        if rc != 0:
            raise RuntimeError(f"submit {rc}")
        tickets.append(t)
    done = {}
    while len(done) < len(tickets):
        for k, t in enumerate(tickets):
            if k in done:
                continue
            rc, phi, rho, st = srv.poll(t)
            if rc != pnp.PENDING:
                done[k] = (rc, rho, st, time.perf_counter() - t0)
                print(f"served {k}: status {rc} it {st['iterations']} at {done[k][3]:.1f} s", file=log, flush=True)
        time.sleep(0.002)
    wall = time.perf_counter() - t0
    srv.close()
    # solves that converged in both runs
    both = [k for k in seq_res if seq_res[k][1]["status"] == 0 and done[k][0] == 0]
    errs = [max(float(np.abs(done[k][1][i] - seq_res[k][0][i]).max() / np.abs(seq_res[k][0][i]).max())
                for i in range(specs[k].s)) for k in both]
    lat = [v[3] for v in done.values()]
    # time from submission to the start of the solve (admission and problem
    # creation) = latency - the solve's own seconds
    adm = [v[3] - v[2]["seconds"] for v in done.values()]
    grids = sorted({(s.nx, s.ny, s.nz) for s in specs})
    return {
        "workload": f"{len(specs)} independent Gummel solves of the batch recipe (seed 4): grids "
                    + ", ".join(f"{a}x{b}x{c}" for a, b, c in grids)
                    + ", T U(250,400) K, wells 0.3 eV/kT, packing U(0.1,0.35), residual 1e-8; served "
                      "concurrently (one CUDA graph per solve) vs one at a time in plain FP64",
        "mu_ex_precision": solve_prec,
        "served_solver": (f"Anderson depth {aa} on the step-limited geometric relaxation (0.05)" if aa > 0 else
                          "the recipe's relaxation") + f", policy {policy}, {slots} slots",
        "sequential_solver": "the recipe's relaxation (per-point adaptive, 0.05), plain FP64 mu_ex",
        "served": {"solves": len(specs), "solves_per_s": len(specs) / wall, "wall_s": wall,
                   "latency_p50_s": _pct(lat, 50), "latency_p99_s": _pct(lat, 99),
                   "admission_mean_s": float(np.mean(adm)), "admission_max_s": float(np.max(adm)),
                   "solve_mean_s": float(np.mean([v[2]["seconds"] for v in done.values()])),
                   "converged": sum(1 for v in done.values() if v[0] == 0),
                   "status": [done[k][0] for k in range(len(specs))],
                   "iterations": [done[k][2]["iterations"] for k in range(len(specs))],
                   "repeated_sweeps": [done[k][2].get("repeated_sweeps", 0) for k in range(len(specs))]},
        "sequential_fp64": {"solves": len(seq), "solves_per_s": len(seq) / sum(seq) if seq else None,
                            "wall_s": sum(seq), "converged": sum(1 for k in seq_res if seq_res[k][1]["status"] == 0),
                            "iterations": [seq_res[k][1]["iterations"] for k in seq_res]},
        "speedup_vs_sequential_fp64": (len(specs) / wall) / (len(seq) / sum(seq)) if seq else None,
        "max_rel_err_rho_vs_fp64": max(errs) if errs else None, "compared_solves": len(both),
        "error_bar": 1e-6,
    }


def run_solves(args, world, rank, local):
    """Gummel workloads: film (one solve), batch (many solves through the
    server against the same solves one at a time), serve (Poisson arrivals)."""
    import numpy as np
    import torch
    from paper_1407_0674_gb300 import build as lb
    from paper_1407_0674_gb300 import pnp
    from workloads import batch_specs, film3, film_gummel, serving_arrivals, serving_spec

    torch.cuda.set_device(local)
    lb.build()
    if args.workload == "film":
        spec = film_gummel(32, 32, 32)
        with pnp.Problem(spec) as P:
            P.gummel_solve()                       # builds the solve graph
            t0 = time.perf_counter()
            phi, rho, st = P.gummel_solve()
            dt = time.perf_counter() - t0
        line = {"metric": "PNP solves/s", "value": world / dt, "unit": "solves/s", "n_gpus": world, "steps": 1,
                "warmup": 1, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "Gummel solve of the 32^3 film (2 ions, R 2h, packing 0.2 each, wells 1 kT on "
                                       "64 sites, bias 0.1 kT/e) to residual 1e-8"},
                "iterations": st["iterations"], "linear_iterations": st["linear_iterations"],
                "residual": st["residual"]}
        # where an iteration's device time goes (the solve graph's phase marks)
        sp = dataclasses.replace(spec, phase_timing=True)
        with pnp.Problem(sp) as P:
            P.gummel_solve()
            _, _, stp = P.gummel_solve()
            ph = P.gummel_phase_times()
        line["phases_ms_per_iteration"] = {k: v / max(stp["iterations"], 1) for k, v in ph.items()}
        if args.film_aa > 0:
            # the same solve with Anderson mixing (same fixed point)
            sa = dataclasses.replace(spec, anderson=args.film_aa)
            with pnp.Problem(sa) as P:
                P.gummel_solve()
                t0 = time.perf_counter()
                _, rho_a, sta = P.gummel_solve()
                dta = time.perf_counter() - t0
            line["anderson"] = {"depth": args.film_aa, "solves_per_s": world / dta, "ms_per_solve": dta * 1e3,
                                "iterations": sta["iterations"],
                                "max_rel_err_rho_vs_plain": max(float(np.abs(rho_a[i] - rho[i]).max() /
                                                                      np.abs(rho[i]).max()) for i in range(2))}
        if rank == 0 and not args.no_cpu_baseline:
            k = 2
            per, threads = oracle_sweep_seconds(spec, k)
            est = per * st["iterations"]
            line["cpu_baseline"] = {"value": 1.0 / est, "unit": "solves/s", "cores": threads, "kind": "oracle",
                                    "cpu_model": cpu_model(),
                                    "sample": f"first {k} Gummel sweeps of the same film ({per * k:.1f} s), "
                                              f"extrapolated to the {st['iterations']} iterations of the GPU solve"}
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    if args.workload == "film3":
        # bias sweep on the 128x128x256 film: the first point from its
        # equilibrium (Sec 3.2), the others warm-started from the previous
        # point (or each from its equilibrium with --film3-start eq); plain
        # FP64 against the mixed-precision mu_ex
        biases = [k / max(1, args.bias_points - 1) for k in range(args.bias_points)]
        runs = {}
        for prec in ("fp64", args.solve_prec):
            phi0 = rho0 = None
            solve_s = wall_s = 0.0
            rec = []
            for b in biases:
                spec = film3(bias=b, max_iter=args.max_iter3)
                t0 = time.perf_counter()
                with pnp.Problem(spec, precision=prec) as P:
                    t1 = time.perf_counter()
                    phi, rho, st = P.gummel_solve(phi0, rho0, raise_on_error=False)
                    solve_s += time.perf_counter() - t1
                wall_s += time.perf_counter() - t0
                if args.film3_start == "warm" and st["status"] == 0:
                    phi0, rho0 = phi, rho
                rec.append((b, st, rho))
                print(f"film3 {prec} bias {b:.2f}: status {st['status']} init {st['init_iterations']} "
                      f"it {st['iterations']} {time.perf_counter() - t0:.1f} s", file=sys.stderr, flush=True)
            runs[prec] = (solve_s, wall_s, rec)
        s64, w64, r64 = runs["fp64"]
        sm, wm, rm = runs[args.solve_prec]
        errs = [max(float(np.abs(a[2][i] - c[2][i]).max() / np.abs(c[2][i]).max()) for i in range(3))
                for a, c in zip(rm, r64)]
        n = len(biases)
        line = {"metric": "PNP solves/s", "value": world * n / wm, "unit": "solves/s", "n_gpus": world,
                "steps": n, "warmup": 0, "ms_per_step": wm / n * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": DTYPE[args.solve_prec] + " / f64 Gummel", "data": "synthetic",
                "config": {"workload": f"film 128x128x256, 3 mobile species (R 2/2/1 h), wells 3 kT on 4096 "
                                       f"sites, bias sweep 0..1 kT/e in {n} points, "
                                       + ("each from its equilibrium" if args.film3_start == "eq" else
                                          "first from its equilibrium, then warm-started") + ", residual 1e-8",
                           "mu_ex_precision": args.solve_prec},
                "solve_seconds": sm, "fp64_plain": {"solves_per_s": n / w64, "wall_s": w64, "solve_seconds": s64,
                                                    "iterations": [r[1]["iterations"] for r in r64],
                                                    "init_iterations": [r[1]["init_iterations"] for r in r64],
                                                    "status": [r[1]["status"] for r in r64]},
                "speedup_vs_fp64": w64 / wm,
                "iterations": [r[1]["iterations"] for r in rm], "status": [r[1]["status"] for r in rm],
                "init_iterations": [r[1]["init_iterations"] for r in rm],
                "max_rel_err_rho_vs_fp64": max(errs)}
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    if args.workload == "batch":
        rec = batch_record(batch_specs(args.batch), args.solve_prec, args.autotune, args.seq, aa=args.solve_aa,
                           policy=args.policy, slots=args.slots)
        line = {"metric": "PNP solves/s", "value": world * rec["served"]["solves_per_s"], "unit": "solves/s",
                "n_gpus": world, "steps": 1, "warmup": 0, "ms_per_step": rec["served"]["wall_s"] * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": DTYPE[args.solve_prec] + " / f64 Gummel", "data": "synthetic",
                "config": {"workload": rec["workload"], "mu_ex_precision": args.solve_prec,
                           "autotune": bool(args.autotune)}}
        line.update({k: v for k, v in rec.items() if k != "workload"})
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    # serve
    arr = serving_arrivals(args.requests, rate=args.rate, hi=args.max_edge)
    specs = [serving_spec(n, bias, T) for (_, n, bias, T) in arr]
    served = [served_variant(s, args.autotune, args.solve_aa) for s in specs]
    seq = []
    for s in specs[:args.seq]:
        with pnp.Problem(s) as P:
            t0 = time.perf_counter()
            _, _, st = P.gummel_solve(raise_on_error=False)
            seq.append(time.perf_counter() - t0)
        print(f"serve sequential n {s.nx}: status {st['status']} it {st['iterations']} {seq[-1]:.1f} s",
              file=sys.stderr, flush=True)
    srv = pnp.Server(max_slots=args.slots, policy=args.policy)
    t0 = time.perf_counter()
    pending = {}
    lat = []
    nxt = 0
    statuses = []
    while nxt < len(arr) or pending:
        now = time.perf_counter() - t0
        while nxt < len(arr) and arr[nxt][0] <= now:
            rc, t = srv.submit(served[nxt], precision=args.solve_prec)
            if rc == 0:
                pending[t] = arr[nxt][0]
            else:
                statuses.append(rc)
            nxt += 1
        for t in list(pending):
            rc, phi, rho, st = srv.poll(t)
            if rc != pnp.PENDING:
                lat.append(time.perf_counter() - t0 - pending.pop(t))
                statuses.append(rc)
                print(f"serve: status {rc} it {st['iterations']} latency {lat[-1]:.1f} s", file=sys.stderr,
                      flush=True)
        time.sleep(0.002)
    wall = time.perf_counter() - t0
    srv.close()
    line = {"metric": "PNP solves/s", "value": world * len(lat) / wall, "unit": "solves/s", "n_gpus": world,
            "steps": 1, "warmup": 0, "ms_per_step": wall * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[args.solve_prec] + " / f64 Gummel", "data": "synthetic",
            "config": {"workload": f"{len(arr)} served Gummel solves (32^3-film physics), Poisson arrivals "
                                   f"{args.rate}/s, cubic grids log-uniform 32..{args.max_edge}, bias U(0,1), "
                                   "T U(250,400) K, budget 150 GB",
                       "mu_ex_precision": args.solve_prec, "autotune": bool(args.autotune)},
            "latency_p50_ms": _pct(lat, 50) * 1e3, "latency_p99_ms": _pct(lat, 99) * 1e3,
            "completed_ok": sum(1 for s in statuses if s == 0), "statuses": sorted(set(statuses)),
            "sequential_fp64": {"solves": len(seq), "mean_s": float(np.mean(seq)) if seq else None}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload != "mu_ex":
        run_solves(args, world, rank, local)
    else:
        run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
